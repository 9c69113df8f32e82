"""The byte accounting behind bench.py's roofline fractions, checked against
an independent count: the CPML strip cells of every absorbing axis taken
from explicit masks of the padded grid, and the snapshot steps enumerated
one by one from the snapshot rule (n >= begin, n < end, (n - begin) % k == 0).
CPU only."""
import importlib.util
import os

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def independent_bytes(cfg, nshots):
    nb = cfg["nb"]
    three = cfg["ndim"] == 3
    NZ = nb[0] + cfg["nz"] + nb[1]
    NY = nb[2] + cfg["ny"] + nb[3] if three else 1
    NX = nb[4] + cfg["nx"] + nb[5]
    z, y, x = np.meshgrid(np.arange(NZ), np.arange(NY), np.arange(NX), indexing="ij")
    strips = 0
    if cfg.get("bc") == "cpml":
        masks = [(z < nb[0]) | (z >= NZ - nb[1]), (x < nb[4]) | (x >= NX - nb[5])]
        if three:
            masks.append((y < nb[2]) | (y >= NY - nb[3]))
        strips = sum(int(m.sum()) for m in masks)  # cells x axes
    nsnap = 0
    if cfg.get("snap_every", 0) > 0:
        k, b, e = cfg["snap_every"], cfg["snap_begin"], cfg["snap_end"]
        nsnap = sum(1 for n in range(cfg["nt"]) if b <= n < e and (n - b) % k == 0)
    interior = cfg["nz"] * (cfg["ny"] if three else 1) * cfg["nx"]
    per_shot = 16 * z.size + 16 * strips + 4 * len(cfg["rec"]) + 4 * interior * nsnap / cfg["nt"]
    return nshots * per_shot


def small_3d_cpml():
    c = synth.config_c5(nt=40, n=(20, 24, 28), nb=5, nrec_side=7)
    c["snap_every"], c["snap_begin"], c["snap_end"] = 7, 3, 33
    return c


@pytest.mark.parametrize("name", ["c1", "c2", "c2_sponge", "c3_slice", "c5_small", "c6_gather"])
def test_algorithmic_bytes_match_an_independent_count(bench, name):
    cfg = {"c1": lambda: synth.config_c1(nt=50),
           "c2": lambda: synth.config_c2(nt=120),
           "c2_sponge": lambda: dict(synth.config_c2(nt=120), bc="sponge"),
           "c3_slice": lambda: synth.config_c3(nt=30, nslices=2)[2],
           "c5_small": small_3d_cpml,
           "c6_gather": lambda: synth.config_c6("gather", nt=60)}[name]()
    for nshots in (1, 3):
        got = bench.algorithmic_bytes_per_launch(cfg, nshots)
        want = independent_bytes(cfg, nshots)
        assert abs(got - want) <= 1e-9 * want, (name, nshots, got, want)


def test_padded_cells(bench):
    c = small_3d_cpml()
    nb = c["nb"]
    assert bench.padded_cells(c) == (nb[0] + 20 + nb[1]) * (nb[2] + 24 + nb[3]) * (nb[4] + 28 + nb[5])


@pytest.mark.parametrize("nt", [1, 2, 7, 8001])
def test_two_step_bytes_match_a_pass_by_pass_count(bench, nt):
    # the two-step row march moves, per pass, p^n, p^{n-1}, c in and p^{n+1},
    # p^{n+2} out (20 B per cell), or 16 B when the last pass has one step;
    # every step samples each receiver once (4 B)
    c = synth.config_c6("gather", nt=nt)
    shots = len(c["src"])
    nb = c["nb"]
    cells = (nb[0] + c["nz"] + nb[1]) * (nb[4] + c["nx"] + nb[5])
    total, n = 0, 0
    while n < nt:
        two = n + 1 < nt
        total += cells * (20 if two else 16)
        n += 2 if two else 1
    total = shots * (total + 4 * len(c["rec"]) * nt)
    assert bench.algorithmic_bytes_two_step(c, shots, nt) == total
