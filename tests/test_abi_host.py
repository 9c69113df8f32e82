"""Host-side checks of libsim's C ABI (no GPU): the library loads, exports every
entry point include/sim.h declares, and its host planning reproduces the
constants the paper prints (Table params, Eq. cerjan_damp, App. E.3.2)."""
import ctypes
import json
import math
import os
import re

import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLD = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_constants.json")))


@pytest.fixture(scope="module")
def pkg():
    from paper_2605_30541_gb300 import build
    build.build()
    import paper_2605_30541_gb300 as p
    p.abi.load()
    return p


def declared_entry_points():
    src = open(os.path.join(ROOT, "include", "sim.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sim_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol(pkg):
    names = declared_entry_points()
    assert len(names) >= 11
    lib = ctypes.CDLL(pkg.abi.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(pkg.abi._PROTOS)


def _paper_desc(pkg, nt, k, nb=60):
    cfg = dict(ndim=2, nz=619, nx=1000, h=10.0, dt=1e-3, nt=nt, bc="sponge",
               nb=[0, nb, 0, 0, nb, nb], free_surface=1, snap_every=k, snap_begin=0, snap_end=nt)
    return pkg.make_desc(cfg, max_shots=64, max_rec=1000)


def test_saved_samples_match_table_params(pkg):
    tp = GOLD["table_params"]
    info = pkg.sim_plan(_paper_desc(pkg, tp["N_wavefield"], tp["k"]))
    assert info.nsnap == tp["nsaved_wavefield"]
    info = pkg.sim_plan(_paper_desc(pkg, tp["N_gather"], tp["k"]))
    assert info.nsnap == tp["nsaved_gather"]
    assert (info.nsnap, tp["nz"], tp["nx"]) == (tp["nsaved_gather"], 619, 1000)
    assert [64, info.nsnap, 1000] == tp["gather_cube_shape"]
    assert abs(tp["k"] * tp["dt_s"] - tp["dt_saved_s"]) < 1e-15
    # padded grid: 60-cell sponge left, right and bottom, free top
    assert (info.NZ, info.NX) == (619 + 60, 1000 + 120)


def test_nyquist_margins_of_table_bands():
    dts = GOLD["table_params"]["dt_saved_s"]
    assert abs(1 / (2 * dts) - GOLD["saved_nyquist_hz"]) < 0.05
    for b in GOLD["table_bands"]:
        assert abs(1 / (2 * b["fmax"] * dts) - b["nyquist_margin"]) < 0.006
    # the paper's k = floor(N / (2 fmax T)) gives 20 for the 25 Hz band, yet it uses 14
    assert math.floor(8001 / (2 * 25.0 * 8.0)) == 20


def test_sponge_damping_constant(pkg):
    info = pkg.sim_plan(_paper_desc(pkg, 5001, 14))
    cd = 1.5 * math.log(1 / GOLD["sponge"]["R"]) / GOLD["sponge"]["n_bl"]
    assert abs(info.c_damp[1] - cd) < 1e-15 and abs(info.c_damp[4] - cd) < 1e-15
    assert info.c_damp[0] == 0.0  # free top
    assert abs(20 * math.log10(GOLD["sponge"]["R"]) - GOLD["sponge"]["R_db"]) < 1e-9
    assert abs(GOLD["sponge"]["n_bl"] * GOLD["table_params"]["h_m"] / 1000 - GOLD["sponge"]["thickness_km"]) < 1e-12


def test_courant_bounds_and_cfl_rejection(pkg):
    d2 = _paper_desc(pkg, 100, 0)
    info = pkg.sim_plan(d2, 1500.0, 5000.0)
    s = 8 / 5 + 1 / 5 + 8 / 315 + 1 / 560
    assert abs(info.courant_limit - 1 / math.sqrt(2 * s)) < 1e-12
    assert abs(info.courant_limit - 0.5231) < 1e-4
    assert abs(info.courant_exact - 0.5546) < 1e-4
    assert abs(info.courant - 0.5) < 1e-12          # Table params: 5000 m/s, 10 m, 1 ms is stable in 2D
    # 3D at dt = 1 ms violates the bound; 0.8 ms passes
    c5 = dict(ndim=3, nz=619, ny=1000, nx=1000, h=10.0, dt=1e-3, nt=2000, bc="cpml",
              nb=[0, 30, 30, 30, 30, 30], free_surface=1)
    with pytest.raises(pkg.SimError) as e:
        pkg.sim_plan(pkg.make_desc(c5), 1500.0, 5000.0)
    assert e.value.code == pkg.abi.SIM_ERR_CFL
    c5["dt"] = 8e-4
    info3 = pkg.sim_plan(pkg.make_desc(c5), 1500.0, 5000.0)
    assert abs(info3.courant_limit - 0.4271) < 1e-4 and abs(info3.courant_exact - 0.4529) < 1e-4
    info3 = pkg.sim_plan(pkg.make_desc(c5, skip_cfl_check=True), 1500.0, 6000.0)
    assert info3.courant > info3.courant_limit


def test_dispersion_warning(pkg):
    # h <= v_min / (G f_max), G = 4 (App. E.3.1): 10 m passes for 1500 m/s at 25 Hz (15 m)
    d = _paper_desc(pkg, 100, 0)
    d.f_max = 25.0
    pkg.sim_plan(d, 1500.0, 5000.0)
    d.f_max = 40.0
    with pytest.warns(UserWarning):
        pkg.sim_plan(d, 1500.0, 5000.0)


@pytest.mark.parametrize("mutate", ["ndim", "fs_top", "fp16_f64", "order", "nt"])
def test_invalid_descriptions_are_rejected(pkg, mutate):
    d = _paper_desc(pkg, 100, 10)
    if mutate == "ndim":
        d.ndim = 4
    elif mutate == "fs_top":
        d.nb[0] = 5
    elif mutate == "fp16_f64":
        d.snap_fp16, d.precision = 1, 1
    elif mutate == "order":
        d.space_order = 4
    elif mutate == "nt":
        d.nt = 0
    with pytest.raises(pkg.SimError) as e:
        pkg.sim_plan(d)
    assert e.value.code in (pkg.abi.SIM_ERR_ARG, pkg.abi.SIM_ERR_UNSUPPORTED)
    assert pkg.sim_last_error(None)


def test_configs_respect_the_paper_geometry_rules():
    c2 = synth.config_c2(nt=10)
    assert c2["vel"].min() >= 1500.0 and c2["vel"].max() <= 5000.0
    assert c2["vel"].shape == (619, 1000)
    c3 = synth.config_c3(nt=10, nslices=2)
    xs = c3[0]["src"][:, 0]
    assert len(xs) == 64 and abs(xs[1] - xs[0] - 150.0) < 1e-9
