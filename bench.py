"""Benchmark of the acoustic FDTD hot path on GB300.

Default workload (one "step" = one full solve): the field-scale 3D volume —
619 x 1000 x 1000 cells at 10 m + 30-cell CPML on x, y and bottom, free
surface (1060 x 1060 x 649 = 729.2 M padded cells), seeded procedural
velocity, one Ricker source (8 Hz) at the surface centre, a 201 x 201
receiver grid, dt = 0.8 ms, nt = 2500 (the 2 s record at a stable step).
`--workload` selects the 2D slice (c2), 32 shots on it (c2x32), the batched
uneven slices (c3), the production runs (c6g, c6w) or the model builder.

Metric: cell-updates per second over the padded grid (Gcell/s). `value` is
device-timed (CUDA events on the solver's stream, inputs resident, L2 flushed
between timed solves); `e2e` repeats the solve through the C ABI with pinned
host buffers (model upload, gather and snapshot download inside the timing).
`gradient` times the adjoint-state gradient (2D: 16 shots of the 201 x 201
slice, FP16 vs FP32 checkpoints; 3D: one shot of the full volume with FP16
checkpoints). `--impl reference` times the FP64 CPU oracle on the host cores
instead, on a bounded sample of the same workload.
Under torchrun every rank runs an independent replica (the single-shot solve
does not shard); value = all ranks' cell-updates / max-over-ranks time.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gcell-updates/s (FP32 fwd, adjoint) vs HBM roofline; gradient s/shot at tol"
L2_FLUSH_BYTES = 512 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c5", choices=["c2", "c2x32", "c3", "c4g", "c5", "c5s", "c6g", "c6w", "model"])
    ap.add_argument("--nt", type=int, default=0, help="override nt (profiling runs only)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-grad", action="store_true")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def workload(args):
    import synth
    if args.workload == "c5":
        return synth.config_c5(nt=args.nt or 2500), 1
    if args.workload == "c5s":
        # reduced 3D volume for counter captures (about 1 GB on the device)
        return synth.config_c5(nt=args.nt or 200, n=(190, 400, 400), nrec_side=101), 1
    if args.workload == "c6w":
        return synth.config_c6("wavefield", nt=args.nt or None), 1
    nt = args.nt or 8000
    cfg = synth.config_c2(nt=nt)
    nshots = 32 if args.workload == "c2x32" else 1
    if nshots > 1:
        cfg["src"] = np.stack([500.0 + 280.0 * np.arange(nshots), np.full(nshots, 10.0)], axis=1)
        cfg.update(snap_every=0, snap_end=0)
    return cfg, nshots


PATH_STEP, PATH_RESIDENT, PATH_MARCH = 1, 2, 4  # sim_info.last_path


def padded_cells(cfg):
    nb = cfg["nb"]
    ny = (nb[2] + cfg["ny"] + nb[3]) if cfg["ndim"] == 3 else 1
    return (nb[0] + cfg["nz"] + nb[1]) * ny * (nb[4] + cfg["nx"] + nb[5])


def algorithmic_bytes_per_launch(cfg, nshots):
    """Bytes one step-kernel launch must move at minimum: 16 B per cell (read
    p^n, p^{n-1}, c; write p^{n+1}), 16 B per CPML strip cell and axis (psi,
    zeta read + write), 4 B per receiver sample, 4 B per interior cell at
    snapshot steps (averaged over the launches)."""
    nb = cfg["nb"]
    NZ = nb[0] + cfg["nz"] + nb[1]
    NY = nb[2] + cfg["ny"] + nb[3] if cfg["ndim"] == 3 else 1
    NX = nb[4] + cfg["nx"] + nb[5]
    cells = NZ * NY * NX
    strip = 0
    if cfg.get("bc") == "cpml":
        strip = (nb[4] + nb[5]) * NZ * NY + (nb[0] + nb[1]) * NX * NY
        if cfg["ndim"] == 3:
            strip += (nb[2] + nb[3]) * NZ * NX
    rec = len(cfg["rec"]) * 4
    nsnap = 0
    if cfg.get("snap_every", 0) > 0:
        end = min(cfg["snap_end"], cfg["nt"])
        nsnap = (end - cfg["snap_begin"] + cfg["snap_every"] - 1) // cfg["snap_every"]
    snap = nsnap * cfg["nz"] * cfg.get("ny", 1) * cfg["nx"] * 4 / cfg["nt"]
    return nshots * (16 * cells + 16 * strip + rec + snap)


def algorithmic_bytes_two_step(cfg, nshots, nt):
    """Bytes the two-step row march must move at minimum over nt steps: 20 B
    per cell and pass of two steps (read p^n, p^{n-1}, c; write p^{n+1},
    p^{n+2}), 16 B per cell in the last pass when nt is odd (one step), 4 B
    per receiver sample. Only batches without CPML or snapshots take it."""
    nb = cfg["nb"]
    cells = (nb[0] + cfg["nz"] + nb[1]) * (nb[4] + cfg["nx"] + nb[5])
    return nshots * (cells * (10 * (nt - nt % 2) + 16 * (nt % 2)) + 4 * len(cfg["rec"]) * nt)


def strip_cell_axes(cfg):
    """CPML strip cells counted once per absorbing axis whose strip holds them."""
    if cfg.get("bc") != "cpml":
        return 0
    nb = cfg["nb"]
    NZ = nb[0] + cfg["nz"] + nb[1]
    NY = nb[2] + cfg["ny"] + nb[3] if cfg["ndim"] == 3 else 1
    NX = nb[4] + cfg["nx"] + nb[5]
    s = (nb[4] + nb[5]) * NZ * NY + (nb[0] + nb[1]) * NX * NY
    if cfg["ndim"] == 3:
        s += (nb[2] + nb[3]) * NZ * NX
    return s


def gradient_bytes_per_shot(cfg, fp16, qbytes=None, levels=1):
    """Least DRAM bytes of one shot's adjoint-state gradient: per cell and
    step, the forward sweep 16 B (read p^n, p^{n-1}, c; write p^{n+1}), the
    recompute 16 B plus the imaging-term store, the adjoint sweep 16 B plus
    the imaging-term read and the gradient read + write (8 B); per CPML strip
    cell and axis and step, 16 B (psi, zeta read + write) in each forward-type
    sweep and 24 B in the adjoint (multipliers nu, mu read + write, the
    bracket written and read). Imaging terms are 2 B in FP16 storage, else
    4 B (qbytes overrides). A two-level checkpoint schedule adds one more
    forward sweep. Checkpoint traffic (a few states per segment) is not
    counted."""
    q = qbytes if qbytes is not None else (2 if fp16 else 4)
    cells = padded_cells(cfg)
    extra = 16 * (levels - 1)
    return cfg["nt"] * (cells * (16 + extra + 16 + q + 16 + q + 8) +
                        strip_cell_axes(cfg) * (16 + extra + 16 + 24))


def launches_per_solve(cfg, nsnap, path, x_folded=False):
    """Kernels of ours one solve launches: on the resident path one launch for
    the whole time loop; else the fused step kernel per step in 2D; in 3D the
    z-march plus, per step, receiver sampling, source injection and one CPML
    pass per absorbing axis (the bench volumes' strips are far apart and far
    from the free surface; none for x when the TMA march folds the x strips
    in), plus snapshot kernels; plus the final finite-value check."""
    if path == PATH_RESIDENT:
        return 2
    if cfg["ndim"] == 2:
        return cfg["nt"] + 1
    nb = cfg["nb"]
    axes = sum(1 for a in range(3) if nb[2 * a] + nb[2 * a + 1] > 0) if cfg.get("bc") == "cpml" else 0
    if x_folded and cfg.get("bc") == "cpml" and nb[4] + nb[5] > 0:
        axes -= 1
    return cfg["nt"] * (1 + axes + 2) + nsnap + 1


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def read_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def ncu_traffic(kernel_file, key):
    """DRAM bytes per launch recorded by the committed ncu summary for `key`,
    valid only while the kernel source is unchanged (sha1 recorded beside it)."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    src = os.path.join(ROOT, "paper_2605_30541_gb300", "csrc", kernel_file)
    try:
        sha = hashlib.sha1(open(src, "rb").read()).hexdigest()
        for ln in open(path):
            f = ln.split()
            if len(f) >= 3 and f[0] == key and f[1] == sha:
                return float(f[2])
    except OSError:
        pass
    return None


def oracle_sample(cfg):
    """The problem the FP64 oracle times as a bounded sample of the workload.
    2D: the workload itself (its first steps). 3D: the volume's top corner
    block of 100 x 200 x 200 interior cells (the same velocities) with its
    -x and -y CPML faces and the free top, a source at the block's surface
    centre and the receivers of the grid that fall in the block."""
    if cfg["ndim"] == 2:
        return cfg, cfg["src"][0], cfg["rec"], "the same slice solve"
    nz, ny, nx = 100, 200, 200
    h = cfg["h"]
    nb = cfg["nb"]
    samp = dict(cfg, nz=nz, ny=ny, nx=nx, nb=[0, 0, nb[2], 0, nb[4], 0], cpml_vmax=float(cfg["vel"].max()),
                vel=np.ascontiguousarray(cfg["vel"][:nz, :ny, :nx]))
    rec = cfg["rec"]
    keep = (rec[:, 0] <= (nx - 1) * h) & (rec[:, 1] <= (ny - 1) * h) & (rec[:, 2] <= (nz - 1) * h)
    return samp, np.array([nx // 2 * h, ny // 2 * h, h]), rec[keep], \
        "the volume's top corner block (100 x 200 x 200 cells + its -x, -y CPML, free top)"


def cpu_oracle_rate(cfg, target_s=12.0):
    """FP64 oracle throughput on a bounded sample of the workload (the first
    steps of the sample problem), sized to about target_s seconds of CPU work."""
    import oracle
    oracle.build()
    samp, src, rec, what = oracle_sample(cfg)
    cells = padded_cells(samp)
    v64 = samp["vel"].astype(np.float64)
    w64 = samp["wavelet"].astype(np.float64)
    probe = dict(samp, nt=20, snap_every=0, snap_end=0)
    t0 = time.perf_counter()
    oracle.forward(probe, v64, w64[:20], src=src, rec=rec)
    rate = 20 * cells / (time.perf_counter() - t0)
    nt = int(max(20, min(samp["nt"], target_s * rate / cells)))
    run = dict(samp, nt=nt, snap_end=min(samp.get("snap_end", 0), nt))
    t0 = time.perf_counter()
    oracle.forward(run, v64, w64[:nt], src=src, rec=rec, snaps=run.get("snap_every", 0) > 0)
    dt = time.perf_counter() - t0
    return {"value": nt * cells / dt / 1e9, "unit": "Gcell/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": "first %d of %d steps of %s (FP64, OpenMP over rows), %.1f s" % (nt, cfg["nt"], what, dt)}


def workload_name(args, cfg, nshots, nsnap):
    nt, nrec = cfg["nt"], len(cfg["rec"])
    if cfg["ndim"] == 3:
        return ("%s: 3D volume %dx%dx%d (+30-cell CPML on x, y, bottom, free top), dt=0.8 ms, nt=%d, "
                "%d receivers, %d shot(s) per GPU" % (args.workload, cfg["nz"], cfg["ny"], cfg["nx"], nt, nrec, nshots))
    if args.workload == "c6w":
        return ("c6w: production wavefield, 2D slice 619x1000 (+60-cell sponge left/right/bottom, free top), "
                "band-passed 3-6 Hz source, nt=%d, %d FP32 snapshots (every 14 steps)" % (nt, nsnap))
    return ("c2: 2D slice 619x1000 (+50-cell CPML left/right/bottom, free top), nt=%d, %d receivers, "
            "%d FP32 snapshots, %d shot(s) per GPU" % (nt, nrec, nsnap, nshots))


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    cfg, nshots = workload(args)
    import oracle
    oracle.build()
    samp, src, rec, what = oracle_sample(cfg)
    cells = padded_cells(samp)
    v64 = samp["vel"].astype(np.float64)
    w64 = samp["wavelet"].astype(np.float64)
    probe = dict(samp, nt=20, snap_every=0, snap_end=0)
    t0 = time.perf_counter()
    oracle.forward(probe, v64, w64[:20], src=src, rec=rec)
    rate = 20 * cells / (time.perf_counter() - t0)
    budget = 150.0 / max(1, args.steps + args.warmup)   # whole run within a few minutes
    nt = int(max(20, min(samp["nt"], budget * rate / cells)))
    run = dict(samp, nt=nt, snap_end=min(samp.get("snap_end", 0), nt))
    times = []
    for it in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.forward(run, v64, w64[:nt], src=src, rec=rec, snaps=run.get("snap_every", 0) > 0)
        if it >= args.warmup:
            times.append(time.perf_counter() - t0)
    per = statistics.mean(times)
    value = nt * cells / per / 1e9
    sample = "first %d of %d steps of %s per step" % (nt, cfg["nt"], what)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Gcell/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args, cfg, nshots, 0) + " (bounded sample: %s)" % sample,
                       "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": "Gcell/s", "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "Gcell/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_batch(args):
    """Batched workloads in one sim_batch: every (slice, shot) of the 17-slice
    set (c3), or the paper's production shot-gather run (c6g: 64 shots, 8 s,
    band-passed wavelet from the library's band-pass kernel)."""
    import torch
    import synth
    import paper_2605_30541_gb300 as pkg
    torch.cuda.set_device(0)
    if args.workload == "c6g":
        c6 = synth.config_c6("gather", nt=args.nt or None)
        lo, hi, f0 = c6["band"]
        c6["wavelet"] = pkg.bandpass_ricker(c6["nt"], c6["dt"], f0, lo, hi).cpu().numpy()
        slices = [c6]
        nt = c6["nt"]
    else:
        nt = args.nt or 4000
        slices = synth.config_c3(nt=nt)
    sims = [pkg.Simulator(c, c["vel"], max_shots=len(c["src"]), max_rec=len(c["rec"])) for c in slices]
    cells = sum(padded_cells(c) * len(c["src"]) for c in slices)
    gathers = [torch.empty((len(c["src"]), nt, len(c["rec"])), dtype=torch.float32, device="cuda") for c in slices]
    entries = [dict(sim=s, wavelet=torch.as_tensor(c["wavelet"], device="cuda"), src=c["src"], rec=c["rec"],
                    gather=g) for s, c, g in zip(sims, slices, gathers)]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        pkg.batch(entries)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with Clocks(0) as clk:
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            pkg.batch(entries)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
    total = sum(a.elapsed_time(b) for a, b in ev) / 1e3
    value = args.steps * nt * cells / total / 1e9
    peak, peak_kind = read_peaks()
    inf = pkg.sim_get_info(sims[0].handle)
    sched = {1: "march", 2: "march2", 3: "stepped", 4: "persistent"}.get(inf.batch_sched, "march")
    if sched == "march2":
        algo = sum(algorithmic_bytes_two_step(c, len(c["src"]), nt) for c in slices)
    else:
        algo = sum(algorithmic_bytes_per_launch(c, len(c["src"])) for c in slices) * nt
    # a batch with CPML runs its CPML and plain row-march items as two kernels per step
    split = sched == "march" and any(c.get("bc") == "cpml" for c in slices) and \
        os.environ.get("GSIM_MARCH_SPLIT", "1") != "0"
    per_step = 2 if split else 1
    kfile, kname, kkey = (("fwd2d_f32.cu", "k_multi2d", "multi_") if sched == "stepped" else
                          ("fwd2d_f32.cu", "k_batch2d", "batch_") if sched == "persistent" else
                          ("march2x.cu", "k_march2x", "march2_") if sched == "march2" else
                          ("march2d.cu", "k_march2d", "march_"))
    line = {"metric": METRIC, "value": value, "unit": "Gcell/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": ("c6g: production shot gathers, 64 shots on a 619x1000 slice (+60-cell sponge, "
                                    "free top), band 3-6 Hz, nt=%d, 1000 receivers, saved every 14 steps" % nt)
                                   if args.workload == "c6g" else
                                   ("c3: 64 shots on a 619x1000 slice + 16 uneven slices x 8 shots, nt=%d, "
                                    "one launch per step over all slices and shots (%s batch)" % (nt, sched)),
                       "seconds_per_slice_band": total / args.steps if args.workload == "c6g" else None,
                       "batch_schedule": sched + ("" if sched in ("march", "march2") else " tile %d" % inf.batch_tile),
                       "padded_cells_x_shots": cells,
                       "l2": "flushed between timed solves"},
            "roofline": {"bound": "hbm", "achieved": algo / (total / args.steps) / 1e9, "peak": peak,
                         "unit": "GB/s", "frac": algo / (total / args.steps) / 1e9 / peak,
                         "traffic": ncu_traffic(kfile, kkey + args.workload),
                         "traffic_per": "pass launch (two steps)" if sched == "march2" else
                         ("step (its two launches)" if split else "step launch"),
                         "kernel": kname, "peak_kind": peak_kind,
                         "algorithmic_bytes_per_solve": algo},
            "clocks": clk.summary(),
            "gpu_launches": args.steps * (2 * ((nt + 1) // 2) if sched == "march2" else per_step * nt)}
    print(json.dumps(line), flush=True)
    for s in sims:
        s.close()


def gradient_timing(reps=2):
    """FWI gradient workload (201 x 201 procedural model, 16 shots, 4 s): seconds
    per shot of (a) all 16 shots in one sim_adjoint with FP16-scaled checkpoints
    and imaging terms and (b) one shot per call with FP32 storage, plus their
    relative difference (the tests bound them against the FP64 oracle gradient:
    FP32 <= 1e-4, FP16 <= 1e-2 relative L2)."""
    import torch
    import synth
    import paper_2605_30541_gb300 as pkg
    c = synth.config_c4()
    ns, nt, nrec = len(c["src"]), c["nt"], len(c["rec"])
    true = pkg.Simulator(c, c["vel_true"], max_shots=ns, max_rec=nrec)
    d = true.forward(c["wavelet"], c["src"], c["rec"])["gather"].contiguous()
    true.close()
    sim = pkg.Simulator(c, c["vel"], max_shots=ns, max_rec=nrec)
    w = torch.as_tensor(c["wavelet"], device="cuda")
    src, rec = np.ascontiguousarray(c["src"]), np.ascontiguousarray(c["rec"])

    def batched():
        g = torch.zeros(c["vel"].shape, device="cuda")
        pkg.sim_adjoint(sim.handle, ns, w, src, nrec, rec, d, None, None, 1, g)
        return g

    def one_by_one():
        g = torch.zeros(c["vel"].shape, device="cuda")
        for k in range(ns):
            pkg.sim_adjoint(sim.handle, 1, w, np.ascontiguousarray(src[k:k + 1]), nrec, rec, d[k:k + 1].contiguous(),
                            None, None, 0, g)
        return g

    out = {}
    for name, fn in (("batched_fp16", batched), ("one_shot_fp32", one_by_one)):
        g = fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            g = fn()
        e1.record()
        torch.cuda.synchronize()
        out[name] = (e0.elapsed_time(e1) / 1e3 / reps / ns, g)
    sim.close()
    g16, g32 = out["batched_fp16"][1], out["one_shot_fp32"][1]
    peak, peak_kind = read_peaks()
    t16 = out["batched_fp16"][0]
    ach = gradient_bytes_per_shot(c, True) / t16 / 1e9
    return {"workload": "c4: 201x201 + 20-cell CPML on every side, 16 shots, nt=4000, sqrt(nt) checkpoints",
            "s_per_shot_batched_fp16": t16, "s_per_shot_one_shot_fp32": out["one_shot_fp32"][0],
            "speedup": out["one_shot_fp32"][0] / t16,
            "rel_l2_fp16_vs_fp32": float(torch.linalg.norm(g16 - g32) / torch.linalg.norm(g32)),
            "tolerance_vs_fp64_oracle": {"fp32": 1e-4, "fp16": 1e-2},
            "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                         "peak_kind": peak_kind, "case": "batched FP16 gradient, whole call per shot",
                         "algorithmic_bytes_per_shot": gradient_bytes_per_shot(c, True),
                         "note": "16 shots of 58,081 cells: fields L2-resident, imaging terms and checkpoints "
                                 "(~350 MB) are not; an effective rate on algorithmic bytes"}}


def gradient3d_timing(pkg, sim, cfg, wav_d, src, rec, dev):
    """The 3D volume's gradient: one shot, sim_adjoint with FP16 checkpoints
    on the same handle (d_obs = 0, so the residual is the gather), timed on
    its second call (the first plans and allocates the buffers and captures
    the graph). The checkpoint schedule is the one the device-memory budget
    allows; FP32 checkpoints are then tried and reported (on the full volume
    they do not fit)."""
    import torch
    nt, nrec = cfg["nt"], len(rec)
    d = torch.zeros((1, nt, nrec), device=dev)
    grad = torch.zeros((cfg["nz"], cfg["ny"], cfg["nx"]), device=dev)
    mis = np.zeros(1)

    def call(fp16):
        pkg.sim_adjoint(sim.handle, 1, wav_d, src, nrec, rec, d, None, mis, fp16, grad)

    t0 = time.perf_counter()
    call(1)
    torch.cuda.synchronize()
    first = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    call(1)
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    info = pkg.sim_get_info(sim.handle)
    peak, peak_kind = read_peaks()
    algo = gradient_bytes_per_shot(cfg, True, qbytes=4, levels=info.adj_levels)
    out = {"workload": "3D volume (the forward workload), 1 shot, nt=%d, FP16 checkpoints (FP32 imaging terms)" % nt,
           "s_per_shot_3d": t, "first_call_s": first, "misfit": float(mis[0]),
           "checkpoints": {"levels": info.adj_levels, "imaging_slots": info.adj_slots,
                           "inner_segments": info.adj_inner, "top_checkpoints": info.adj_top,
                           "inner_checkpoint_slots": info.adj_sub},
           "adjoint_bytes": info.adj_bytes, "handle_device_bytes": info.device_bytes,
           "roofline": {"bound": "hbm", "achieved": algo / t / 1e9, "peak": peak, "unit": "GB/s",
                        "frac": algo / t / 1e9 / peak, "peak_kind": peak_kind,
                        "algorithmic_bytes_per_shot": algo}}
    try:
        call(0)
        torch.cuda.synchronize()
        out["fp32_checkpoints"] = "fit: %d level(s)" % pkg.sim_get_info(sim.handle).adj_levels
    except pkg.SimError as e:
        out["fp32_checkpoints"] = "do not fit: " + str(e)
    return out


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2605_30541_gb300 as pkg

    cfg, nshots = workload(args)
    if "band" in cfg:  # the production runs' band-passed wavelet, made by the library
        lo, hi, f0 = cfg["band"]
        cfg["wavelet"] = pkg.bandpass_ricker(cfg["nt"], cfg["dt"], f0, lo, hi).cpu().numpy()
    nt = cfg["nt"]
    cells = padded_cells(cfg)
    rec = np.ascontiguousarray(cfg["rec"])
    src = np.ascontiguousarray(cfg["src"][:nshots])
    stream = torch.cuda.current_stream()
    sim = pkg.Simulator(cfg, cfg["vel"], max_shots=nshots, max_rec=len(rec), stream=stream)
    nsnap = sim.info.nsnap
    dev = torch.device("cuda", local)
    vel_d = torch.as_tensor(cfg["vel"], device=dev)
    wav_d = torch.as_tensor(cfg["wavelet"], device=dev)
    gather_d = torch.empty((nshots, nt, len(rec)), dtype=torch.float32, device=dev)
    ishape = (cfg["nz"], cfg["ny"], cfg["nx"]) if cfg["ndim"] == 3 else (cfg["nz"], cfg["nx"])
    snaps_d = torch.empty((nshots, nsnap) + ishape, dtype=torch.float32, device=dev) if nsnap else None
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def solve():
        pkg.sim_forward(sim.handle, nshots, wav_d, src, len(rec), rec, gather_d, snaps_d, None)

    for _ in range(args.warmup):
        solve()
    torch.cuda.synchronize()
    sim.sync()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with Clocks(local) as clk:
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            solve()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
    sim.sync()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total = sum(step_ms) / 1e3
    t = torch.tensor([total], dtype=torch.float64, device=dev)
    if dist:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.barrier()
    tmax = float(t.item())
    units = world * args.steps * nshots * nt * cells
    value = units / tmax / 1e9

    # roofline of the dominant kernel: the per-step kernel runs nt launches per
    # solve (gaps included in the duration); the resident kernel runs the whole
    # time loop in one launch
    path = pkg.sim_get_info(sim.handle).last_path
    launches = 1 if path == PATH_RESIDENT else nt
    per_launch_s = (total / args.steps) / launches
    algo = algorithmic_bytes_per_launch(cfg, nshots) * (nt if path == PATH_RESIDENT else 1)
    peak, peak_kind = read_peaks()
    achieved = algo / per_launch_s / 1e9
    pname = {PATH_RESIDENT: "resident", PATH_MARCH: "march"}.get(path, "step")
    key = "%s_%s" % (pname, args.workload)
    kfile, kname = (("fwd3d.cu", "k_step3d") if cfg["ndim"] == 3 else
                    ("resident2d.cu", "k_resident2d") if path == PATH_RESIDENT else
                    ("march2d.cu", "k_march2d") if path == PATH_MARCH else ("fwd2d_f32.cu", "k_step2d_f32"))
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": ncu_traffic(kfile, key), "kernel": kname,
            "peak_kind": peak_kind + " (MEASURED_PEAKS hbm_gbs)" if peak_kind == "measured" else peak_kind,
            "algorithmic_bytes_per_launch": algo, "avg_launch_us": per_launch_s * 1e6,
            "path": {PATH_RESIDENT: "resident", PATH_MARCH: "row march, one launch per step"}.get(path, "per-step")}
    if cfg["ndim"] == 3:
        inf = pkg.sim_get_info(sim.handle)
        roof["z_march"] = {"staging": {1: "cp.async", 2: "TMA, x strips folded in", 3: "TMA",
                                       4: "TMA, plane loop not unrolled",
                                       5: "TMA, x strips folded in, plane loop not unrolled",
                                       6: "TMA, plane loop unrolled by 3"}.get(
            inf.z_variant, inf.z_variant), "planes_per_cta": inf.z_chunk}
        if inf.z_variant in (2, 3, 4, 5, 6):
            roof["kernel"] = "k_step3d_tma"
            roof["traffic"] = ncu_traffic(kfile, "tma_" + args.workload)

    # end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        vel_h = torch.as_tensor(cfg["vel"]).pin_memory()
        wav_h = torch.as_tensor(cfg["wavelet"]).pin_memory()
        gather_h = torch.empty((nshots, nt, len(rec)), dtype=torch.float32).pin_memory()
        snaps_h = torch.empty((nshots, nsnap) + ishape, dtype=torch.float32).pin_memory() if nsnap else None
        for _ in range(max(1, min(2, args.warmup))):
            pkg.sim_set_model(sim.handle, vel_h)
            pkg.sim_forward(sim.handle, nshots, wav_h, src, len(rec), rec, gather_h, snaps_h, None)
        # long solves (the 3D volume: seconds each) repeat a few times only
        ke = args.steps if total / args.steps < 2.0 else max(1, min(args.steps, 3))
        et = []
        for _ in range(ke):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            pkg.sim_set_model(sim.handle, vel_h)
            pkg.sim_forward(sim.handle, nshots, wav_h, src, len(rec), rec, gather_h, snaps_h, None)
            torch.cuda.synchronize()
            et.append(time.perf_counter() - t0)
        te = torch.tensor([sum(et)], dtype=torch.float64, device=dev)
        if dist:
            dist.all_reduce(te, op=dist.ReduceOp.MAX)
        h2d = vel_h.numel() * 4 + wav_h.numel() * 4
        d2h = gather_h.numel() * 4 + (snaps_h.numel() * 4 if snaps_h is not None else 0)
        e2e = {"value": world * ke * nshots * nt * cells / float(te.item()) / 1e9, "unit": "Gcell/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "ms_per_step": float(te.item()) / ke * 1e3, "steps": ke}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_oracle_rate(cfg)
    grad = None
    if rank == 0 and not args.no_grad:
        grad = gradient_timing()
        if cfg["ndim"] == 3:
            grad["volume"] = gradient3d_timing(pkg, sim, cfg, wav_d, src, rec, dev)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "Gcell/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": tmax / args.steps * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": workload_name(args, cfg, nshots, nsnap),
                           "padded_cells": cells, "l2": "flushed between timed solves (%d MB write)" %
                                                        (L2_FLUSH_BYTES >> 20),
                           "parallelism": "replicas x%d" % world},
                "roofline": roof, "cpu_baseline": cpu, "clocks": clk.summary(), "e2e": e2e, "gradient": grad,
                "gpu_launches": args.steps * launches_per_solve(
                    cfg, nsnap, path, x_folded=cfg["ndim"] == 3 and pkg.sim_get_info(sim.handle).z_variant in (2, 5))}
        print(json.dumps(line), flush=True)
    sim.close()
    if dist:
        dist.destroy_process_group()


def model_recipe(nz, nx, seed):
    """Seeded inputs of one paper-shaped 2D slice build: four deposits of six
    beds (noisy boundaries, texture, tapers), a squish and two faults."""
    import synth
    rng = np.random.default_rng(seed)
    ops = []
    for k in range(4):
        t, nb = nz // 5, 6
        base = np.sort(rng.uniform(2, t - 2, nb - 1))
        b = base[:, None, None] + 2.0 * synth.smooth(rng.standard_normal((nb - 1, 1, nx)).astype(np.float32), 3.0)
        ops.append(("deposit", dict(t=t, bounds=np.clip(b, 0, t - 1).astype(np.float32),
                                    vbed=rng.normal(1800.0 + 500.0 * (3 - k), 150.0, nb).astype(np.float32),
                                    beta=1.0, a_eta=30.0, f_top=0.1, f_base=0.1,
                                    eta=rng.standard_normal((t + 40, 1, nx)).astype(np.float32),
                                    offsets=rng.integers(0, 40, nb), label0=10 * (k + 1))))
    dz = synth.smooth(rng.uniform(-1, 1, (1, nx)).astype(np.float32), 40.0)
    ops.append(("squish", dict(dz=(dz / np.abs(dz).max() * 20.0).astype(np.float32), fill=1500.0, fill_label=0)))
    for k in range(2):
        ops.append(("fault", dict(cz=nz * rng.uniform(0.3, 0.6), cx=nx * rng.uniform(0.2, 0.8),
                                  dip=np.deg2rad(rng.uniform(50, 70)), radius=rng.uniform(300, 3000),
                                  slip=rng.uniform(3, 15), direction=int(rng.choice([-1, 1])),
                                  d_die=rng.uniform(20, 60), theta_die=np.deg2rad(40.0), fill=1500.0,
                                  fill_label=0)))
    return ops


def run_model(args):
    """Model-builder warps (App. model builder modules): one 619 x 1000 slice
    built from a 4500 m/s half-space by four deposits, a squish and two
    faults, all on the GPU; value = voxel updates per second of the chain."""
    import torch
    import paper_2605_30541_gb300 as pkg
    from paper_2605_30541_gb300 import model
    torch.cuda.set_device(0)
    nz, nx = 619, 1000
    ops = model_recipe(nz, nx, 7000)
    # the drawn fields live on the device before the timed builds
    dev_ops = [(kind, {k: (torch.as_tensor(a, device="cuda") if k in ("bounds", "eta", "dz") else a)
                       for k, a in p.items()}) for kind, p in ops]
    base = torch.full((nz, nx), 4500.0, device="cuda")
    lab0 = torch.zeros((nz, nx), dtype=torch.int32, device="cuda")

    def build():
        v, lab = base, lab0
        for kind, p in dev_ops:
            if kind == "deposit":
                v, lab = model.deposit(v, lab, p["t"], p["bounds"], p["vbed"], beta=p["beta"], a_eta=p["a_eta"],
                                       f_top=p["f_top"], f_base=p["f_base"], eta=p["eta"], offsets=p["offsets"],
                                       label0=p["label0"])
            elif kind == "squish":
                v, lab = model.squish(v, lab, p["dz"], p["fill"], p["fill_label"])
            else:
                v, lab = model.fault(v, lab, **p)
        return v, lab

    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        build()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with Clocks(0) as clk:
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            v, lab = build()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
    per = sum(a.elapsed_time(b) for a, b in ev) / args.steps / 1e3
    updates = len(ops) * nz * nx
    # the warps alone on a 619 x 64 x 1000 volume (41 M voxels, far above L2),
    # outputs preallocated, through the C ABI: squish for its HBM roofline
    # (16 B per voxel: velocity and label, in and out), the 3D fault (8^3 taps)
    ny3 = 64
    v3 = torch.empty((nz, ny3, nx), device="cuda").uniform_(1500.0, 4500.0)
    l3 = torch.randint(0, 9, (nz, ny3, nx), dtype=torch.int32, device="cuda")
    vo3, lo3 = torch.empty_like(v3), torch.empty_like(l3)
    dz3 = torch.empty((ny3, nx), device="cuda").uniform_(-12.0, 12.0)
    f3 = pkg.abi.SimFault(cz=300.0, cy=32.0, cx=500.0, azimuth=0.6, dip=np.deg2rad(60.0), radius=800.0, slip=9.0,
                          direction=1, pad=0, d_die=40.0, d_perp=400.0, theta_die=np.deg2rad(40.0))

    def timed(fn, reps):
        fn()
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps / 1e3

    t_sq = timed(lambda: pkg.sim_model_squish(nz, ny3, nx, v3, l3, dz3, 1500.0, 0, vo3, lo3), 10)
    t_f3 = timed(lambda: pkg.sim_model_fault(nz, ny3, nx, v3, l3, f3, 1500.0, 0, vo3, lo3), 3)
    vox3 = nz * ny3 * nx
    peak, peak_kind = read_peaks()
    ach = 16.0 * vox3 / t_sq / 1e9
    cpu = None
    if not args.no_cpu:
        from oracle import model as om
        import time as _t
        cols = 100  # bounded sample: the same chain on the first 100 columns
        v = np.full((nz, 1, cols), 4500.0)
        lab = np.zeros((nz, 1, cols), np.int32)
        t0 = _t.perf_counter()
        for kind, p in ops:
            if kind == "deposit":
                v, lab = om.deposit(v, lab, p["t"], p["bounds"][..., :cols].astype(np.float64), p["vbed"], p["beta"],
                                    p["a_eta"], p["f_top"], p["f_base"], p["eta"][..., :cols].astype(np.float64),
                                    p["offsets"], p["label0"])
            elif kind == "squish":
                v, lab = om.squish(v, lab, p["dz"][..., :cols].astype(np.float64), p["fill"], p["fill_label"])
            else:
                q = {k2: v2 for k2, v2 in p.items() if k2 not in ("fill", "fill_label")}
                q.update(cy=0.0, azimuth=np.pi / 2, d_perp=1e9)
                v, lab = om.fault(v, lab, q, p["fill"], p["fill_label"])
        dt = _t.perf_counter() - t0
        cpu = {"value": len(ops) * nz * cols / dt / 1e6, "unit": "Mvoxel/s", "cores": 1, "kind": "oracle",
               "sample": "the same chain on the first %d of %d columns (numpy FP64), %.1f s" % (cols, nx, dt)}
    line = {"metric": "Mvoxel-updates/s (model-builder warps)", "value": updates / per / 1e6, "unit": "Mvoxel/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 (f64 coordinates)",
            "data": "synthetic",
            "config": {"workload": "model: one 619x1000 slice = 4 deposits (6 beds, texture, tapers) + squish + "
                                   "2 faults, from a 4500 m/s half-space", "warps_per_slice": len(ops),
                       "volume_619x64x1000": {"squish_us": t_sq * 1e6, "fault_us": t_f3 * 1e6,
                                              "fault_mvoxel_s": vox3 / t_f3 / 1e6},
                       "l2": "flushed between timed builds"},
            "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                         "traffic": None, "kernel": "k_squish", "peak_kind": peak_kind,
                         "algorithmic_bytes_per_launch": 16.0 * vox3, "avg_launch_us": t_sq * 1e6,
                         "case": "619 x 64 x 1000 volume"},
            "cpu_baseline": cpu, "clocks": clk.summary(), "gpu_launches": args.steps * len(ops)}
    print(json.dumps(line), flush=True)


def run_gradient(args):
    """The FWI gradient workload alone (201 x 201 procedural model + 20-cell
    CPML on every side, 16 shots, nt = 4000): one sim_adjoint of all shots
    with FP16 checkpoints per step; value = padded cells x shots x steps of
    the forward problem per second of gradient (the profiling command of the
    adjoint-state kernels)."""
    import torch
    import synth
    import paper_2605_30541_gb300 as pkg
    torch.cuda.set_device(0)
    c = synth.config_c4(nt=args.nt or 4000)
    ns, nt, nrec = len(c["src"]), c["nt"], len(c["rec"])
    true = pkg.Simulator(c, c["vel_true"], max_shots=ns, max_rec=nrec)
    d = true.forward(c["wavelet"], c["src"], c["rec"])["gather"].contiguous()
    true.close()
    sim = pkg.Simulator(c, c["vel"], max_shots=ns, max_rec=nrec)
    w = torch.as_tensor(c["wavelet"], device="cuda")
    src, rec = np.ascontiguousarray(c["src"]), np.ascontiguousarray(c["rec"])
    g = torch.zeros(c["vel"].shape, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        pkg.sim_adjoint(sim.handle, ns, w, src, nrec, rec, d, None, None, 1, g)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(0) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
    per = e0.elapsed_time(e1) / 1e3 / args.steps
    cells = padded_cells(c) * ns
    peak, peak_kind = read_peaks()
    algo = gradient_bytes_per_shot(c, True) * ns
    line = {"metric": "Gcell-updates/s of the gradient (FP16 checkpoints)", "value": cells * nt / per / 1e9,
            "unit": "Gcell/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 (f16 storage)",
            "data": "synthetic",
            "config": {"workload": "c4g: gradient, 201x201 + 20-cell CPML on every side, 16 shots, nt=%d, "
                                   "FP16 checkpoints" % nt, "s_per_shot": per / ns, "l2": "not flushed (a whole "
                                   "gradient per step)"},
            "roofline": {"bound": "hbm", "achieved": algo / per / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": algo / per / 1e9 / peak, "peak_kind": peak_kind, "traffic": None,
                         "algorithmic_bytes_per_step": algo},
            "cpu_baseline": None, "clocks": clk.summary(), "gpu_launches": None}
    print(json.dumps(line), flush=True)
    sim.close()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "model":
        run_model(args)
    elif args.workload in ("c3", "c6g"):
        run_batch(args)
    elif args.workload == "c4g":
        run_gradient(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
