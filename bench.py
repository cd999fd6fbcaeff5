"""Throughput of the e-ph hot path on the silicon-like fcc workload.

One step = one pass of the hot path over the whole workload: interpolate
eps, U on the 40^3 k grid and omega, e on the 40^3 q grid is done once per
model (set_grids); each timed step evaluates, for every k-point in the
0.3 eV window above the band minimum and every q of the 40^3 grid, the
Wannier interpolation of g (Re-sum with the U(k) fold, Rp-sum), the rotation
by U(k+q), the mode projection, |g|^2, the Gaussian weights and Gamma_nk.
The unit is the (k, q) pair.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--precision fp32|fp64|bf16x3|tf32x3]
Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("(k,q) |g|² pairs/s and Γ_nk collision sums/s at stated err vs FP64; % of roofline")
WORKLOAD = "fcc Si-like 8 bands, 2 atoms, 381 R_e x 381 R_p; 40^3 k (0.3 eV window) x 40^3 q; T=300 K, sigma=10 meV"
KGRID = (40, 40, 40)
T_K, SIGMA, WIN = 300.0, 0.010, 0.3
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
SM_COUNT, FP32_LANES, SM_MAX_MHZ = 152, 128, 2070.0
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per unit of work from one
# ncu capture of each kernel: the fused rates kernel on 64 window k x 40^3 q, the
# collision kernel on the 30^3 list.  An entry is None while its kernel has changed
# since the capture.
TRAFFIC = {"k_tc_rates_bf16x3_bytes_per_pair": (1.134679e9 + 23.895552e6) / (64 * 64000),
           "k_collision_bytes_per_entry": (383152384 + 3583744) / 31890730}


def load_peaks():
    try:
        with open(PEAKS) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu_id}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) == 8:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[4 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_setup():
    from paper_2002_02045_gb300.dist import rank_world
    return rank_world()


def barrier(world):
    from paper_2002_02045_gb300.dist import barrier as _b
    _b()


def max_over_ranks(x, world):
    from paper_2002_02045_gb300.dist import max_over_ranks as _m
    return _m(x)


def cpu_baseline(model, n_k=2, with_result=False):
    """The FP64 oracle as it stands on a bounded sample: n_k window k-points x all 40^3 q.
    With with_result, also returns the sampled k-grid indices and their oracle Gamma."""
    from oracle import eph as O
    import synthetic as S
    t0 = time.perf_counter()
    pts = S.mp_grid(*KGRID)
    eps, _ = O.bands(model, pts)
    emin = eps.min()
    # k-points with a band strictly inside the window (not on an edge to rounding)
    win = np.nonzero(((eps >= emin + 1e-9) & (eps <= emin + WIN - 1e-9)).any(1))[0]
    sample = win[np.linspace(0, len(win) - 1, n_k).astype(int)]
    ref = O.scattering_rates_grid(model, KGRID, KGRID, sample, T_K, emin - WIN, SIGMA, q_chunk=16000)
    dt = time.perf_counter() - t0
    nq = int(np.prod(KGRID))
    info = {"value": n_k * nq / dt, "unit": "pairs/s", "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
            "sample": f"{n_k} window k-points x {nq} q (FP64 NumPy oracle, band interpolation of the 40^3 grid "
                      f"included), {dt:.1f} s"}
    if with_result:
        return info, sample.astype(np.int32), ref, emin - WIN
    return info


def rel_err(got, ref):
    """max over states of |got - ref| / (|ref| + 1e-6 max|ref|): the norm of the parity tests."""
    got, ref = np.asarray(got, np.float64), np.asarray(ref, np.float64)
    return float(np.max(np.abs(got - ref) / (np.abs(ref) + 1e-6 * np.abs(ref).max())))


def cpu_baseline_list(ctx, grid, nnz, es, f, n_sample=4_000_000):
    """The FP64 oracle's I[f] and its transposed product (collision, collision_vjp) on the
    first n_sample entries of the device-built list, timed on the host cores."""
    import torch
    from oracle import eph as O
    n = int(min(nnz, n_sample))
    dev = {k: torch.empty(nnz, dtype=dt, device="cuda")
           for k, dt in (("row", torch.int32), ("col", torch.int32), ("mode", torch.int32), ("g2", torch.float32))}
    ctx.pgb_collision_list(dev["row"], dev["col"], dev["mode"], dev["g2"])
    h = {k: v[:n].cpu().numpy() for k, v in dev.items()}
    del dev
    nk = int(np.prod(grid))
    hw = torch.empty((nk, ctx.nmode), dtype=torch.float64, device="cuda")
    ctx.pgb_get_grid_energies(None, hw)
    hw = hw.cpu().numpy()
    k, kp = h["row"] // 2, h["col"] // 2
    c = [np.stack([x // (grid[1] * grid[2]), (x // grid[2]) % grid[1], x % grid[2]], -1) for x in (k, kp)]
    qv = (c[1] - c[0]) % np.array(grid)
    q = (qv[:, 0] * grid[1] + qv[:, 1]) * grid[2] + qv[:, 2]
    hw_e = hw[q, h["mode"]]
    es_h, f_h = es.cpu().numpy(), f.cpu().numpy()
    row, col, g2 = h["row"].astype(np.int64), h["col"].astype(np.int64), h["g2"].astype(np.float64)
    t0 = time.perf_counter()
    O.collision(f_h, es_h, row, col, hw_e, g2, T_K, SIGMA, nk)
    t_fwd = time.perf_counter() - t0
    t0 = time.perf_counter()
    O.collision_vjp(f_h, np.ones_like(f_h), es_h, row, col, hw_e, g2, T_K, SIGMA, nk)
    t_vjp = time.perf_counter() - t0
    cores = len(os.sched_getaffinity(0))
    sample = f"first {n} entries of the {nnz}-entry list, one application (FP64 NumPy oracle)"
    return ({"value": n / t_fwd, "unit": "entries/s", "cores": cores, "kind": "oracle", "sample": sample},
            {"value": n / t_vjp, "unit": "entries/s", "cores": cores, "kind": "oracle", "sample": sample})


def run_reference(args, rank, world):
    if rank != 0:
        return
    import synthetic as S
    model = S.model_c2()
    for _ in range(args.warmup):
        cpu_baseline(model, n_k=1)
    t0 = time.perf_counter()
    vals = [cpu_baseline(model, n_k=1) for _ in range(args.steps)]
    dt = time.perf_counter() - t0
    v = float(np.mean([x["value"] for x in vals]))
    cb = dict(vals[-1])
    cb["value"] = v
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "pairs/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / max(1, args.steps),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample_per_step": "1 window k-point x 64000 q"},
        "cpu_baseline": cb, "e2e": {"value": v, "unit": "pairs/s", "h2d_bytes_per_step": 0,
                                    "d2h_bytes_per_step": 0}}), flush=True)


def run_ours(args, rank, world, local):
    import torch
    import synthetic as S
    from paper_2002_02045_gb300 import PRECISIONS, Context, build as _b
    from paper_2002_02045_gb300.native import PROF_EPILOGUE, PROF_QSUM, PROF_RSUM

    _b.build()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    prec = PRECISIONS[args.precision]
    model = S.model_c2()
    ctx = Context(local)
    ctx.pgb_set_model(model)
    ctx.pgb_set_grids(KGRID, KGRID)
    nk_grid = int(np.prod(KGRID))
    eps = torch.empty((nk_grid, model.nw), dtype=torch.float64, device="cuda")
    ctx.pgb_get_grid_energies(eps, None)
    emin = float(eps.min())
    mu = emin - WIN
    kbuf = torch.empty((nk_grid,), dtype=torch.int32, device="cuda")
    nwin = ctx.pgb_window(emin, emin + WIN, kbuf)
    if args.max_k:
        nwin = min(nwin, args.max_k)
    k0 = 0
    if args.shard and world > 1:
        # strong scaling: the window k-points are split across ranks (no exchange)
        from paper_2002_02045_gb300.dist import partition
        k0, k1 = partition(nwin, rank, world)
        nwin = k1 - k0
    kidx = kbuf[k0:k0 + nwin].contiguous()
    gam = torch.empty((nwin, model.nw), dtype=torch.float64, device="cuda")
    nq = nk_grid
    pairs = nwin * nq

    def step():
        ctx.pgb_scattering_rates(kidx, T_K, mu, SIGMA, prec, gam)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ctx.pgb_profile(True)
    for c in (PROF_QSUM, PROF_RSUM, PROF_EPILOGUE):
        ctx.pgb_profile_read(c)
    props = torch.cuda.get_device_properties(local)
    clocks = ClockSampler(f"GPU-{props.uuid}" if getattr(props, "uuid", None) else str(local))
    n0 = ctx.pgb_launch_count()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier(world)
    ms = max_over_ranks(e0.elapsed_time(e1), world)
    launches = ctx.pgb_launch_count() - n0
    q_ms, q_n = ctx.pgb_profile_read(PROF_QSUM)
    r_ms, _ = ctx.pgb_profile_read(PROF_RSUM)
    p_ms, _ = ctx.pgb_profile_read(PROF_EPILOGUE)
    ctx.pgb_profile(False)
    from paper_2002_02045_gb300.dist import sum_over_ranks
    total_pairs = sum_over_ranks(pairs) if world > 1 else pairs
    value = total_pairs * args.steps / (ms * 1e-3)

    # roofline of the dominant kernel: the Fourier sum over R_p (a complex contraction)
    peaks, peak_src = load_peaks()
    flop_per_pair = 8.0 * len(model.R_gp) * model.nmode * model.nw ** 2
    achieved = flop_per_pair * pairs * args.steps / (q_ms * 1e-3) / 1e12
    peak_burst = None
    if args.precision in ("bf16x3", "tf32x3"):
        # the timed loop runs for seconds under the power cap: the sustained peak applies
        ratio = 1.0 if args.precision == "bf16x3" else 0.5
        peak = peaks["bf16_tflops_sustained"] * ratio
        peak_burst = peaks["bf16_tflops"] * ratio
        roof = {"bound": "tensor",
                "peak_source": f"{peak_src} bf16 sustained (seconds-long loop under the power cap)" +
                               (" x 1/2 (tf32 nominal ratio)" if args.precision == "tf32x3" else "")}
    else:
        lanes = FP32_LANES if args.precision == "fp32" else 2   # FP64 units per SM on GB300 are few
        peak = SM_COUNT * lanes * 2 * SM_MAX_MHZ * 1e6 / 1e12
        roof = {"bound": "alu", "peak_source": f"derived: {SM_COUNT} SMs x {lanes} lanes x 2 flop x {SM_MAX_MHZ:.0f} MHz"}
    issue = 3.0 if args.precision in ("bf16x3", "tf32x3") else 1.0
    roof.update({"achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                 "traffic": (TRAFFIC["k_tc_rates_bf16x3_bytes_per_pair"] * pairs * args.steps / max(1, q_n)
                             if args.precision == "bf16x3" and TRAFFIC["k_tc_rates_bf16x3_bytes_per_pair"] else None),
                 "traffic_note": "DRAM bytes per launch scaled by pairs from a 64-k capture (grows with the k count)",
                 "kernel": ("fused q-sum + rotation/projection/Gamma epilogue (k_tc_rates)"
                            if issue > 1 else "q-sum complex GEMM (k_cgemm)"),
                 "algorithmic_flop_per_pair": flop_per_pair, "launches": q_n,
                 "pairs_per_launch": pairs * args.steps / max(1, q_n),
                 "issued_mma_achieved": achieved * issue, "issued_mma_frac": achieved * issue / peak})
    if peak_burst:
        roof.update({"peak_burst": peak_burst, "frac_of_burst": achieved / peak_burst,
                     "issued_mma_frac_of_burst": achieved * issue / peak_burst})
    out = {
        "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "strong" if (args.shard and world > 1) else "weak",
        "vs_baseline": None, "dtype": {"fp32": "f32", "fp64": "f64", "bf16x3": "bf16x3", "tf32x3": "tf32x3"}[args.precision],
        "data": "synthetic",
        "tolerance_vs_fp64": {"bf16x3": 1e-3, "tf32x3": 1e-5, "fp32": 1e-5, "fp64": 1e-10}[args.precision],
        "config": {"workload": WORKLOAD, "kgrid": list(KGRID), "qgrid": list(KGRID), "nk_window": nwin,
                   "pairs_per_step": pairs, "precision": args.precision,
                   "l2": "inputs larger than L2 (g~ 446 MB, per-step intermediates > 1 GB)"},
        "delta_terms_per_s": value * 2 * model.nw ** 2 * model.nmode,
        "kernel_ms_per_step": {"q_sum": q_ms / args.steps, "r_sum": r_ms / args.steps,
                               "epilogue": p_ms / args.steps},
        "roofline": roof, "gpu_launches": launches, "clocks": clk,
    }

    if args.variants and rank == 0:
        out["variants"] = {}
        for name in ("tf32x3", "fp32"):
            if name == args.precision:
                continue
            p2 = PRECISIONS[name]
            ctx.pgb_scattering_rates(kidx, T_K, mu, SIGMA, p2, gam)
            torch.cuda.synchronize()
            v0, v1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            v0.record(stream)
            ctx.pgb_scattering_rates(kidx, T_K, mu, SIGMA, p2, gam)
            v1.record(stream)
            torch.cuda.synchronize()
            out["variants"][name] = {"value": pairs / (v0.elapsed_time(v1) * 1e-3), "unit": "pairs/s",
                                     "ms_per_step": v0.elapsed_time(v1),
                                     "tolerance_vs_fp64": {"tf32x3": 1e-5, "fp32": 1e-5}[name]}
    # (before the sections below, which change the context's grids)
    if args.cpu_baseline and rank == 0 and world == 1:
        # the oracle's Gamma of its sample doubles as the measured error of every form
        info, ks, ref, mu_o = cpu_baseline(model, with_result=True)
        out["cpu_baseline"] = info
        errs = {}
        for name in dict.fromkeys([args.precision, "bf16x3", "tf32x3", "fp32"]):
            g = np.zeros((len(ks), model.nw))
            ctx.pgb_scattering_rates(ks, T_K, mu_o, SIGMA, PRECISIONS[name], g)
            errs[name] = rel_err(g, ref)
        out["measured_rel_err_vs_fp64"] = {
            "value": errs[args.precision], "by_precision": errs,
            "norm": "max over states |G - G_oracle| / (|G_oracle| + 1e-6 max G_oracle)",
            "sample": f"Gamma_nk of the cpu_baseline k-points {ks.tolist()} (all 8 bands, every q of the 40^3 grid)"}
    if args.dynamics:
        out["dynamics"] = dynamics(ctx, model, args, world, peaks, peak_src)
    if args.polar:
        out["polar"] = polar(ctx, args, world)
    if args.batched:
        out["batched"] = batched(args, world)
    if args.general and rank == 0:
        out["general_shape"] = general_shape(args, world)
    if args.e2e and rank == 0:
        out["e2e"] = e2e(ctx, model, prec, steps=1)
    if rank == 0:
        print(json.dumps(out), flush=True)
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


DYN_GRID = (30, 30, 30)
DYN_WINDOW = 0.6


def dynamics(ctx, model, args, world, peaks, peak_src):
    """Real-time BTE on the 30^3 grid: two lowest bands, states within 0.6 eV of
    the band minimum, list built on the device (untimed setup), then RK4 steps
    of dt = 1 fs from the hot-carrier pulse (timed)."""
    import torch
    import synthetic as S
    from paper_2002_02045_gb300.native import PROF_COLLISION
    grid = (args.dyn_grid,) * 3
    ctx.pgb_set_grids(grid, grid)
    nk = int(np.prod(grid))
    eps = torch.empty((nk, model.nw), dtype=torch.float64, device="cuda")
    ctx.pgb_get_grid_energies(eps, None)
    emin = float(eps[:, :2].min())
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    nnz = ctx.pgb_build_collision_grid(0, 2, emin, emin + DYN_WINDOW, T_K, SIGMA)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    es = torch.empty((2 * nk,), dtype=torch.float64, device="cuda")
    ctx.pgb_collision_energies(es)
    f = torch.as_tensor(S.pulse_occupations(es.cpu().numpy(), emin)).cuda()
    f_pulse = f.clone()
    n0 = float(f.sum())
    ctx.pgb_step_rk4(f, 1.0, 5)                       # warm-up
    torch.cuda.synchronize()
    ctx.pgb_profile(True)
    ctx.pgb_profile_read(PROF_COLLISION)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    e0.record(stream)
    ctx.pgb_step_rk4(f, 1.0, args.dyn_steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1), world)
    k_ms, k_n = ctx.pgb_profile_read(PROF_COLLISION)
    ctx.pgb_profile(False)
    # carrier population N(E) of the final f on 401 energies (tetrahedron method)
    Egrid = torch.linspace(emin - 0.05, emin + DYN_WINDOW + 0.05, 401, dtype=torch.float64, device="cuda")
    Npop = torch.empty_like(Egrid)
    ctx.pgb_population(f, Egrid, Npop)
    torch.cuda.synchronize()
    t0p = time.perf_counter()
    ctx.pgb_population(f, Egrid, Npop)
    torch.cuda.synchronize()
    pop_ms = 1e3 * (time.perf_counter() - t0p)
    evals = 4 * args.dyn_steps
    byte_per_entry = 12.0
    achieved = byte_per_entry * nnz * evals / (k_ms * 1e-3) / 1e9
    adj = adjoint(ctx, f_pulse, nnz, args, world, peaks, peak_src, ms / args.dyn_steps) if args.adj_steps > 0 else None
    cb_fwd = cb_adj = None
    if args.cpu_baseline and world == 1:
        cb_fwd, cb_adj = cpu_baseline_list(ctx, grid, nnz, es, f_pulse)
        if adj is not None:
            adj["cpu_baseline"] = cb_adj
    return {
        "metric": "collision-entry evaluations/s (RK4, 4 evaluations per step)",
        "value": world * nnz * evals / (ms * 1e-3), "unit": "entries/s",
        "rk4_steps_per_s": world * args.dyn_steps / (ms * 1e-3), "steps": args.dyn_steps,
        "ms_per_rk4_step": ms / args.dyn_steps, "nnz": nnz, "states": 2 * nk,
        "config": {"workload": f"same model, {grid[0]}^3 k = q grid, 2 lowest bands, states within "
                               f"{DYN_WINDOW} eV of the band minimum, 7 sigma screen, dt = 1 fs, hot-carrier pulse",
                   "list_build_s": build_s},
        "carrier_number_drift": abs(float(f.sum()) - n0) / n0,
        "cpu_baseline": cb_fwd,
        "population": {"energies": 401, "ms": pop_ms, "carriers_in_window_per_cell": float(Npop[-1] - Npop[0]),
                       "method": "linear tetrahedron, 6 per cell, both bands"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / peaks["hbm_gbs"],
                     "traffic": (TRAFFIC["k_collision_bytes_per_entry"] * nnz
                                 if TRAFFIC["k_collision_bytes_per_entry"] else None),
                     "kernel": "k_collision",
                     "peak_source": peak_src, "algorithmic_bytes_per_entry": byte_per_entry,
                     "entries_per_launch": nnz, "launches": k_n},
        "adjoint": adj,
    }


def adjoint(ctx, f, nnz, args, world, peaks, peak_src, fwd_ms_per_step):
    """Reverse-mode RK4 on the same list: dL/df0 and dL/d|g|^2 of the mean carrier
    energy at t_end, L = sum_s e_s f_s / sum_s f_s, through adj_steps steps from
    the pulse (forward with checkpoints, segment recompute, four transposed-list
    column passes per step), timed after one warm-up call that also builds the
    transposed list.  dL/df(t_end) = (e_s - L) / sum_s f_s is the loss's own
    derivative, formed by the caller."""
    import torch
    from paper_2002_02045_gb300.native import PROF_ADJOINT
    ns = f.numel()
    es = torch.empty(ns, dtype=torch.float64, device="cuda")
    ctx.pgb_collision_energies(es)
    fe = f.clone()
    ctx.pgb_step_rk4(fe, 1.0, args.adj_steps)
    n_end = fe.sum()
    w = (es - (es * fe).sum() / n_end) / n_end
    lam0 = torch.empty_like(f)
    dg2 = torch.empty(nnz, dtype=torch.float64, device="cuda")
    ck = args.adj_checkpoint
    ctx.pgb_rk4_adjoint(f, 1.0, 2, ck, w, lam0, dg2)          # warm-up, transposed list
    torch.cuda.synchronize()
    ctx.pgb_profile(True)
    ctx.pgb_profile_read(PROF_ADJOINT)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    e0.record(stream)
    ctx.pgb_rk4_adjoint(f, 1.0, args.adj_steps, ck, w, lam0, dg2)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1), world)
    k_ms, k_n = ctx.pgb_profile_read(PROF_ADJOINT)
    ctx.pgb_profile(False)
    # per entry and column pass: src, a, b, alpha, beta (4 B each) + FP64 read-modify-write of dL/d|g|^2
    byte_per_entry = 36.0
    achieved = byte_per_entry * nnz * k_n / (k_ms * 1e-3) / 1e9
    return {
        "metric": "reverse-mode RK4 steps/s (dL/df0 and dL/d|g|^2 of the final mean carrier energy, "
                  "forward + recompute + reverse)",
        "value": world * args.adj_steps / (ms * 1e-3), "unit": "steps/s", "steps": args.adj_steps,
        "checkpoint": ck, "ms_per_step": ms / args.adj_steps,
        "ratio_to_forward_step": (ms / args.adj_steps) / fwd_ms_per_step,
        "finite": bool(torch.isfinite(lam0).all() and torch.isfinite(dg2).all()),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / peaks["hbm_gbs"], "traffic": None, "kernel": "k_adj_col",
                     "peak_source": peak_src, "algorithmic_bytes_per_entry": byte_per_entry,
                     "entries_per_launch": nnz, "launches": k_n,
                     "kernel_ms_share": k_ms / ms},
    }


POLAR_GRID = (60, 60, 60)
POLAR_WINDOW = 0.2
MC_SAMPLES = 65536


def monte_carlo(ctx, args, world, m, kw, mu, stream, e0, e1):
    """Monte-Carlo q rates on the polar model: Cauchy samples about q = 0 for the 16 lowest
    window k-points, TF32x3 (the FP32 tier's tensor-core form) timed with the FP32 SIMT form
    beside it, and the oracle on a bounded sample of the same call."""
    import torch
    import synthetic as S
    # Monte-Carlo q: Cauchy samples about q = 0 for the 16 lowest window k-points
    from paper_2002_02045_gb300 import PGB_FP32, PGB_TC_TF32X3, PGB_Q_CAUCHY
    pts = torch.as_tensor(S.mp_grid(*POLAR_GRID)).cuda()
    kmc = pts[kw[:16].long()].contiguous()
    u = torch.as_tensor(np.random.default_rng(S.SEED_BASE + 33).uniform(size=(MC_SAMPLES, 3))).cuda()
    gmc = torch.empty((len(kmc), m.nw), dtype=torch.float64, device="cuda")
    emc = torch.empty_like(gmc)
    from paper_2002_02045_gb300.native import PROF_BANDS

    def mc_run(prec):
        ctx.pgb_scattering_rates_mc(kmc, u[:1024].contiguous(), PGB_Q_CAUCHY, 0.1, T_K, mu, SIGMA, prec, gmc, emc)
        torch.cuda.synchronize()
        ctx.pgb_profile(True)
        ctx.pgb_profile_read(PROF_BANDS)
        e0.record(stream)
        ctx.pgb_scattering_rates_mc(kmc, u, PGB_Q_CAUCHY, 0.1, T_K, mu, SIGMA, prec, gmc, emc)
        e1.record(stream)
        torch.cuda.synchronize()
        prof = ctx.pgb_profile_read(PROF_BANDS)
        ctx.pgb_profile(False)
        return e0.elapsed_time(e1), prof, gmc.clone()

    ms_mc32, _, g32 = mc_run(PGB_FP32)
    ms_mc, (hk_ms, hk_n), _ = mc_run(PGB_TC_TF32X3)   # TF32x3: the FP32 tier (1e-5) on the tensor cores
    dev_mc = float(((gmc - g32).abs() / (g32.abs() + 1e-6 * g32.abs().max())).max())
    # the k+q points' H(k) Fourier sums: real cos/sin form over one representative of each
    # {R, -R} (K = 2 n_rep rows) into the nw^2 packed Hermitian columns, 2 FLOP per term, in
    # double-float on the FP32 pipe: 13.5 FP32 instructions per term (the product and its error in
    # 4, TwoSum and the low-part update in 8, a renormalisation of 3 every second term), so its ALU
    # peak is the FP32 instruction rate / 13.5
    n_rep = (len(m.R_H) + 1) // 2
    hk_flop_pt = 2.0 * (2 * n_rep) * m.nw ** 2
    hk_flop = hk_flop_pt * len(kmc) * MC_SAMPLES
    hk_tf = hk_flop / (hk_ms * 1e-3) / 1e12 if hk_ms > 0 else None
    df_peak = 152 * 128 * 2.07e9 / 13.5 * 2 / 1e12      # TFLOP/s of double-float multiply-adds
    rel = (emc / gmc.clamp_min(1e-300))[gmc > 0]
    cb = None
    if args.cpu_baseline and world == 1:
        from oracle import eph as O
        ns_cpu = 2048
        t0 = time.perf_counter()
        O.scattering_rates_mc(m, kmc[:1].cpu().numpy(), u[:ns_cpu].cpu().numpy(), O.Q_CAUCHY, 0.1, T_K, mu, SIGMA)
        dt_cpu = time.perf_counter() - t0
        cb = {"value": ns_cpu / dt_cpu, "unit": "pairs/s", "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
              "sample": f"1 k-point x {ns_cpu} Cauchy q samples of the same polar model (FP64 NumPy oracle: "
                        f"bands at every k+q, short- and long-range g, rates), {dt_cpu:.1f} s"}
    mc = {"metric": "(k,q) pairs/s, Gamma_nk by Cauchy-sampled random q (FP32 tier: TF32x3 R_p sums, "
                                  "FP32 epilogue, bands and phonons at every sample with FP64-refined energies)",
                        "value": len(kmc) * MC_SAMPLES / (ms_mc * 1e-3), "unit": "pairs/s", "ms": ms_mc,
                        "precision": "tf32x3", "k_points": len(kmc), "samples": MC_SAMPLES, "cauchy_width": 0.1,
                        "median_relative_stderr": float(rel.median()) if rel.numel() else None,
                        "fp32_simt": {"value": len(kmc) * MC_SAMPLES / (ms_mc32 * 1e-3), "unit": "pairs/s",
                                      "ms": ms_mc32, "max_rel_dev_tf32x3_vs_fp32": dev_mc},
                        "roofline": {"bound": "alu", "kernel": "k_herm_sum: packed Hermitian H(k+q) = sum_R "
                                                                "cos(k.R) C_R + sin(k.R) S_R at every sample "
                                                                "(double-float on the FP32 pipe)",
                                     "achieved": hk_tf, "peak": df_peak, "unit": "TFLOP/s",
                                     "frac": hk_tf / df_peak if hk_tf else None,
                                     "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2.07 GHz / 13.5 FP32 "
                                                    "instructions per double-float multiply-add, x 2 FLOP",
                                     "algorithmic_flop_per_sample_point": hk_flop_pt,
                                     "kernel_ms": hk_ms, "launches": hk_n,
                                     "share_of_call": hk_ms / ms_mc if ms_mc > 0 else None}}
    return mc, cb


def polar(ctx, args, world):
    """Polar zincblende model with the long-range (Froehlich) coupling: Gamma_nk of
    the k-points within 0.2 eV of the band minimum over the 60^3 q grid (timed, the
    same precision as the headline), then the iterative BTE and mobility on the
    window's scattering list (list build and transport timed separately)."""
    import torch
    import synthetic as S
    from paper_2002_02045_gb300 import PRECISIONS
    m = S.model_c3()
    prec = PRECISIONS[args.precision]
    ctx.pgb_set_model(m)
    ctx.pgb_set_lattice(m.A, m.tau)
    ctx.pgb_set_polar(m.zstar, m.eps_inf, m.ewald_lambda)
    ctx.pgb_set_grids(POLAR_GRID, POLAR_GRID)
    nk = int(np.prod(POLAR_GRID))
    eps = torch.empty((nk, m.nw), dtype=torch.float64, device="cuda")
    ctx.pgb_get_grid_energies(eps, None)
    emin = float(eps.min())
    mu = emin - 0.3
    kbuf = torch.empty((nk,), dtype=torch.int32, device="cuda")
    nwin = ctx.pgb_window(emin - 1e-6, emin + POLAR_WINDOW, kbuf)
    kw = kbuf[:nwin].clone()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if args.mc_only:     # the Monte-Carlo part alone (profiling)
        mc, cb = monte_carlo(ctx, args, world, m, kw, mu, stream, e0, e1)
        return {"monte_carlo": mc, "cpu_baseline": cb}
    gam = torch.empty((nwin, m.nw), dtype=torch.float64, device="cuda")
    ctx.pgb_scattering_rates(kw, T_K, mu, SIGMA, prec, gam)     # warm-up (tables)
    barrier(world)
    torch.cuda.synchronize()
    e0.record(stream)
    ctx.pgb_scattering_rates(kw, T_K, mu, SIGMA, prec, gam)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1), world)
    pairs = nwin * nk
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    nnz = ctx.pgb_build_collision_grid(0, 2, emin - 1e-6, emin + POLAR_WINDOW, T_K, SIGMA)
    torch.cuda.synchronize()
    t_list = time.perf_counter() - t0
    from paper_2002_02045_gb300.native import PROF_COLLISION
    peaks, peak_src = load_peaks()
    ctx.pgb_profile(True)
    ctx.pgb_profile_read(PROF_COLLISION)             # reset the class: the BTE iterations are timed in it
    t0 = time.perf_counter()
    mob_rta, mob, it = ctx.pgb_transport(mu, prec, 3000, 1e-6)
    t_tr = time.perf_counter() - t0
    it_ms, it_n = ctx.pgb_profile_read(PROF_COLLISION)
    ctx.pgb_profile(False)
    bte_bytes = 12.0 * nnz        # col (4 B) + W (8 B) per entry; F is gathered from L2
    bte_gbs = bte_bytes * it_n / (it_ms * 1e-3) / 1e9 if it_ms > 0 else None
    bte_flops = 6.0 * nnz         # three FP64 multiply-adds per entry (x, y, z)
    bte_tf = bte_flops * it_n / (it_ms * 1e-3) / 1e12 if it_ms > 0 else None
    FP64_PEAK = ctx.pgb_diag_fp64_rate()   # TFLOP/s, measured on this device (the iteration is FP64-bound)
    mc, cb = monte_carlo(ctx, args, world, m, kw, mu, stream, e0, e1)
    return {
        "metric": "(k,q) pairs/s, polar Gamma_nk (short-range Wannier sum + long-range Ewald term)",
        "value": world * pairs / (ms * 1e-3), "unit": "pairs/s", "ms": ms, "pairs": pairs, "nk_window": nwin,
        "precision": args.precision,
        "config": {"workload": f"polar zincblende 8 bands, 2 atoms (69.7, 74.9 amu), 381 R_e x 381 R_p + 6 "
                               f"long-range rows (Z* = +-2, eps_inf = 10.9); {POLAR_GRID[0]}^3 k = q grid, "
                               f"k within {POLAR_WINDOW} eV of the band minimum; T = 300 K, sigma = 10 meV"},
        "transport": {"list_entries": nnz, "list_build_s": t_list, "solve_s": t_tr, "iterations": it,
                      "tolerance": 1e-6, "mobility_cm2_per_Vs": np.diag(mob).tolist(),
                      "mobility_rta_cm2_per_Vs": np.diag(mob_rta).tolist(),
                      "includes": "tau from the rates over the full q grid, velocities, W, iterations, mobility",
                      "iteration_ms": it_ms / max(1, it_n),
                      "roofline": {"bound": "alu", "kernel": "k_bte_iter (FP64)", "achieved": bte_tf,
                                   "peak": FP64_PEAK, "unit": "TFLOP/s",
                                   "frac": bte_tf / FP64_PEAK if bte_tf else None,
                                   "peak_source": "measured FP64 FMA rate of this device (pgb_diag_fp64_rate)",
                                   "algorithmic_flop_per_entry": 6.0, "launches": it_n,
                                   "hbm_achieved_gbs": bte_gbs,
                                   "hbm_frac": bte_gbs / peaks["hbm_gbs"] if bte_gbs else None,
                                   "hbm_peak_source": peak_src}},
        "cpu_baseline": cb,
        "monte_carlo": mc,
    }


BATCH_INSTANCES = 64
BATCH_K = 8


def batched(args, world):
    """64 seeded random instances (nw in {2..16}, 1-5 atoms, R shells of radius 1-3,
    grids 8^3..32^3), Gamma_nk of 8 k-points each over the full q grid at 300 K and
    5 meV, all in one graph launch (persistent kernel); timed over replays after
    the first call (tile autotuning and graph capture)."""
    import torch
    import synthetic as S
    from paper_2002_02045_gb300 import Batch, Context
    t0 = time.perf_counter()
    ids = [int(x) for x in args.batch_ids.split(",")] if args.batch_ids else list(range(args.batch_instances))
    models = [S.model_batch_instance(i) for i in ids]
    t_gen = time.perf_counter() - t0
    rng = np.random.default_rng(S.SEED_BASE + 55)
    ctxs, ks, mus, outs = [], [], [], []
    pairs = 0
    t0 = time.perf_counter()
    for m in models:
        c = Context(torch.cuda.current_device())
        c.pgb_set_model(m)
        g = m.meta["grid"]
        c.pgb_set_grids(g, g)
        nk = int(np.prod(g))
        eps = torch.empty((nk, m.nw), dtype=torch.float64, device="cuda")
        c.pgb_get_grid_energies(eps, None)
        ctxs.append(c)
        ks.append(np.sort(rng.choice(nk, BATCH_K, replace=False)).astype(np.int32))
        mus.append(float(0.5 * (eps.min() + eps.max())))
        outs.append(np.zeros((BATCH_K, m.nw)))
        pairs += BATCH_K * nk
    t_setup = time.perf_counter() - t0
    b = Batch(ctxs)
    t0 = time.perf_counter()
    b.pgb_batch_rates(ks, T_K, mus, 0.005, outs)       # autotune + capture + first run
    t_first = time.perf_counter() - t0
    reps = 3
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(reps):
        b.pgb_batch_rates(ks, T_K, mus, 0.005, outs)
    dt = max_over_ranks((time.perf_counter() - t0) / reps, world)
    tun = b.pgb_batch_tuning()
    finite = all(np.all(np.isfinite(o)) for o in outs)
    cb = None
    if args.cpu_baseline and world == 1:
        from oracle import eph as O
        small = [i for i, m in enumerate(models) if m.meta["grid"][0] == 8][:3]
        t0 = time.perf_counter()
        for i in small:
            g = models[i].meta["grid"]
            O.scattering_rates_grid(models[i], g, g, ks[i][:1], T_K, mus[i], 0.005)
        dt_cpu = time.perf_counter() - t0
        cb = {"value": 512 * len(small) / dt_cpu, "unit": "pairs/s", "cores": len(os.sched_getaffinity(0)),
              "kind": "oracle", "sample": f"1 k-point x 512 q of each of the {len(small)} first 8^3 instances "
                                          f"(FP64 NumPy oracle), {dt_cpu:.1f} s"}
    # algorithmic q-sum work: 8 FLOP per complex multiply-add, nR_p x (nmode nw^2) per (k, q) pair
    flops = sum(BATCH_K * int(np.prod(m.meta["grid"])) * len(m.R_gp) * m.nmode * m.nw ** 2 * 8 for m in models)
    fp32_peak = 152 * 128 * 2 * 2.07e9 / 1e12     # SMs x FP32 lanes x FMA x max clock, TFLOP/s
    # the same batch with the BF16x3 split: every (non-polar) instance takes its R_p sum on
    # the tensor cores
    from paper_2002_02045_gb300 import PGB_TC_BF16X3
    b.pgb_batch_set_precision(PGB_TC_BF16X3)
    outs_tc = [np.zeros_like(o) for o in outs]
    t0 = time.perf_counter()
    b.pgb_batch_rates(ks, T_K, mus, 0.005, outs_tc)
    t_first_tc = time.perf_counter() - t0
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(reps):
        b.pgb_batch_rates(ks, T_K, mus, 0.005, outs_tc)
    dt_tc = max_over_ranks((time.perf_counter() - t0) / reps, world)
    tc_inst = [True for m in models]       # every instance's R_p sum on the tensor cores
    flops_tc = sum(BATCH_K * int(np.prod(m.meta["grid"])) * len(m.R_gp) * m.nmode * m.nw ** 2 * 8
                   for m, e in zip(models, tc_inst) if e)
    dev = max(float(np.max(np.abs(x - y) / (np.abs(y) + 1e-6 * np.abs(y).max()))) for x, y in zip(outs_tc, outs))
    bf16 = {"value": world * pairs / dt_tc, "unit": "pairs/s", "ms_per_call": 1e3 * dt_tc,
            "first_call_s": t_first_tc, "tensor_core_instances": int(sum(tc_inst)),
            "tensor_core_flop_share": flops_tc / flops, "tuning": b.pgb_batch_tuning(),
            "tolerance_vs_fp64": 1e-3, "max_rel_dev_from_fp32_batch": dev}
    # and with the TF32x3 split: the FP32 tier (1e-5) on the tensor cores
    from paper_2002_02045_gb300 import PGB_TC_TF32X3
    b.pgb_batch_set_precision(PGB_TC_TF32X3)
    outs_tf = [np.zeros_like(o) for o in outs]
    b.pgb_batch_rates(ks, T_K, mus, 0.005, outs_tf)
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(reps):
        b.pgb_batch_rates(ks, T_K, mus, 0.005, outs_tf)
    dt_tf = max_over_ranks((time.perf_counter() - t0) / reps, world)
    dev_tf = max(float(np.max(np.abs(x - y) / (np.abs(y) + 1e-6 * np.abs(y).max()))) for x, y in zip(outs_tf, outs))
    tf32 = {"value": world * pairs / dt_tf, "unit": "pairs/s", "ms_per_call": 1e3 * dt_tf,
            "tuning": b.pgb_batch_tuning(), "tolerance_vs_fp64": 1e-5, "max_rel_dev_from_fp32_batch": dev_tf}
    b.close()
    for c in ctxs:
        c.close()
    return {
        "metric": "(k,q) pairs/s over uneven instances in one graph launch (FP32 products, FP64 energies)",
        "value": world * pairs / dt, "unit": "pairs/s", "ms_per_call": 1e3 * dt, "pairs": pairs,
        "instances": len(models), "k_per_instance": BATCH_K, "first_call_s": t_first,
        "model_generation_s": t_gen, "setup_s": t_setup, "tuning": tun, "finite": finite,
        "timing": "host clock around pgb_batch_rates (graph replay + output copies, synchronised)",
        "cpu_baseline": cb, "bf16x3": bf16, "tf32x3": tf32,
        "roofline": {"bound": "alu", "kernel": "batched graph (FP32): per-instance R_p sums on k_cgemm + the "
                                               "persistent warp epilogue k_batch_warp", "achieved": flops / dt / 1e12,
                     "peak": fp32_peak, "unit": "TFLOP/s", "frac": flops / dt / 1e12 / fp32_peak,
                     "algorithmic_flop": flops,
                     "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz (whole graph timed)"},
    }


def general_shape(args, world):
    """A shape the fused kernel does not cover: batched instance 44 (16 bands, 5 atoms =
    15 modes, 123 R vectors, 32^3 k = q grid), Gamma_nk of 16 k-points over the whole q
    grid at 300 K and 5 meV.  BF16x3: tensor-core q-sums in L2-sized q slabs, each read
    at once by the warp epilogue; FP32: the SIMT complex GEMM into HBM, then the SIMT
    epilogue.  Both timed with CUDA events over the whole call."""
    import torch
    import synthetic as S
    from paper_2002_02045_gb300 import PGB_FP32, PGB_TC_BF16X3, Context
    from paper_2002_02045_gb300.native import PROF_EPILOGUE, PROF_QSUM
    m = S.model_batch_instance(44)
    g = m.meta["grid"]
    ctx = Context(torch.cuda.current_device())
    ctx.pgb_set_model(m)
    ctx.pgb_set_grids(g, g)
    nk = int(np.prod(g))
    eps = torch.empty((nk, m.nw), dtype=torch.float64, device="cuda")
    ctx.pgb_get_grid_energies(eps, None)
    mu = float(0.5 * (eps.min() + eps.max()))
    kidx = torch.as_tensor(np.linspace(0, nk - 1, 16).astype(np.int32)).cuda()
    pairs = 16 * nk
    flop_per_pair = 8.0 * len(m.R_gp) * m.nmode * m.nw ** 2
    stream = torch.cuda.current_stream()
    out = {"workload": "batched-workload instance 44: 16 bands, 15 modes, 123 R_e x 123 R_p, 32^3 k = q grid, "
                       "16 k-points x all q, T = 300 K, sigma = 5 meV",
           "pairs": pairs, "algorithmic_flop_per_pair": flop_per_pair}
    peaks, _ = load_peaks()
    res = {}
    for name, prec in (("bf16x3", PGB_TC_BF16X3), ("fp32", PGB_FP32)):
        gam = torch.empty((16, m.nw), dtype=torch.float64, device="cuda")
        ctx.pgb_scattering_rates(kidx, T_K, mu, 0.005, prec, gam)
        torch.cuda.synchronize()
        ctx.pgb_profile(True)
        ctx.pgb_profile_read(PROF_QSUM)
        ctx.pgb_profile_read(PROF_EPILOGUE)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.pgb_scattering_rates(kidx, T_K, mu, 0.005, prec, gam)
        e1.record(stream)
        torch.cuda.synchronize()
        q_ms, q_n = ctx.pgb_profile_read(PROF_QSUM)
        p_ms, _ = ctx.pgb_profile_read(PROF_EPILOGUE)
        ctx.pgb_profile(False)
        ms = e0.elapsed_time(e1)
        res[name] = gam.cpu().numpy()
        out[name] = {"value": pairs / (ms * 1e-3), "unit": "pairs/s", "ms": ms, "q_sum_ms": q_ms,
                     "epilogue_ms": p_ms, "q_sum_launches": q_n}
    qb = out["bf16x3"]["q_sum_ms"]
    achieved = flop_per_pair * pairs / (qb * 1e-3) / 1e12
    peak = peaks["bf16_tflops"]
    out["bf16x3"]["roofline"] = {"bound": "tensor", "kernel": "k_tc_qsum (q slabs)", "achieved": achieved,
                                 "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                                 "issued_mma_frac": 3 * achieved / peak,
                                 "peak_source": "measured bf16 burst (short launches)"}
    y, x = res["bf16x3"], res["fp32"]
    out["bf16x3_vs_fp32_max_rel_dev"] = rel_err(y, x)
    ctx.close()
    return out


def e2e(ctx, model, prec, steps=1):
    """Same metric through the public API with host buffers: model upload,
    grids, window and rates, copies included."""
    import dataclasses
    import torch
    nk_grid = int(np.prod(KGRID))
    # the caller keeps its g~ table (the one large input) in pinned host memory
    g = torch.empty(model.g.shape, dtype=torch.complex64, pin_memory=True).numpy()
    g[...] = model.g
    model = dataclasses.replace(model, g=g)
    h2d = sum(np.asarray(a).nbytes for a in (model.mass, model.R_H, model.H, model.R_D, model.D, model.R_ge,
                                             model.R_gp, g))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        ctx.pgb_set_model(model)
        ctx.pgb_set_grids(KGRID, KGRID)
        eps = np.empty((nk_grid, model.nw))
        ctx.pgb_get_grid_energies(eps, None)
        emin = float(eps.min())
        kl = np.empty(nk_grid, np.int32)
        n = ctx.pgb_window(emin, emin + WIN, kl)
        gam = np.empty((n, model.nw))
        ctx.pgb_scattering_rates(np.ascontiguousarray(kl[:n]), T_K, emin - WIN, SIGMA, prec, gam)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / steps
    return {"value": n * nk_grid / dt, "unit": "pairs/s", "h2d_bytes_per_step": int(h2d + 4 * n),
            "d2h_bytes_per_step": int(eps.nbytes + 4 * n + gam.nbytes),
            "includes": "set_model (host validation + upload of g~ from pinned memory), set_grids, window, rates"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16x3", choices=["fp32", "fp64", "bf16x3", "tf32x3"])
    ap.add_argument("--no-batched", dest="batched", action="store_false",
                    help="skip the 64-instance batched-rates measurement")
    ap.add_argument("--no-polar", dest="polar", action="store_false",
                    help="skip the polar-model rates and transport measurement")
    ap.add_argument("--no-dynamics", dest="dynamics", action="store_false",
                    help="skip the real-time BTE (collision + RK4) measurement")
    ap.add_argument("--dyn-steps", type=int, default=1000)
    ap.add_argument("--adj-steps", type=int, default=1000,
                    help="reverse-mode RK4 steps timed on the dynamics list (0: skip)")
    ap.add_argument("--adj-checkpoint", type=int, default=50)
    ap.add_argument("--no-variants", dest="variants", action="store_false",
                    help="skip the one-step TF32x3 and FP32 SIMT measurements")
    ap.add_argument("--shard", action="store_true",
                    help="with several ranks, split the window k-points across them (strong scaling) "
                         "instead of one full workload per rank (weak scaling)")
    ap.add_argument("--dyn-grid", type=int, default=DYN_GRID[0],
                    help="k = q grid of the dynamics workload (smaller for profiling runs)")
    ap.add_argument("--batch-instances", type=int, default=BATCH_INSTANCES,
                    help="instances of the batched workload (fewer for profiling runs)")
    ap.add_argument("--max-k", type=int, default=0,
                    help="use only the first N window k-points (small case for profiler captures)")
    ap.add_argument("--no-e2e", dest="e2e", action="store_false")
    ap.add_argument("--batch-ids", default="",
                    help="comma-separated instance indices for the batched section (profiling subsets)")
    ap.add_argument("--no-general", dest="general", action="store_false",
                    help="skip the 16-band, 15-mode shape outside the fused kernel")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--mc-only", action="store_true",
                    help="in the polar section, run only the Monte-Carlo rates (profiling)")
    ap.add_argument("--kgrid", type=int, default=40, help="grid size per axis (40 = the workload; smaller "
                    "values give the small case used for profiler captures)")
    args = ap.parse_args()
    rank, world, local = dist_setup()
    global KGRID
    KGRID = (args.kgrid,) * 3
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
