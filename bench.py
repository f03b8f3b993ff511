"""Benchmark: Stokes solves/s on the 1024 x 1024 random-viscosity workload (one GPU per rank).

One step = one complete solve (hierarchy set-up + multigrid-preconditioned FGMRES to relative
energy residual 1e-10 + output) with the inputs already resident in HBM. Ranks solve independent
problems (replicas, weak scaling, no collective on the data path).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Stokes solves/s"
UNIT = "solves/s"
# headline solver options (FP64) and the mixed-precision line's: the weighted BFBt pressure block,
# pressure scaling alpha_p 0.8 and a 16 x 16 coarsest velocity level (fewer iterations on this field
# and on another seed of it), and the restart length that converges fastest at each precision; both
# meet the 1e-8 error bar at tol 1e-10
HEADLINE_OPTS = {"schur": 1, "restart_m": 80, "alpha_p": 0.8, "coarsest_min": 16}
MIXED_OPTS = {"schur": 1, "restart_m": 60, "alpha_p": 0.8, "coarsest_min": 16}
WORKLOAD = {"workload": "stokes2d_grf_1024", "nx": 1024, "ny": 1024, "box": [1.0, 1.0], "bc": "free_slip",
            "eta": "log10 eta clipped Gaussian random field, corr 0.05, [-2,2], seed 2",
            "rho": "1 + 32 density inclusions r~U[0.01,0.05], rho~U[0.9,1.1]", "g": [0.0, 1.0],
            "tol_rel_energy": 1e-10, "precision": "fp64", "global_batch": 1,
            "solver": ("FGMRES(80), Uzawa block preconditioner: velocity geometric-multigrid V(2,2) with RBGS down to "
                       "16 x 16, pressure block the weighted BFBt Schur approximation (two smoothed-aggregation "
                       "pressure V-cycles) scaled by 0.8; the paper's eta_c pressure block with FGMRES(30) is timed "
                       "beside it"),
            "l2": "working set per solve > L2 (Krylov basis ~1.5 GB) and L2 flushed (256 MB write) between steps",
            "parallelism": "replicas"}


def env_rank():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        import tempfile
        self.path = os.path.join(tempfile.gettempdir(), f"pyro_bench_clocks_rank{gpu_index}_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1])); smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def make_fields(n=1024):
    from synth import grf_config
    return grf_config(n, n, seed=2)


def oracle_baseline(workload, target_cells, sizes=(48, 64, 96), budget_s=25.0):
    """The FP64 CPU oracle (sparse direct solve of the assembled system) as it stands, timed on a
    bounded sample of the same generator at three sizes; the per-solve time is fitted as
    t = a N^b (N = cells) and extrapolated to the workload's cell count. SuperLU factorises on one
    thread; the fit exponent is reported (about 1.5-2 for these saddle-point systems)."""
    from oracle import stokes as S
    gen = {"layered": lambda n: __import__("synth").layered_config(n, n, seed=3),
           "grf": lambda n: __import__("synth").grf_config(n, n, seed=2)}[workload]
    rows = []
    t_all = time.perf_counter()
    for n in sizes:
        f = gen(n)
        ts = []
        while True:
            t0 = time.perf_counter()
            S.solve_fields(n, n, 1.0, 1.0, f.eta_n, f.eta_c, f.rho, (0.0, 1.0))
            ts.append(time.perf_counter() - t0)
            if sum(ts) > budget_s / (2 * len(sizes)) or len(ts) >= 5:
                break
        rows.append((n * n, float(np.median(ts)), len(ts)))
        if time.perf_counter() - t_all > budget_s:
            break
    N = np.array([r[0] for r in rows], dtype=float)
    T = np.array([r[1] for r in rows])
    b, loga = np.polyfit(np.log(N), np.log(T), 1) if len(rows) >= 2 else (1.0, np.log(T[0] / N[0]))
    t_target = float(np.exp(loga) * target_cells ** b)
    threads = len(os.sched_getaffinity(0))
    return {"value": 1.0 / t_target, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": (f"direct FP64 solves (SuperLU, COLAMD, 2 refinement steps) of the same {workload} generator at "
                       + ", ".join(f"{int(round(np.sqrt(r[0])))}^2 ({r[1]:.3f} s, median of {r[2]})" for r in rows)
                       + f"; fitted t = a N^{b:.2f} over cells N and extrapolated to {target_cells} cells; SuperLU "
                       f"factorises on one thread (host affinity {threads} threads)"),
            "fit_exponent": float(b), "sample_seconds": [r[1] for r in rows], "sample_cells": [r[0] for r in rows],
            "extrapolated_seconds_per_solve": t_target, "host_threads": threads}


def vcycle_roofline_4096(peaks, iters=6, label="", launches=1, **opts):
    """Level-0 FP32 V-cycle smoother kernels at 4096^2 (every level-0 array is 67 MB, far above
    L2), inside a mixed-precision solve of the layered workload. Each smoothing launch moves
    32 B/cell of algorithmic traffic (reads vx, vy, fx, fy, eta_n, eta_c, writes vx, vy): one RBGS
    sweep or two (tile kernels), one damped Jacobi sweep, or one RAS pass of `ras_inner` local
    Jacobi iterations. achieved = bytes / measured launch duration (CUDA events inside the solve,
    l0_pre_smooth phase / launches per pre-smoothing)."""
    import torch
    import paper_2603_14040_b300 as P
    from synth import layered_config
    n = 4096
    f = layered_config(n, n, seed=3)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    en, ec, rho = dev(f.eta_n), dev(f.eta_c), dev(f.rho)
    del f
    outs = [torch.zeros((n + 2, n + 2), dtype=torch.float64, device="cuda") for _ in range(3)]
    h = P.Stokes(n, n, prec=P.PREC_MIXED, max_iter=2, **opts)
    h.solve(en, ec, rho, (0.0, 1.0), 1e-10, *outs)           # warm-up (graph capture)
    h.close()
    h = P.Stokes(n, n, prec=P.PREC_MIXED, max_iter=iters, **opts)
    h.set_timing(True)
    h.solve(en, ec, rho, (0.0, 1.0), 1e-10, *outs)
    torch.cuda.synchronize()
    ph, cnt = h.get_timing()
    it = max(cnt["iterations"], 1)
    pre_ms = ph["l0_pre_smooth"] / it / launches
    cells = n * n
    bytes_pre = 32.0 * cells
    gbs_pre = bytes_pre / (pre_ms / 1e3) / 1e9
    peak = peaks.get("hbm_gbs", 6400.0)
    h.close()
    del outs, en, ec, rho
    torch.cuda.empty_cache()
    # the whole V-cycle against its algorithmic bytes: 208 B per fine cell for V(2,2) over all levels
    # when fused (FP32, per level: 32 B per RBGS sweep x 4 sweeps, 26 B for the residual-restriction,
    # about 2 B for the prolongation fused into the post-sweep, about 156 B, times 4/3 for the
    # coarser levels), scaled by the sweeps per level
    vcycle_ms = (ph["l0_pre_smooth"] + ph["coarse_levels"] + ph["l0_post_smooth"]) / it
    nu = opts.get("nu1", 2)
    vbytes = (208.0 + (nu - 2) * 2 * 32 * 4.0 / 3.0) * cells
    return {"kernel": f"{label} level 0, 4096x4096 layered, mixed", "opts": opts,
            "vcycle_alg_bytes": vbytes, "vcycle_GBps": vbytes / (vcycle_ms / 1e3) / 1e9,
            "vcycle_frac": vbytes / (vcycle_ms / 1e3) / 1e9 / peak,
            "bound": "hbm", "achieved": gbs_pre, "peak": peak, "unit": "GB/s", "frac": gbs_pre / peak,
            "peak_source": "MEASURED_PEAKS.json hbm_gbs" if "hbm_gbs" in peaks else "fallback 6400 GB/s",
            "bytes_per_launch": bytes_pre, "launch_ms": pre_ms,
            "vcycle_ms_per_iter": (ph["l0_pre_smooth"] + ph["coarse_levels"] + ph["l0_post_smooth"]) / it,
            "phase_ms_per_iter": {k: v / it for k, v in ph.items()}, "iters_timed": it}


def vcycle_rooflines(peaks):
    """The damped-Jacobi smoother's kernel (the paper's fully parallel smoother, one HBM pass per
    sweep) heads the object; the default RBGS tile kernels and the RAS-type pass are variants."""
    main = vcycle_roofline_4096(peaks, label="k_jacobi<float> (damped Jacobi sweep, smoother=JACOBI, omega 0.6)",
                                launches=2, smoother=1, omega_v=0.6)
    main["traffic"] = 518.10e6
    main["traffic_source"] = "ncu dram__bytes_read+write of one launch (profiles/k_jacobi_fp32_4096_level0.md)"
    main["sweeps_per_launch"] = 1
    main["variants"] = {}
    # sweeps: smoothing sweeps (RBGS) or local Jacobi iterations (RAS) one launch performs for its
    # one HBM pass; effective = sweeps x algorithmic bytes of one sweep / launch time
    for key, label, launches, sweeps, opts in [
            ("rbgs_tiles_2_sweeps_default", "k_rbgs_tile_w<2,48> (2 RBGS sweeps per launch, the default)", 1, 2,
             dict(tile_sweeps=2)),
            ("rbgs_tiles_1_sweep", "k_rbgs_tile_w<1,48> (1 RBGS sweep per launch)", 2, 1, dict(tile_sweeps=1)),
            ("ras_inner_2", "k_ras_tile<float,32,32> (RAS pass of 2 local Jacobi iterations)", 1, 2,
             dict(smoother=2, ras_inner=2, omega_v=0.6)),
            ("ras_inner_4", "k_ras_tile<float,32,32> (RAS pass of 4 local Jacobi iterations, the paper's T_inner)",
             1, 4, dict(smoother=2, ras_inner=4, omega_v=0.6))]:
        v = vcycle_roofline_4096(peaks, label=label, launches=launches, **opts)
        main["variants"][key] = {k: v[k] for k in ("kernel", "achieved", "frac", "launch_ms", "vcycle_ms_per_iter",
                                                   "vcycle_GBps", "vcycle_frac")}
        main["variants"][key].update({"sweeps_per_launch": sweeps, "effective_sweep_GBps": sweeps * v["achieved"],
                                      "effective_frac": sweeps * v["frac"]})
    return main


def accelerator_sample(f, n, steps=3):
    """The paper's own outer accelerators and smoothers on the bench workload (same 1e-10
    energy-residual stop): flexible GCR(30) and Anderson AA(m, beta) around the default
    preconditioner (FP64 and mixed), and the damped-Jacobi / RAS-type smoothers and the paper's
    "Mixed" smoother configuration (Jacobi on the finest level, RAS below; mixed precision)."""
    import torch
    import paper_2603_14040_b300 as P
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    en, ec, rho = dev(f.eta_n), dev(f.eta_c), dev(f.rho)
    outs = [torch.zeros((n + 2, n + 2), dtype=torch.float64, device="cuda") for _ in range(3)]
    res = {}
    for name, kw in [("gcr30", dict(accel=P.ACCEL_GCR, restart_m=30)),
                     ("anderson10_beta1", dict(accel=P.ACCEL_ANDERSON, restart_m=10, aa_beta=1.0)),
                     ("anderson15_beta0.8", dict(accel=P.ACCEL_ANDERSON, restart_m=15, aa_beta=0.8)),
                     ("fgmres30_jacobi_smoother", dict(smoother=P.SMOOTH_JACOBI, omega_v=0.6)),
                     ("fgmres30_ras4_smoother", dict(smoother=P.SMOOTH_RAS, ras_inner=4, omega_v=0.6)),
                     ("fgmres30_mixed_jacobi_ras4_smoother", dict(smoother=P.SMOOTH_MIXED, ras_inner=4, omega_v=0.6)),
                     ("anderson15_beta0.8_jacobi_smoother", dict(accel=P.ACCEL_ANDERSON, restart_m=15, aa_beta=0.8,
                                                                 smoother=P.SMOOTH_JACOBI, omega_v=0.6))]:
        for prec, pn in ((P.PREC_FP64, "fp64"), (P.PREC_MIXED, "mixed")):
            if "smoother" in name and prec == P.PREC_FP64:
                continue
            h = P.Stokes(n, n, prec=prec, max_iter=3000, **kw)
            h.solve(en, ec, rho, (0.0, 1.0), 1e-10, *outs)
            ts = []
            for _ in range(steps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record()
                st = h.solve(en, ec, rho, (0.0, 1.0), 1e-10, *outs)
                e1.record()
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            h.close()
            res[f"{name}_{pn}"] = {"solves_per_s": 1e3 / float(np.median(ts)), "ms": float(np.median(ts)),
                                   "iters": st.iters, "status": st.status, "rel_energy_res": st.rel_energy_res}
    return res


def layered_sample(n=1024, steps=3):
    """The layered workload's recipe (stiff lid 1e6, mantle 1 +- 50 %, 64 inclusions 10^U[-3,3]) at
    n x n, solved to 1e-10 with the options that converge on it: weighted BFBt pressure block, 5
    inner flexible-CG steps per preconditioner application, FGMRES(200), V(4,4); mixed (the block in
    FP32; and the block in FP64 after the FP32 V-cycle with the finest residual in FP64: schur 2,
    res64, the form that converges at 4096^2) and FP64."""
    import torch
    import paper_2603_14040_b300 as P
    from synth import layered_config
    f = layered_config(n, n, seed=3)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    en, ec, rho = dev(f.eta_n), dev(f.eta_c), dev(f.rho)
    outs = [torch.zeros((n + 2, n + 2), dtype=torch.float64, device="cuda") for _ in range(3)]
    res = {"grid": [n, n], "options": "schur=1 (weighted BFBt), inner_cg=5, restart_m=200, V(4,4), tol 1e-10"}
    sols = {}
    for prec, name, sc in ((P.PREC_MIXED, "mixed", 1), (P.PREC_MIXED, "mixed_schur2", 2), (P.PREC_FP64, "fp64", 1)):
        h = P.Stokes(n, n, prec=prec, schur=sc, inner_cg=5, restart_m=200, nu1=4, nu2=4, max_iter=3000,
                     res64=1 if sc == 2 else 0)
        h.solve(en, ec, rho, (0.0, 1.0), 1e-10, *outs)
        ts = []
        for _ in range(steps if name != "fp64" else 1):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            st = h.solve(en, ec, rho, (0.0, 1.0), 1e-10, *outs)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        sols[name] = [o.clone() for o in outs]
        res[name] = {"ms": float(np.median(ts)), "solves_per_s": 1e3 / float(np.median(ts)), "iters": st.iters,
                     "status": st.status, "rel_energy_res": st.rel_energy_res}
        h.close()
    c = sols["mixed_schur2"]
    res["rel_diff_mixed_schur2_vs_fp64_v"] = float(
        torch.linalg.norm(torch.cat([c[0].flatten(), c[1].flatten()]) - torch.cat([sols["fp64"][0].flatten(),
                                                                                   sols["fp64"][1].flatten()])) /
        torch.linalg.norm(torch.cat([sols["fp64"][0].flatten(), sols["fp64"][1].flatten()])))
    a, b = sols["mixed"], sols["fp64"]
    res["rel_diff_mixed_vs_fp64_v"] = float(torch.linalg.norm(torch.cat([a[0].flatten(), a[1].flatten()]) -
                                                              torch.cat([b[0].flatten(), b[1].flatten()])) /
                                            torch.linalg.norm(torch.cat([b[0].flatten(), b[1].flatten()])))
    res["rel_diff_mixed_vs_fp64_p"] = float(torch.linalg.norm(a[2] - b[2]) / torch.linalg.norm(b[2]))
    return res


def config3_sample(n=4096, max_iter=6000, restart_m=256, prec="mixed", schur=1, **extra):
    """Config 3 itself: the 4096^2 layered workload (lid 1e6 over a mantle with 64 inclusions of
    10^U[-3,3]) to relative energy residual 1e-10 with the weighted BFBt pressure block, 5 inner
    flexible-CG steps and FGMRES(restart_m), V(4,4). FP64 converges in 2527 iterations (284 s on a
    B300); mixed precision converges with the block in FP64 (schur 2) and the finest V-cycle residual
    in FP64 (res64) in 3072 iterations (253 s), the V-cycle otherwise FP32; with the block in FP32 it
    stalls near 6e-6. `extra` passes further solver options. One timed solve (it includes the graph
    captures); about 220 GB on the device at restart 256."""
    import torch
    import paper_2603_14040_b300 as P
    from synth import layered_config
    f = layered_config(n, n, seed=3)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    en, ec, rho = dev(f.eta_n), dev(f.eta_c), dev(f.rho)
    del f
    outs = [torch.zeros((n + 2, n + 2), dtype=torch.float64, device="cuda") for _ in range(3)]
    h = P.Stokes(n, n, prec=P.PREC_MIXED if prec == "mixed" else P.PREC_FP64, schur=schur, inner_cg=5,
                 restart_m=restart_m, nu1=4, nu2=4, max_iter=max_iter, **extra)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    st = h.solve(en, ec, rho, (0.0, 1.0), 1e-10, *outs)
    e1.record()
    torch.cuda.synchronize()
    res = {"grid": [n, n], "options": f"{prec}, schur={schur}, inner_cg=5, restart_m={restart_m}, V(4,4), tol 1e-10, {extra}",
           "ms": e0.elapsed_time(e1), "iters": st.iters, "restarts": st.restarts, "status": st.status,
           "rel_energy_res": st.rel_energy_res, "rel_l2_res": st.rel_l2_res,
           "footprint_GB": P.footprint(n, n, h.opts) / 1e9, "note": "first solve (includes the graph captures)"}
    h.close()
    del outs, en, ec, rho
    torch.cuda.empty_cache()
    return res


def marker_sample(n=1024, per_cell=16, reps=5):
    """The marker steps of the marker-in-cell loop around the solve: 16 markers per cell on 1024^2,
    uniform random positions; marker -> basic nodes (deterministic bucketed gather), grid -> markers
    (bilinear), and one advection step per scheme, CUDA events. Minimal traffic: 24 B per marker
    read (x, y, phi) for the scatter, 24 B per marker (x, y in, phi out) for the gather, 32 B per
    marker for advection."""
    import torch
    import paper_2603_14040_b300 as P
    m = per_cell * n * n
    g = torch.Generator(device="cuda").manual_seed(5)
    xm = torch.rand(m, dtype=torch.float64, device="cuda", generator=g)
    ym = torch.rand(m, dtype=torch.float64, device="cuda", generator=g)
    ph = torch.rand(m, dtype=torch.float64, device="cuda", generator=g)
    grid = torch.zeros((n + 2, n + 2), dtype=torch.float64, device="cuda")
    back = torch.zeros(m, dtype=torch.float64, device="cuda")
    mk = P.Markers(n, n, 1.0, 1.0, max_markers=m)
    res = {}
    for name, fn in (("markers_to_grid", lambda: mk.to_grid(P.LATTICE_NODES, xm, ym, ph, grid)),
                     ("grid_to_markers", lambda: mk.to_markers(P.LATTICE_NODES, xm, ym, grid, back))):
        fn()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        ms = float(np.median(ts))
        res[name] = {"ms": ms, "markers_per_s": m / (ms / 1e3), "min_traffic_GBps": 24.0 * m / (ms / 1e3) / 1e9}
    # advection in a cellular flow u = sin(pi x) cos(pi y), v = -cos(pi x) sin(pi y) sampled on the
    # staggered velocity lattices, one CFL-0.5 step per call (positions updated in place: 32 B per
    # marker of minimal traffic, the 2 x 8.4 MB velocity arrays stay in L2)
    h = 1.0 / n
    jj = torch.arange(n + 2, dtype=torch.float64, device="cuda")
    ii = jj.view(-1, 1)
    vx = torch.sin(np.pi * jj * h) * torch.cos(np.pi * (ii - 0.5) * h)
    vy = -torch.cos(np.pi * (jj - 0.5) * h) * torch.sin(np.pi * ii * h)
    dt = mk.max_dt(vx, vy, 0.5)
    for name, scheme in (("advect_euler", P.ADVECT_EULER), ("advect_heun", P.ADVECT_HEUN), ("advect_rk4", P.ADVECT_RK4),
                         ("advect_taylor", P.ADVECT_TAYLOR)):
        mk.advect(xm, ym, vx, vy, dt, scheme=scheme)
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            mk.advect(xm, ym, vx, vy, dt, scheme=scheme)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        ms = float(np.median(ts))
        res[name] = {"ms": ms, "markers_per_s": m / (ms / 1e3), "min_traffic_GBps": 32.0 * m / (ms / 1e3) / 1e9}
    mk.close()
    res["markers"] = m
    res["grid"] = [n, n]
    return res


def sinker_e1_sample():
    """The robustness sinker at the paper's grid (501 x 601 nodes = 500 x 600 cells, box 1 x 1.2,
    contrast 1e8, density contrast 1.03125), mixed precision, lithostatic start, tol 1e-8: the
    default hierarchy (halving, then ratio-2 general coarsening) and the paper's ratio 2.5; then the
    paper's four smoother configurations (RBGS, damped Jacobi, RAS-type with T_inner 4, and "Mixed")
    at its relaxation factors omega_v = 0.3, omega_p (alpha_p) = 0.6, inside FGMRES(30); and the
    viscosity-contrast continuation (4 stages of 25 outer iterations at eta_comp = (1 - theta)
    eta_min + theta eta before the full-contrast solve) with the default and the paper's smoother
    settings (iters and levels describe the final full-contrast solve; the stages add at most
    4 x 25 outer iterations, and ms covers the whole call)."""
    import torch
    import paper_2603_14040_b300 as P
    from synth import sinker
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    nx, ny = 500, 600
    f = sinker(nx, ny, 1.0, 1.2, eta_bg=1.0, rho_bg=1.0, eta_inc=1e8, rho_inc=1.03125, r=0.2)
    en, ec, rho = dev(f.eta_n), dev(f.eta_c), dev(f.rho)
    outs = [torch.zeros((ny + 2, nx + 2), dtype=torch.float64, device="cuda") for _ in range(3)]
    res = {}
    relax = {"omega_v": 0.3, "alpha_p": 0.6, "ras_inner": 4}
    for name, kw in (("ratio2_default", {}), ("ratio2.5", {"coarsen_ratio": 2.5}),
                     ("ratio2.5_restart100", {"coarsen_ratio": 2.5, "restart_m": 100}),
                     ("paper_relaxation_rbgs", dict(relax, smoother=P.SMOOTH_RBGS)),
                     ("paper_relaxation_jacobi", dict(relax, smoother=P.SMOOTH_JACOBI)),
                     ("paper_relaxation_ras4", dict(relax, smoother=P.SMOOTH_RAS)),
                     ("paper_relaxation_mixed", dict(relax, smoother=P.SMOOTH_MIXED)),
                     ("continuation_4x25", {"cont_stages": 4, "cont_iters": 25}),
                     ("continuation_4x25_paper_relaxation_rbgs", dict(relax, smoother=P.SMOOTH_RBGS,
                                                                       cont_stages=4, cont_iters=25))):
        h = P.Stokes(nx, ny, 1.0, 1.2, prec=P.PREC_MIXED, max_iter=3000, litho_guess=1, **kw)
        h.solve(en, ec, rho, (0.0, 1.0), 1e-8, *outs)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        st = h.solve(en, ec, rho, (0.0, 1.0), 1e-8, *outs)
        e1.record()
        torch.cuda.synchronize()
        res[name] = {"ms": e0.elapsed_time(e1), "iters": st.iters, "status": st.status, "levels": st.levels,
                     "rel_energy_res": st.rel_energy_res}
        h.close()
    return res


def serving_sample(n_req=48, slots=4, max_iter=3000, restart_m=200, seed=4, nu=8):
    """Continuous batching on a bounded sample of the serving workload: requests with n in
    {128, 256, 512}, aspect in {1, 2, 4}, 16 inclusions of contrast 10^U[2,6], tol 1e-8, Poisson
    arrivals at 0.8 x the measured single-slot service rate; mixed precision, FGMRES with the
    longest restart (<= 200) whose handle fits a quarter of the device budget, V(nu, nu) cycles
    (on these sharp-inclusion requests 8 sweeps per level halve the total solve time of V(2, 2):
    fewer iterations of the long-restart FGMRES outweigh the cheaper cycles)."""
    import torch
    from synth import serving_request
    from paper_2603_14040_b300.serving import SolveServer, Request, PyroBackend, latency_stats, poisson_arrivals
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    reqs = []
    for k in range(n_req):
        f, C = serving_request(k, base_seed=seed, sizes=(128, 256, 512))
        reqs.append((Request(rid=k, nx=f.nx, ny=f.ny, Lx=f.Lx, Ly=f.Ly, eta_n=dev(f.eta_n), eta_c=dev(f.eta_c),
                             rho=dev(f.rho), g=(0.0, 1.0), tol=1e-8), C))
    be = PyroBackend(opts_kw={"max_iter": max_iter, "prec": 1, "nu1": nu, "nu2": nu},
                     restart_choices=tuple(m for m in (restart_m, 100, 50, 30) if m <= restart_m))
    # service rate from a sequential pass over the first requests (also warms the handle pool)
    srv = SolveServer(be, max_slots=1)
    t0 = time.perf_counter()
    probe = 8
    for r, _ in reqs[:probe]:
        srv.submit(Request(**{k: getattr(r, k) for k in ("rid", "nx", "ny", "Lx", "Ly", "eta_n", "eta_c", "rho",
                                                          "g", "tol")}))
    srv.drain(timeout=600)
    srv.close()
    mean_service = (time.perf_counter() - t0) / probe
    rate = 0.8 / mean_service
    arr = poisson_arrivals(n_req, rate, seed)
    srv = SolveServer(be, max_slots=slots)
    t_start = time.perf_counter()
    for (r, _), a in zip(reqs, arr):
        while time.perf_counter() - t_start < a:
            time.sleep(0.0005)
        r.arrival = 0.0
        srv.submit(r)
    done = srv.drain(timeout=1800)
    srv.close()
    st = latency_stats(done)
    conv = sum(1 for r in done if r.status == 0)
    st.update({"requests": n_req, "slots": slots, "arrival_rate_per_s": rate, "mean_single_service_ms":
               mean_service * 1e3, "converged_to_tol": conv, "not_converged_at_max_iter": n_req - conv,
               "max_iter": max_iter, "cycle": f"V({nu},{nu})", "max_concurrent": srv.max_concurrent,
               "mean_iters": float(np.mean([r.iters for r in done]))})
    return st


def serving_sweep(n_req=40, slots=4, sizes=(128, 256, 512, 1024), seed=4, nu=8, max_iter=3000):
    """Serving on the config-4 request distribution (ny = n, nx = a n, a in {1, 2, 4}, 16 inclusions of
    contrast 10^U[2,6], tol 1e-8), n restricted to `sizes` (the 2048 rows of the distribution need
    handles of up to 170 GB each, more than a 4-slot share of the device). Measures: the
    single-slot service capacity (sequential pass, warm handle pool); saturation throughput with all
    requests submitted at once on 1 slot and on `slots` slots (the device overlap of concurrent
    solves); and p50 / p99 latency and throughput for Poisson arrivals at 0.5, 0.8, 1.0 and 1.2 x
    the single-slot capacity."""
    import torch
    from synth import serving_request
    from paper_2603_14040_b300.serving import SolveServer, Request, PyroBackend, latency_stats, poisson_arrivals
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    src = []
    for k in range(n_req):
        f, C = serving_request(k, base_seed=seed, sizes=sizes)
        src.append((f, C))

    def fresh():
        return [Request(rid=k, nx=f.nx, ny=f.ny, Lx=f.Lx, Ly=f.Ly, eta_n=dev(f.eta_n), eta_c=dev(f.eta_c),
                        rho=dev(f.rho), g=(0.0, 1.0), tol=1e-8) for k, (f, C) in enumerate(src)]

    be = PyroBackend(opts_kw={"max_iter": max_iter, "prec": 1, "nu1": nu, "nu2": nu},
                     restart_choices=(200, 100, 50, 30))
    out = {"requests": n_req, "sizes": list(sizes), "aspects": [1, 2, 4], "cycle": f"V({nu},{nu})",
           "cells_total": int(sum(f.nx * f.ny for f, _ in src))}
    # warm pass (creates and captures every shape's handle), then the timed sequential pass
    for label, nslots in (("warm", 1), ("sequential", 1)):
        srv = SolveServer(be, max_slots=nslots)
        reqs = fresh()
        t0 = time.perf_counter()
        for r in reqs:
            srv.submit(r)
            srv.drain(timeout=3600)
        dt = time.perf_counter() - t0
        srv.close()
        if label == "sequential":
            out["single_slot_capacity_per_s"] = n_req / dt
            out["converged"] = sum(1 for r in reqs if r.status == 0)
            out["mean_iters"] = float(np.mean([r.iters for r in reqs]))
    cap = out["single_slot_capacity_per_s"]
    for nslots in (1, slots):
        srv = SolveServer(be, max_slots=nslots)
        reqs = fresh()
        t0 = time.perf_counter()
        for r in reqs:
            srv.submit(r)
        srv.drain(timeout=3600)
        dt = time.perf_counter() - t0
        srv.close()
        out[f"saturation_{nslots}_slots"] = {"throughput_per_s": n_req / dt, "max_concurrent": srv.max_concurrent}
    out["overlap_speedup"] = (out[f"saturation_{slots}_slots"]["throughput_per_s"] /
                              out["saturation_1_slots"]["throughput_per_s"])
    out["arrival_sweep"] = {}
    for frac in (0.5, 0.8, 1.0, 1.2):
        rate = frac * cap
        arr = poisson_arrivals(n_req, rate, seed)
        srv = SolveServer(be, max_slots=slots)
        reqs = fresh()
        t_start = time.perf_counter()
        for r, a in zip(reqs, arr):
            while time.perf_counter() - t_start < a:
                time.sleep(0.0005)
            r.arrival = 0.0
            srv.submit(r)
        done = srv.drain(timeout=3600)
        srv.close()
        st = latency_stats(done)
        st.update({"arrival_rate_per_s": rate, "max_concurrent": srv.max_concurrent,
                   "converged": sum(1 for r in done if r.status == 0)})
        out["arrival_sweep"][f"{frac}x"] = st
    return out


def serving_large_sample(seed=4, per_aspect=1, slots=4, nu=8, max_iter=3000):
    """The n = 2048 rows of the serving distribution (ny = 2048, nx = a 2048, a in {1, 2, 4}: up to
    16.8 M cells, 16 inclusions of contrast 10^U[2,6], tol 1e-8), served through the same server with
    the whole memory budget open to one handle, so every request gets FGMRES(200) (up to 170 GB) and
    the footprint admission runs one such request at a time. Reports per request: size, contrast,
    restart, footprint, iterations, status (0: converged to tol) and the latency of the first solve of
    its shape (handle creation and graph capture included) and of a second solve on the warm handle."""
    import torch
    from synth import serving_request
    from paper_2603_14040_b300.serving import SolveServer, Request, PyroBackend
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    be = PyroBackend(opts_kw={"max_iter": max_iter, "prec": 1, "nu1": nu, "nu2": nu},
                     restart_choices=(200, 100, 50, 30), per_handle_bytes=None)
    be.per_handle_bytes = be.default_budget()
    rows = []
    k = 0
    for a in (1, 2, 4):
        for r in range(per_aspect):
            f, C = serving_request(10_000 + k, base_seed=seed, force_n=2048, force_a=a)
            k += 1
            shape = (f.nx, f.ny, f.Lx, f.Ly)
            rec = {"nx": f.nx, "ny": f.ny, "contrast": float(C), "restart_m": be.opts_for(shape)["restart_m"],
                   "footprint_GB": be.footprint(shape) / 1e9}
            srv = SolveServer(be, max_slots=slots)
            for label in ("first", "warm"):
                req = Request(rid=k, nx=f.nx, ny=f.ny, Lx=f.Lx, Ly=f.Ly, eta_n=dev(f.eta_n), eta_c=dev(f.eta_c),
                              rho=dev(f.rho), g=(0.0, 1.0), tol=1e-8)
                srv.submit(req)
                srv.drain(timeout=3600)
                rec[f"latency_ms_{label}"] = req.latency * 1e3
                rec[f"iters_{label}"] = req.iters
                rec[f"status_{label}"] = req.status
                req.result = None
            srv.close()
            rows.append(rec)
            print(json.dumps({"serving_large_row": rec}), flush=True)
            del f
            torch.cuda.empty_cache()
    return {"requests": rows, "cycle": f"V({nu},{nu})", "tol": 1e-8,
            "note": "n = 2048 rows of the serving distribution; one handle may take the whole budget"}


def adjoint_sample(members=64, n=512, slots=4, opts=None):
    """The adjoint batch: 64 members on 512^2 (log10 eta random fields, seeds 500..563), each a forward
    solve, J = 1/2 |vx(top row) - vx_obs|^2, an adjoint solve and the strain-rate products, chained to
    dJ/dlog(eta) (dJ/dlog eta = eta dJ/deta; the same arithmetic as the torch.autograd.Function, called
    directly so that members on different handles run concurrently instead of queueing behind the
    autograd engine's device thread). Members are spread over `slots` handles, each on its own host
    thread and CUDA stream; the batch is also run on one slot. The observation solves (eta perturbed
    by 10^(0.1 xi)) are outside the timed region. Mixed precision, tol 1e-10, with the mixed
    headline's weighted BFBt options (the adjoint solve uses the forward solve's operator and
    preconditioner); the batch on `slots` handles with the paper's eta_c block is timed beside it."""
    opts = dict(MIXED_OPTS if opts is None else opts)
    import threading
    import torch
    import paper_2603_14040_b300 as P
    from synth import adjoint_member
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    data = []
    hobs = P.Stokes(n, n, prec=P.PREC_MIXED, max_iter=3000, **opts)
    for b in range(members):
        base, pert = adjoint_member(b, n, n)
        obs = [torch.zeros((n + 2, n + 2), dtype=torch.float64, device="cuda") for _ in range(3)]
        hobs.solve(dev(pert.eta_n), dev(pert.eta_c), dev(pert.rho), (0.0, 1.0), 1e-10, *obs)
        data.append((dev(base.eta_n), dev(base.eta_c), dev(base.rho), obs[0][1].clone()))
    hobs.close()
    torch.cuda.synchronize()

    def member(h, stream, b, rec):
        en, ec, rho, vx_obs = data[b]
        with torch.cuda.stream(stream):
            t0 = time.perf_counter()
            out = [torch.zeros((n + 2, n + 2), dtype=torch.float64, device="cuda") for _ in range(3)]
            sf = h.solve(en, ec, rho, (0.0, 1.0), 1e-10, *out, stream=stream)
            d = torch.zeros_like(out[0])
            d[1, 1:n] = out[0][1, 1:n] - vx_obs[1:n]
            zero = torch.zeros_like(d)
            gn, gc = torch.zeros_like(d), torch.zeros_like(d)
            sa = h.adjoint(d, zero, zero, 1e-10, gn, gc, None, stream=stream)
            glog_c = gc * ec
            glog_n = gn * en
            gnorm = float(torch.linalg.norm(glog_c))
            stream.synchronize()
            rec[b] = {"ms": (time.perf_counter() - t0) * 1e3, "fwd_iters": sf.iters, "adj_iters": sa.iters,
                      "grad_norm": gnorm, "grad_n_norm": float(torch.linalg.norm(glog_n))}

    def run(nslots, o=opts):
        hs = [P.Stokes(n, n, prec=P.PREC_MIXED, max_iter=3000, **o) for _ in range(nslots)]
        ss = [torch.cuda.Stream() for _ in range(nslots)]
        rec = {}
        for k in range(nslots):       # warm-up: capture each handle's iteration graph
            member(hs[k], ss[k], k, {})
        torch.cuda.synchronize()
        t0 = time.perf_counter()

        def worker(k):
            for b in range(k, members, nslots):
                member(hs[k], ss[k], b, rec)
        th = [threading.Thread(target=worker, args=(k,)) for k in range(nslots)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        wall = time.perf_counter() - t0
        for h in hs:
            h.close()
        return wall, rec

    wall1, rec1 = run(1)
    wallk, reck = run(slots)
    wallp, recp = run(slots, {})
    ms = np.array([reck[b]["ms"] for b in range(members)])
    its = np.array([reck[b]["fwd_iters"] + reck[b]["adj_iters"] for b in range(members)])
    slow = int(np.argmax([rec1[b]["ms"] for b in range(members)]))
    itp = np.array([recp[b]["fwd_iters"] + recp[b]["adj_iters"] for b in range(members)])
    return {"members": members, "grid": n, "slots": slots, "solver_opts": opts, "batch_s": wallk,
            "batch_s_one_slot": wall1,
            "paper_block": {"batch_s": wallp, "members_per_s": members / wallp,
                            "iters_fwd_plus_adj_p50": float(np.median(itp))},
            "overlap_speedup": wall1 / wallk, "members_per_s": members / wallk,
            "ms_per_member_one_slot": {"p50": float(np.percentile([rec1[b]["ms"] for b in range(members)], 50)),
                                       "max": float(max(rec1[b]["ms"] for b in range(members)))},
            "iters_fwd_plus_adj": {"min": int(its.min()), "p50": float(np.median(its)), "max": int(its.max())},
            "slowest_member_one_slot": {"member": slow, **rec1[slow]},
            "ms_in_mix": {"p50": float(np.percentile(ms, 50)), "max": float(ms.max())},
            "grad_norm_log_eta_c_range": [float(min(r["grad_norm"] for r in reck.values())),
                                          float(max(r["grad_norm"] for r in reck.values()))],
            "note": "graphs captured before timing; observation solves outside the timed region"}


def paper_block_sample(one_solve, outs, flush, stream, n, world, steps):
    """The same workload with the paper's own pressure block (the diagonal viscosity surrogate eta_c)
    and FGMRES(30), FP64 and mixed: solves/s, iterations and the difference from the headline
    solution."""
    import torch
    import paper_2603_14040_b300 as P
    res = {"options": "schur=0 (eta_c block), restart_m=30"}
    for name, prec in (("fp64", P.PREC_FP64), ("mixed", P.PREC_MIXED)):
        hp = P.Stokes(n, n, prec=prec, max_iter=3000)
        o = [torch.zeros_like(a) for a in outs]
        st = one_solve(hp, o)
        ms = []
        for k in range(steps):
            flush.fill_(float(k))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = one_solve(hp, o)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        dv = float(torch.linalg.norm(o[0] - outs[0]) / torch.linalg.norm(outs[0]))
        res[name] = {"solves_per_s": world * 1e3 / float(np.mean(ms)), "ms": float(np.mean(ms)), "iters": st.iters,
                     "rel_energy_res": st.rel_energy_res, "rel_diff_vs_headline_v": dv}
        hp.close()
    return res


def profile_solve(args):
    """One solve (for ncu captures): the random-viscosity or layered workload at N x N, given
    precision, restart length, iteration cap and preconditioner options; prints a one-line summary."""
    import torch
    import paper_2603_14040_b300 as P
    from synth import grf_config, layered_config
    n = args.profile
    f = layered_config(n, n, seed=3) if args.workload == "layered" else grf_config(n, n, seed=2)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    en, ec, rho = dev(f.eta_n), dev(f.eta_c), dev(f.rho)
    outs = [torch.zeros((n + 2, n + 2), dtype=torch.float64, device="cuda") for _ in range(3)]
    prec = P.PREC_MIXED if args.prec == "mixed" else P.PREC_FP64
    h = P.Stokes(n, n, prec=prec, max_iter=args.max_iter, restart_m=args.restart, tile_fusion=args.tile_fusion,
                 tile_sweeps=args.tile_sweeps, smoother=args.smoother, omega_v=args.omega, accel=args.accel,
                 schur=args.schur, inner_cg=args.inner_cg, res64=args.res64, nu1=args.nu, nu2=args.nu,
                 alpha_p=args.alpha_p, coarsest_min=args.coarsest_min)
    st = h.solve(en, ec, rho, (0.0, 1.0), 1e-10, *outs)
    torch.cuda.synchronize()
    print(json.dumps({"profile_solve": n, "workload": args.workload, "prec": args.prec, "iters": st.iters,
                      "status": st.status, "kernel_launches": st.kernel_launches}))


def run_reference(args, rank, world):
    """The reference arm of this workload: the FP64 CPU oracle as it stands (direct solve of the
    assembled system) on rank 0's host cores. Each step is one direct solve of the same generator at
    96^2; the power-law exponent of the solve time over the cell count is fitted once from solves at
    48^2 and 64^2 (untimed), and the step time is extrapolated to the workload's cell count with it."""
    if rank != 0:
        return
    from oracle import stokes as S
    from synth import grf_config
    calib = []
    for m in (48, 64):
        f = grf_config(m, m, seed=2)
        t0 = time.perf_counter()
        S.solve_fields(m, m, 1.0, 1.0, f.eta_n, f.eta_c, f.rho, (0.0, 1.0))
        calib.append((m * m, time.perf_counter() - t0))
    n = 96
    f = grf_config(n, n, seed=2)
    times = []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        S.solve_fields(n, n, 1.0, 1.0, f.eta_n, f.eta_c, f.rho, (0.0, 1.0))
        if k >= args.warmup:
            times.append(time.perf_counter() - t0)
    dt = float(np.mean(times))
    pts = calib + [(n * n, float(np.median(times)))]
    b = float(np.polyfit(np.log([p[0] for p in pts]), np.log([p[1] for p in pts]), 1)[0])
    target = WORKLOAD["nx"] * WORKLOAD["ny"]
    t_target = dt * (target / (n * n)) ** b
    value = 1.0 / t_target
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_target * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": WORKLOAD,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": (f"each step one direct FP64 solve (SuperLU, one thread) of the same generator at "
                                        f"{n}x{n} ({dt:.3f} s mean); time extrapolated to {target} cells with the "
                                        f"fitted exponent {b:.2f} (from 48^2, 64^2, 96^2)")},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def job_throughput(local_ms, steps, world, device):
    """Whole-job throughput of independent replicas: every rank ran `steps` solves in local_ms; the
    job took the slowest rank's time (max over ranks), and all ranks' solves count."""
    total_ms = local_ms
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([local_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return world * steps / (total_ms / 1e3), total_ms


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the 4096^2, serving and adjoint samples")
    ap.add_argument("--profile", type=int, default=0, metavar="N",
                    help="profiling driver: one solve of the random-viscosity workload at N x N, then exit")
    ap.add_argument("--prec", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--max-iter", type=int, default=3000)
    ap.add_argument("--restart", type=int, default=30)
    ap.add_argument("--tile-fusion", type=int, default=1, help="pyro_opts.tile_fusion of the --profile solve")
    ap.add_argument("--tile-sweeps", type=int, default=2, help="pyro_opts.tile_sweeps of the --profile solve")
    ap.add_argument("--smoother", type=int, default=0, help="pyro_opts.smoother of the --profile solve")
    ap.add_argument("--omega", type=float, default=1.0, help="pyro_opts.omega_v of the --profile solve")
    ap.add_argument("--accel", type=int, default=0, help="pyro_opts.accel of the --profile solve")
    ap.add_argument("--workload", default="grf", choices=["grf", "layered"], help="field of the --profile solve")
    ap.add_argument("--schur", type=int, default=0,
                    help="pyro_opts.schur of the --profile solve; of the --config3 solve when non-zero")
    ap.add_argument("--inner-cg", type=int, default=0, help="pyro_opts.inner_cg of the --profile solve")
    ap.add_argument("--res64", type=int, default=0, help="pyro_opts.res64 of the --profile solve")
    ap.add_argument("--nu", type=int, default=2, help="pre/post smoothing sweeps of the --profile solve")
    ap.add_argument("--alpha-p", type=float, default=1.0, help="pyro_opts.alpha_p of the --profile solve")
    ap.add_argument("--coarsest-min", type=int, default=4, help="pyro_opts.coarsest_min of the --profile solve")
    ap.add_argument("--serving-sweep", action="store_true",
                    help="only the serving measurement on the config-4 request distribution (n <= 1024): capacity, "
                         "1-slot vs 4-slot saturation, arrival-rate sweep")
    ap.add_argument("--serving-large", action="store_true",
                    help="serve the n = 2048 rows of the serving distribution (one request per aspect) and exit")
    ap.add_argument("--config3", action="store_true",
                    help="only config 3 (4096^2 layered, mixed, weighted BFBt + inner CG): one solve, about 170 GB")
    ap.add_argument("--markers", action="store_true",
                    help="only the marker sample (16.8 M markers on 1024^2: interpolation both ways and one "
                         "advection step per scheme), for ncu captures")
    args = ap.parse_args()
    rank, world, local = env_rank()
    import torch
    import torch.distributed as dist
    if args.profile:
        return profile_solve(args)
    if args.markers:
        print(json.dumps({"markers": marker_sample(reps=1)}))
        return
    if args.config3:
        # mixed precision keeps the pressure block in FP64 (schur 2) unless --schur says otherwise,
        # and forms its finest V-cycle residual in FP64 (res64)
        sc = args.schur if args.schur else (2 if args.prec == "mixed" else 1)
        extra = {"res64": 1} if args.prec == "mixed" else {}
        print(json.dumps({"config3": config3_sample(prec=args.prec, schur=sc, **extra)}))
        return
    if args.serving_sweep:
        print(json.dumps({"serving_sweep": serving_sweep()}))
        return
    if args.serving_large:
        print(json.dumps({"serving_large": serving_large_sample()}))
        return
    if args.impl == "reference":
        # the oracle runs on rank 0's host cores; the other ranks exit without work
        run_reference(args, rank, world)
        return
    if torch.cuda.is_available():
        torch.cuda.set_device(local)
    if world > 1 and not dist.is_initialized():
        if torch.cuda.is_available():
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group("gloo")

    import paper_2603_14040_b300 as P
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    f = make_fields(1024)
    n = 1024
    g_vec = (0.0, 1.0)
    tol = WORKLOAD["tol_rel_energy"]
    d_en, d_ec, d_rho = dev(f.eta_n), dev(f.eta_c), dev(f.rho)
    outs = [torch.zeros((n + 2, n + 2), dtype=torch.float64, device="cuda") for _ in range(3)]
    h = P.Stokes(n, n, prec=P.PREC_FP64, max_iter=3000, **HEADLINE_OPTS)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2
    stream = torch.cuda.current_stream()

    def one_solve(handle, o=outs):
        st = handle.solve(d_en, d_ec, d_rho, g_vec, tol, *o)
        if st.status != 0:
            raise RuntimeError(f"solve status {st.status}")
        return st

    for _ in range(args.warmup):
        one_solve(h)
    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms, stats = [], []
    for k in range(args.steps):
        flush.fill_(float(k))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        stats.append(one_solve(h))
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    value, total_ms = job_throughput(float(np.sum(step_ms)), args.steps, world, "cuda")
    # phase breakdown (CUDA events at the phase boundaries inside the captured iteration) from one
    # more solve outside the timed region, so the timed solves carry no timing events
    h.set_timing(True)
    one_solve(h)     # captures the iteration graph with the timing events
    h.set_timing(True)
    one_solve(h)
    torch.cuda.synchronize()
    phases, counts = h.get_timing()
    h.set_timing(False)

    # end to end through the public API with host (pinned) buffers: H2D of the inputs and D2H of
    # the solution happen inside the C-ABI call
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    h_en, h_ec, h_rho = pin(f.eta_n), pin(f.eta_c), pin(f.rho)
    h_out = [torch.zeros((n + 2, n + 2), dtype=torch.float64).pin_memory() for _ in range(3)]
    h.solve(h_en, h_ec, h_rho, g_vec, tol, *h_out)     # warm-up (re-captures the graph without timing)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_steps = max(2, args.steps // 2)
    for _ in range(e2e_steps):
        st = h.solve(h_en, h_ec, h_rho, g_vec, tol, *h_out)
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    plane = (n + 2) * (n + 2) * 8
    e2e = {"value": world / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 3 * plane, "d2h_bytes_per_step": 3 * plane,
           "api": "pyro_stokes_solve with host pointers (library stages the copies)"}

    # roofline of the FP64 smoother (the largest share after the Gram-Schmidt step): finest-level RBGS sweep (4 launches vx-red, vx-black, vy-red,
    # vy-black), FP64. Algorithmic per cell and sweep: read eta_n, eta_c, fx, fy, vx, vy + write vx,
    # vy = 64 B in FP64; arithmetic: per velocity point the off-diagonal sum on precomputed
    # coefficients (6 products, 2 differences, 5 sums) and the update (2) = 15 flop, 30 per cell.
    # B300's FP64 rate binds it, so the bound is the FP64 rate measured in this run.
    peaks = load_peaks()
    sweeps = max(counts["l0_sweeps"], 1)
    sweep_ms = (phases["l0_pre_smooth"] + phases["l0_post_smooth"]) / sweeps
    cells = n * n
    bytes_per_sweep = 64 * cells
    flops_per_sweep = 30 * cells
    achieved_flops = flops_per_sweep / (sweep_ms / 1e3) / 1e12
    fp64_peak = P.fp64_fma_rate()
    sm_mhz = clk.get("sm_mhz") or 2032.0
    fp64_derived = 148 * 2.08 * 2 * sm_mhz * 1e6 / 1e12
    hbm_peak = peaks.get("hbm_gbs", 6400.0)
    hbm_achieved = bytes_per_sweep / (sweep_ms / 1e3) / 1e9
    roof = {"kernel": "k_rbgs<double> finest level (one sweep = 4 launches; the largest share after k_mgs_step)",
            "bound": "alu",
            "achieved": achieved_flops, "peak": fp64_peak, "unit": "TFLOP/s", "frac": achieved_flops / fp64_peak,
            "peak_source": "FP64 FMA rate measured in this run (pyro_fp64_fma_rate: FMA chains, CUDA events), of measured",
            "traffic": 4 * 59.579e6, "traffic_unit": "B per sweep",
            "traffic_source": "ncu dram__bytes_read+write of the level-0 vx-red launch (59.58 MB, profiles/k_rbgs_fp64_1024_level0.md) x 4 half-sweeps",
            "fp64_pipe_active_pct_ncu": 78.1, "flop_per_cell_sweep": 30, "alg_bytes_per_cell_sweep": 64,
            "peak_derived": fp64_derived, "frac_of_derived": achieved_flops / fp64_derived,
            "peak_derived_source": ("148 SMs x 2.08 FP64 FMA per clock per SM (the nominal 1.25 TFLOP/s at 2032 MHz) x 2 flop "
                                    f"x the median SM clock sampled during the timed region ({sm_mhz:.0f} MHz)"),
            "hbm": {"achieved_GBps": hbm_achieved, "peak_GBps": hbm_peak, "frac": hbm_achieved / hbm_peak,
                    "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if "hbm_gbs" in peaks else "fallback 6400 GB/s"},
            "sweep_ms": sweep_ms, "phase_ms_per_iter": {k: v / max(counts["iterations"], 1) for k, v in phases.items()}}

    # dominant kernel of the headline solve: the modified Gram-Schmidt step k_mgs_step (ncu launch list
    # of the whole solve, profiles/launches_grf1024_bfbt_fp64.md). One step reads w, v_{k-1}, v_k and
    # writes w: 4 vectors of n3 = 3 (ny + 2)(nx + 2) doubles (algorithmic; w and v_{k-1} may be served
    # from L2, so DRAM traffic can be lower); 2 FP64 FMA per entry. Column j of a restart cycle
    # takes min(j + 2, m + 1) steps; the column's closing k_scale_next moves 2 more vectors.
    it_t = max(counts["iterations"], 1)
    m_r = HEADLINE_OPTS["restart_m"]
    cols = [m_r] * (it_t // m_r) + ([it_t % m_r] if it_t % m_r else [])
    mgs_steps = sum(min(j + 2, m_r + 1) for c in cols for j in range(c))
    n3 = 3 * (n + 2) * (n + 2)
    orth_ms = phases["orthogonalise"]
    mgs_bytes = (4 * mgs_steps + 2 * it_t) * n3 * 8.0
    mgs_gbs = mgs_bytes / (orth_ms / 1e3) / 1e9
    mgs_tflops = 2 * 2 * mgs_steps * n3 / (orth_ms / 1e3) / 1e12
    roof_smoother = roof
    roof = {"kernel": "k_mgs_step (modified Gram-Schmidt step of FGMRES(80) on the W^(1/2)-scaled basis)",
            "bound": "hbm", "achieved": mgs_gbs, "peak": hbm_peak, "unit": "GB/s", "frac": mgs_gbs / hbm_peak,
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if "hbm_gbs" in peaks else "fallback 6400 GB/s",
            "traffic": 75.81e6 + 1.96e6,
            "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one step at 1024^2 under ncu's "
                               "cold caches (profiles/k_mgs_step_fp64_1024.md); in the solve w and v_{k-1} are "
                               "partly served from L2"),
            "alg_bytes_per_step": 4 * n3 * 8, "steps_per_iteration": mgs_steps / it_t,
            "ms_per_step": orth_ms / mgs_steps,
            "timing": ("CUDA events around the orthogonalisation phase of each captured iteration (all MGS steps of "
                       "the column plus its k_mgs_finish and k_scale_next), one solve after the timed ones"),
            "fp64": {"achieved_TFLOPs": mgs_tflops, "peak": fp64_peak, "frac": mgs_tflops / fp64_peak,
                     "source": "2 FMA per entry and step against the FP64 FMA rate measured in this run (of measured)"},
            "fp64_smoother": roof_smoother}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": WORKLOAD,
            "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99))},
            "solver": {"iters": stats[-1].iters, "restarts": stats[-1].restarts, "levels": stats[-1].levels,
                       "rel_energy_res": stats[-1].rel_energy_res, "rel_l2_res": stats[-1].rel_l2_res,
                       "setup_ms": stats[-1].t_setup_ms},
            "clocks": clk, "e2e": e2e, "roofline": roof,
            "gpu_launches": int(sum(s.kernel_launches for s in stats))}

    if not args.no_mixed:
        hm = P.Stokes(n, n, prec=P.PREC_MIXED, max_iter=3000, **MIXED_OPTS)
        outm = [torch.zeros_like(o) for o in outs]
        for _ in range(2):
            sm = one_solve(hm, outm)
        torch.cuda.synchronize()
        ms = []
        for k in range(max(3, args.steps // 2)):
            flush.fill_(float(k))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sm = one_solve(hm, outm)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        errv = float(torch.linalg.norm(outm[0] - outs[0]) / torch.linalg.norm(outs[0]))
        errp = float(torch.linalg.norm(outm[2] - outs[2]) / torch.linalg.norm(outs[2]))
        line["mixed_precision"] = {"solves_per_s": world * 1e3 / float(np.mean(ms)), "iters": sm.iters,
                                   "rel_energy_res": sm.rel_energy_res, "rel_diff_vs_fp64_v": errv,
                                   "rel_diff_vs_fp64_p": errp, "p50_ms": float(np.percentile(ms, 50)),
                                   "p99_ms": float(np.percentile(ms, 99)), "options": MIXED_OPTS}
        hm.close()
    line["paper_preconditioner"] = paper_block_sample(one_solve, outs, flush, stream, n, world,
                                                      max(3, args.steps // 2))
    # single-GPU samples and the CPU baseline: at N = 1 only (at N > 1 they would hold every GPU of
    # the job while rank 0 alone works)
    if rank == 0 and world == 1 and not args.no_extras:
        line["layered_1024"] = layered_sample()
        line["vcycle_roofline"] = vcycle_rooflines(peaks)
        line["accelerators"] = accelerator_sample(f, n)
        line["markers"] = marker_sample()
        line["sinker_1e8_500x600"] = sinker_e1_sample()
        line["serving"] = serving_sample()
        line["adjoint"] = adjoint_sample()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_baseline("grf", n * n)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
