"""Benchmark of the Green-function-preconditioned fixed-point iteration on one GB300.

A step is one iteration of the hot path (stress, forward 3D transform, Green operator, residual,
inverse transform, strain update) over the whole cell.  The default workload is a 256^3 cell of
random non-overlapping voxelised spheres (radius U[6, 16] voxels, volume fraction 0.25, contrast 100,
seed 0), PCD sampling, AFB/R wave vectors.  The metric is voxel-iterations per second.

Prints one JSON line.  --impl reference times the FP64 CPU oracle on a bounded sample instead.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "voxel-iterations/s"

# DRAM bytes (read + write) per launch of the dominant kernel from ncu captures, recorded in
# profiles/ncu_traffic.json with the hash of the kernel sources they were taken on; a record counts only
# while the sources still hash to that value, otherwise the traffic is unknown (null).
KERNEL_SOURCES = ("gfp_fft.cuh", "gfp_fftc.cuh", "gfp_kernels.cuh", "gfp_kimpl.cuh", "gfp_tma.cuh")
TRAFFIC_PATH = os.path.join(ROOT, "profiles", "ncu_traffic.json")


def kernel_sources_sha1():
    import hashlib
    h = hashlib.sha1()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2009_03762_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def ncu_traffic(kernel, n, prec, tiles):
    """Recorded DRAM traffic per launch for this kernel, grid, precision and tile record, or None."""
    try:
        with open(TRAFFIC_PATH) as f:
            recs = json.load(f)["records"]
    except (OSError, ValueError, KeyError):
        return None
    sha = kernel_sources_sha1()
    for rec in recs:
        key = (rec.get("kernel"), rec.get("n"), rec.get("prec"), list(rec.get("tiles") or []))
        if key == (kernel, n, prec, list(tiles or [])) and rec.get("sources_sha1") == sha:
            return rec["dram_read_bytes"] + rec["dram_write_bytes"]
    return None
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")


def workload(n, seed=0):
    from paper_2009_03762_gb300 import microstructure as M
    return M.random_spheres(n, vf=0.25, rmin=6.0, rmax=16.0, contrast=100.0, seed=seed)


def hbm_peak():
    try:
        with open(PEAKS_PATH) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    def __init__(self):
        self.f = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "--query-gpu=" + q, "--format=csv,noheader,nounits",
                                       "-i", os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0],
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.f.name)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def bytes_per_voxel(n, prec):
    """Algorithmic HBM bytes per voxel of each pass.  pass_x reads the half spectrum, the state and
    lambda, mu and writes the state and the half spectrum; pass_y reads and writes the half spectrum;
    pass_z_gamma does the same and, in the mixed inner iteration, also reads the FP64 source T kt
    (3 complex FP32 per half-spectrum point)."""
    h = (n // 2 + 1) / n
    if prec == "FP64":
        spec = 6 * 16 * h
        return {"pass_x": 2 * spec + 2 * 48 + 16, "pass_y": 2 * spec, "pass_z_gamma": 2 * spec,
                "pass_y_inv": 2 * spec}
    spec = 6 * 8 * h
    return {"pass_x": 2 * spec + 2 * 24 + 8, "pass_y": 2 * spec, "pass_z_gamma": 2 * spec + 3 * 8 * h,
            "pass_y_inv": 2 * spec}


def flops_per_voxel(n):
    """FP64 flops per voxel of each pass, by the conventional count of 5 m log2 m flops for a complex
    line transform of length m (the figure FFT benchmarks report) plus the pointwise arithmetic:
    pass_x: inverse and forward R2C x-transforms of 6 real components (3 complex lines per x-line)
    and about 30 flops of pack/split, strain update and stress per voxel; pass_y: 6 components on the
    half spectrum; pass_z_gamma: forward and inverse z-transforms and about 70 flops of Green step and
    residual per half-spectrum point."""
    import math
    h = (n // 2 + 1) / n
    line = 5.0 * math.log2(n)              # per element of a complex line
    x = 2 * 3 * line + 30.0
    y = 6 * h * line
    z = 2 * 6 * h * line + 70.0 * h
    return {"pass_x": x, "pass_y": y, "pass_z_gamma": z, "pass_y_inv": y}


def dist_setup():
    """(rank, world, local_rank); initialises torch.distributed when launched by torchrun."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if not dist.is_initialized():
            backend = "nccl" if torch.cuda.is_available() else "gloo"
            if backend == "nccl":
                torch.cuda.set_device(local)
            dist.init_process_group(backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    """Largest value of x over the ranks (the job time is the slowest replica's)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_gfp(args, rank=0, world=1, local=0):
    import torch
    from paper_2009_03762_gb300 import gfp

    n = args.n
    N = n ** 3
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    lam, mu = workload(n)
    stream = torch.cuda.current_stream()
    g = gfp.Grid(n, n, n, 1.0, stream.cuda_stream)
    lam_d = torch.from_numpy(lam).to(dev)
    mu_d = torch.from_numpy(mu).to(dev)
    g.set_phases(lam_d, mu_d)
    prec = args.prec
    sch = gfp.scheme(args.op, "PCD", prec)
    tiles = g.tune(sch) if args.tune else None
    if args.tune and prec == "MIXED":
        g.tune(gfp.scheme(args.op, "PCD", "FP64"))
    E = [0.0, 0.0, 0.0, 0.0, 0.0, 0.5]
    K, W = args.steps, args.warmup
    g.solve(sch, E, 0.0, W)                   # warm-up
    torch.cuda.synchronize()
    clocks = Clocks() if rank == 0 else None
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    e0.record(stream)
    r = g.solve(sch, E, 0.0, K)               # exactly K iterations (tol = 0), inputs resident in HBM
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    ms = max_over_ranks(e0.elapsed_time(e1), world)
    clk = clocks.stop() if clocks else None
    assert r.iters == K, (r.iters, K)
    value = world * N * K / (ms * 1e-3)       # whole job: every replica solves its own cell
    # per-kernel durations on the same stream
    pass_ms = g.time_passes(sch, max(3, min(K, 20)))
    names = ["pass_x", "pass_y", "pass_z_gamma", "reduce_eta", "pass_y_inv"]
    bpv = bytes_per_voxel(n, prec)
    shares = {nm: float(t) for nm, t in zip(names, pass_ms)}
    dom = max(("pass_x", "pass_y", "pass_z_gamma", "pass_y_inv"), key=lambda k: shares[k])
    peak, peak_kind = hbm_peak()
    achieved = bpv[dom] * N / (shares[dom] * 1e-3) / 1e9
    it_ms = sum(shares.values())
    it_bytes = sum(bpv.values()) * N
    roofline_alu = None
    if prec == "FP64":
        # the FP64 transforms are bound by the FP64 units of this GPU, not by HBM: their arithmetic
        # roofline against the FMA peak measured here (gfp_measure_fma_peak)
        fpv = flops_per_voxel(n)
        p64 = gfp.measure_fma_peak("f64")
        rates = {k: fpv[k] * N / (shares[k] * 1e-3) / 1e12 for k in fpv}
        roofline_alu = {"bound": "alu", "kernel": dom, "achieved": rates[dom], "peak": p64, "unit": "TFLOP/s",
                        "frac": rates[dom] / p64, "peak_kind": "measured (gfp_measure_fma_peak, FP64 FMA)",
                        "flops_per_voxel": fpv[dom], "per_pass_tflops": rates,
                        "flop_model": "5 m log2 m per complex line of length m, plus pointwise terms"}
    # time to the 1e-8 residual, mixed vs plain FP64, on the same cell
    ttt = None
    steady = None
    if args.ttt:
        ttt = {}
        for pr in ("MIXED", "FP64"):
            s2 = gfp.scheme(args.op, "PCD", pr)
            f0 = torch.cuda.Event(enable_timing=True)
            f1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            f0.record(stream)
            rr = g.solve(s2, E, 1e-8, args.ttt_maxit)
            f1.record(stream)
            torch.cuda.synchronize()
            dt = f0.elapsed_time(f1) * 1e-3
            ttt[pr] = {"seconds": dt, "iters": rr.iters, "outer": rr.outer, "residual": rr.residual,
                       "converged": rr.converged, "sigma_mean": [float(x) for x in rr.sigma_mean]}
        sm, sf = np.array(ttt["MIXED"]["sigma_mean"]), np.array(ttt["FP64"]["sigma_mean"])
        ttt["speedup"] = ttt["FP64"]["seconds"] / ttt["MIXED"]["seconds"]
        ttt["sigma_mean_rel_diff"] = float(np.linalg.norm(sm - sf) / np.linalg.norm(sf))
        if prec == "MIXED":
            # the rate of a whole solve, free of the step count: CUDA events around the mixed solve to
            # eta < 1e-8 (setup excluded), over its FP32 inner iterations plus its FP64 outer passes
            m = ttt["MIXED"]
            steady = {"value": world * N * (m["iters"] + m["outer"]) / m["seconds"], "unit": "voxel-iterations/s",
                      "inner_only": world * N * m["iters"] / m["seconds"], "seconds": m["seconds"],
                      "inner": m["iters"], "outer": m["outer"], "tol": 1e-8}
    # end to end through the C ABI with host buffers: H2D of lambda, mu from pinned host memory, K
    # iterations, D2H of the strain into pinned host memory
    lam_pin = torch.from_numpy(np.ascontiguousarray(lam)).pin_memory()
    mu_pin = torch.from_numpy(np.ascontiguousarray(mu)).pin_memory()
    eps_host = torch.empty((6, n, n, n), dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g.set_phases(lam_pin, mu_pin)
    g.solve(sch, E, 0.0, K)
    g.strain(eps_host)
    t_e2e = max_over_ranks(time.perf_counter() - t0, world)
    e2e = world * N * K / t_e2e
    launches = r.launches                     # counted by the library for the timed solve call
    line = {
        "metric": METRIC, "value": value, "unit": "voxel-iterations/s", "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if prec == "MIXED" else "f64", "data": "synthetic",
        "config": {"workload": "random spheres %d^3, vf 0.25, r U[6,16], contrast 100, PCD %s, %s"
                   % (n, args.op, "FP32 bulk / FP64 residual+refinement" if prec == "MIXED" else "FP64"),
                   "grid": n, "scheme": args.op, "precision": prec, "tiles": tiles,
                   "parallelism": "replicas x%d (one cell per GPU, no collective on the data path)" % world,
                   "l2": "inputs larger than L2 (spectrum %.0f MB)" % (6 * (8 if prec == "MIXED" else 16)
                                                                      * (n // 2 + 1) * n * n / 1e6)},
        "roofline": roofline_alu if roofline_alu else {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": peak_kind,
                     "traffic": ncu_traffic(dom, n, prec, tiles),
                     "bytes_per_voxel": bpv[dom],
                     "iteration": {"achieved": it_bytes / (it_ms * 1e-3) / 1e9, "frac": it_bytes / (it_ms * 1e-3) / 1e9 / peak,
                                   "bytes_per_voxel": sum(bpv.values()), "ms": it_ms}},
        "roofline_hbm": {"kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "bytes_per_voxel": bpv[dom]} if roofline_alu else None,
        "pass_ms": shares,
        "time_to_1e-8": ttt,
        "steady": steady,
        "e2e": {"value": e2e, "unit": "voxel-iterations/s", "h2d_bytes_per_step": 2 * N * 8 / K,
                "d2h_bytes_per_step": 6 * N * 8 / K},
        "gpu_launches": launches,
        "clocks": clk,
        "cufft_comparison": cufft_comparison(n) if prec == "MIXED" else None,
    }
    g.close()
    return line


def cufft_comparison(n, reps=20):
    """Comparison point only (not on the hot path): cuFFT through torch.fft, R2C + C2R of the six
    FP32 components of an n^3 field, CUDA events, inputs larger than L2."""
    import torch
    x = torch.randn(6, n, n, n, device="cuda", dtype=torch.float32)
    for _ in range(3):
        y = torch.fft.irfftn(torch.fft.rfftn(x, dim=(1, 2, 3)), s=(n, n, n), dim=(1, 2, 3))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        y = torch.fft.irfftn(torch.fft.rfftn(x, dim=(1, 2, 3)), s=(n, n, n), dim=(1, 2, 3))
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    del x, y
    torch.cuda.empty_cache()
    return {"library": "cuFFT via torch.fft", "what": "R2C + C2R of 6 FP32 components, %d^3" % n,
            "ms": ms, "note": "the solver's FP32 iteration does these transforms plus stress, Green step, "
                              "residual and update"}


def passes_only(args):
    """Set phases, one FP64 residual pass (mixed), then K timed iterations: the small profiling case."""
    import torch
    from paper_2009_03762_gb300 import gfp
    n = args.n
    lam, mu = workload(n)
    g = gfp.Grid(n, n, n, 1.0, torch.cuda.current_stream().cuda_stream)
    g.set_phases(lam, mu)
    if args.tiles:
        tiles = [int(v) for v in args.tiles.split(",")]
        g.set_tiles(gfp.MIXED if args.prec == "MIXED" else gfp.FP64, tiles)
    else:
        tiles = g.tune(gfp.scheme(args.op, "PCD", args.prec)) if args.tune else None
    ms = g.time_passes(gfp.scheme(args.op, "PCD", args.prec), args.passes_only)
    bpv = bytes_per_voxel(n, args.prec)
    names = ["pass_x", "pass_y", "pass_z_gamma", "reduce_eta", "pass_y_inv"]
    out = {"n": n, "prec": args.prec, "tiles": tiles, "pass_ms": dict(zip(names, map(float, ms)))}
    out["gbs"] = {k: bpv[k] * n ** 3 / (out["pass_ms"][k] * 1e-3) / 1e9 for k in bpv}
    g.close()
    return out


def convergence_experiment(args):
    """Iterations to convergence versus phase contrast for the paper's 3D matrix-inclusion cell (Sec. 6,
    Fig. Conv3D): cube of edge n/2 by voxel index (sharp) or with the tanh interface of half-width
    eps = l/100 in the Lame constants (--conv-interface smooth, the paper's linear mixing of Sec. 6),
    lambda_M = mu_M = 0.6, chi = lambda_I/lambda_M = mu_I/mu_M, mean strain E_xy = 1; reference medium
    C_H = C_I (the paper's, chi > 1 only) or 1/2 (min + max).
    --conv-rule residual: eta < --conv-tol (ACD and AFB/R mixed precision, F FP64);
    --conv-rule increment: the paper's rule sum |du^(it) - du^(it-1)| < --conv-tol for ACD and AFB/R
    (FP64; the increment rule needs a single real wave vector per mode, so F keeps the residual rule).
    F runs to --conv-maxit-f iterations (the paper reports it unconverged after 10^4 at high contrast), at
    the contrasts of --conv-f-chi only."""
    import torch
    from paper_2009_03762_gb300 import gfp, microstructure as M
    n = args.n
    if args.conv_interface == "smooth":
        f = M.cube_density(n, n // 2, n / 100.0, sampling="TD")
    else:
        f = M.cube_indicator(n, n // 2).astype(np.float64)
    out = []
    g = gfp.Grid(n, n, n, 1.0, torch.cuda.current_stream().cuda_stream)
    inc = args.conv_rule == "increment"
    f_chis = [float(v) for v in args.conv_f_chi.split(",")] if args.conv_f_chi else None
    for chi in [float(v) for v in args.conv_chi.split(",")]:
        lam = 0.6 * (1.0 + f * (chi - 1.0))
        mu = lam.copy()
        refs = [("mean", None)] + ([("C_I", (0.6 * chi, 0.6 * chi))] if chi > 1 else [])
        for ref_name, ref in refs:
            g.set_phases(lam, mu, ref)
            runs = [("F", "FP64", 0, args.conv_maxit_f)] if f_chis is None or chi in f_chis else []
            for op in ("ACD", "AFB_R"):
                runs.append((op, "FP64" if inc else "MIXED", 1 if inc else 0, 20000))
            for op, prec, rule, maxit in runs:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                r = g.solve(gfp.scheme(op, "TD", prec, stop_rule=rule), [0, 0, 0, 0, 0, 1.0], args.conv_tol, maxit)
                torch.cuda.synchronize()
                out.append({"chi": chi, "ref": ref_name, "scheme": op, "precision": prec,
                            "rule": "increment" if rule else "residual", "interface": args.conv_interface,
                            "iters": r.iters, "status": gfp.STATUS[r.status], "criterion": r.residual,
                            "seconds": time.perf_counter() - t0, "sigma_xy": float(r.sigma_mean[5])})
                print(json.dumps(out[-1]), flush=True)
    g.close()
    return out


def schemes128_experiment(args):
    """All schemes in FP64 on the 128^3 smooth-interface cube (edge 64, tanh of half-width 2 voxels in
    log-moduli, nu = 0.3), contrasts 1e-3, 1e-1, 10, 1e3, six Voigt unit loads to eta < 1e-10 (DGO:
    its own residual, m = n/2): inner iterations per load, status and voxel-iterations/s.  TD and PCD
    give the same iterates for these schemes (the oracle pins it), so PCD is run."""
    import torch
    from paper_2009_03762_gb300 import gfp, microstructure as M
    n = 128
    g = gfp.Grid(n, n, n, 1.0, torch.cuda.current_stream().cuda_stream)
    chis = [float(v) for v in args.schemes_chi.split(",")]
    ops = args.schemes_ops.split(",")
    for chi in chis:
        lam, mu = M.smooth_cube(n, 64, chi, width=2.0)
        g.set_phases(lam, mu)
        for op in ops:
            maxit = args.schemes_maxit_slow if op in ("F", "HC") else 20000
            sch = gfp.scheme(op, "PCD", "FP64", dgo_m=n // 2 if op == "DGO" else 0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            try:
                C, its, rc = g.effective_stiffness(sch, 1e-10, maxit)
            except gfp.GfpError as err:
                print(json.dumps({"chi": chi, "scheme": op, "error": str(err)}), flush=True)
                continue
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            rec = {"chi": chi, "scheme": op, "iters": list(its), "status": gfp.STATUS[rc], "seconds": dt,
                   "voxel-iterations/s": n ** 3 * float(sum(its)) / dt,
                   "C1111": float(C[0, 0]), "C1212": float(C[5, 5])}
            print(json.dumps(rec), flush=True)
    g.close()


def batch_experiment(args):
    """Batched homogenization: random-sphere cells (n from {64, 96, 128}, volume fraction U[0.1, 0.3],
    contrast log-uniform on [1e-2, 1e3]) x 6 Voigt loads, mixed precision to eta < 1e-8, as one batch
    graph (gfp_batch_create once; each gfp_batch_solve is one graph launch in which every slot loops on
    the device), against the same cells solved one after another (gfp_effective_stiffness).
    Aggregate voxel-iterations/s = sum over cells and loads of N x inner iterations / wall time."""
    import torch
    from paper_2009_03762_gb300 import gfp, microstructure as M
    specs = M.batch_specs(args.batch_count, seed=0)
    sch = gfp.scheme(args.op, "PCD", "MIXED")
    grids = []
    tuned = {}
    for sp in specs:
        lam, mu = M.batch_item(sp)
        g = gfp.Grid(sp["n"], sp["n"], sp["n"], 1.0, torch.cuda.current_stream().cuda_stream)
        g.set_phases(lam, mu)
        if sp["n"] not in tuned:
            tuned[sp["n"]] = g.tune(sch)
        else:
            g.set_tiles(gfp.MIXED, tuned[sp["n"]])
        grids.append(g)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    batch = gfp.Batch(grids, sch)
    t_create = time.perf_counter() - t0
    C, its, rc = batch.solve(tol=1e-8, maxit=args.batch_maxit)  # first launch of the instantiated graph
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    C, its, rc = batch.solve(tol=1e-8, maxit=args.batch_maxit)
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    batch.close()
    vox_its = float(sum(sp["n"] ** 3 * int(its[i].sum()) for i, sp in enumerate(specs)))
    t0 = time.perf_counter()
    seq_its = 0.0
    max_rel = 0.0
    for i, (sp, g) in enumerate(zip(specs, grids)):
        Cs, it_s, rcs = g.effective_stiffness(sch, 1e-8, args.batch_maxit)
        seq_its += sp["n"] ** 3 * float(np.sum(it_s))
        max_rel = max(max_rel, float(np.abs(C[i] - Cs).max() / np.abs(Cs).max()))
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    for g in grids:
        g.close()
    return {"experiment": "batch", "cells": len(specs), "loads": 6 * len(specs), "status": gfp.STATUS[rc],
            "sizes": {str(n): sum(1 for sp in specs if sp["n"] == n) for n in sorted(tuned)},
            "tiles": {str(k): v for k, v in tuned.items()},
            "batch": {"seconds": t_batch, "voxel_iterations": vox_its, "voxel-iterations/s": vox_its / t_batch,
                      "create_seconds": t_create,
                      "note": "second gfp_batch_solve of the handle (one graph launch); create_seconds: slot "
                              "allocation, capture and instantiation, once per batch shape"},
            "sequential": {"seconds": t_seq, "voxel_iterations": seq_its, "voxel-iterations/s": seq_its / t_seq},
            "speedup": t_seq / t_batch, "C_eff_max_rel_diff_batch_vs_sequential": max_rel,
            "inner_iterations": {"min": int(its.min()), "max": int(its.max()), "total": int(its.sum())}}


def batch_sharded_experiment(args, rank, world, local):
    """The batched homogenization across the ranks of torchrun (one GPU each): the cells are dealt to
    the ranks by voxel count (gfp.batch_shard), each rank runs gfp_solve_batch on its share, and the
    C_eff are all-gathered (the only exchange).  Job time = slowest rank (barrier, max over ranks)."""
    import torch
    from paper_2009_03762_gb300 import gfp, microstructure as M
    specs = M.batch_specs(args.batch_count, seed=0)
    sch = gfp.scheme(args.op, "PCD", "MIXED")
    costs = [sp["n"] ** 3 for sp in specs]
    make_cell = lambda i: M.batch_item(specs[i])
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    C, its, rc = gfp.solve_batch_sharded(make_cell, costs, sch, tol=1e-8, maxit=args.batch_maxit)
    torch.cuda.synchronize()
    dt = max_over_ranks(time.perf_counter() - t0, world)
    vox_its = float(sum(costs[i] * int(its[i].sum()) for i in range(len(specs))))
    return {"experiment": "batch_sharded", "ranks": world, "cells": len(specs), "loads": 6 * len(specs),
            "status": gfp.STATUS[rc], "seconds": dt, "voxel_iterations": vox_its,
            "voxel-iterations/s": vox_its / dt, "C_eff_finite": bool(np.isfinite(C).all()),
            "shards": [gfp.batch_shard(costs, r, world) for r in range(world)],
            "note": "cells built and solved on each rank (phase fields generated there, inside the timing)"}


_SAMPLE_CELLS = {}


def oracle_sample(n, op, iters):
    """Time the FP64 oracle as it stands on `iters` iterations of the same workload (the cell is
    generated once per size, outside the timing)."""
    from oracle import gfp_oracle as O
    if n not in _SAMPLE_CELLS:
        _SAMPLE_CELLS[n] = workload(n)
    lam, mu = _SAMPLE_CELLS[n]
    t0 = time.perf_counter()
    O.solve(lam, mu, op, [0, 0, 0, 0, 0, 0.5], disc="PCD", max_iters_exact=iters)
    dt = time.perf_counter() - t0
    return n ** 3 * iters / dt, dt


def reference_arm(args, budget_s=120.0):
    """The oracle as it stands on the host cores: W untimed and K timed single iterations of the
    workload's random-sphere cell, at the largest grid (<= --oracle-n) for which K iterations take
    about budget_s (the dense-DFT oracle costs O(n^4) per iteration)."""
    from oracle import gfp_oracle as O
    K, W = max(1, args.steps), max(0, args.warmup)
    E = [0, 0, 0, 0, 0, 0.5]

    def one(lam, mu):
        t0 = time.perf_counter()
        O.solve(lam, mu, args.op, E, disc="PCD", max_iters_exact=1)
        return time.perf_counter() - t0

    sizes = [n for n in (128, 96, 64, 48, 32, 24, 16) if n <= args.oracle_n] or [args.oracle_n]
    n = sizes[0]
    lam, mu = workload(n)
    t_probe = one(lam, mu)  # untimed
    pick = sizes[-1]
    for cand in sizes:
        if t_probe * (cand / n) ** 4 * K <= budget_s:
            pick = cand
            break
    if pick != n:
        lam, mu = workload(pick)
    # the O(n^4) model underestimates small grids: measure at the chosen size and step down if needed
    t_pick = one(lam, mu)  # untimed
    while t_pick * K > budget_s and pick != sizes[-1]:
        pick = sizes[sizes.index(pick) + 1]
        lam, mu = workload(pick)
        t_pick = one(lam, mu)
    for _ in range(W):
        one(lam, mu)
    dt = float(sum(one(lam, mu) for _ in range(K)))
    value = pick ** 3 * K / dt
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "voxel-iterations/s", "n_gpus": args.gpus,
            "steps": K, "warmup": W, "ms_per_step": 1e3 * dt / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "random spheres %d^3 sample of the %d^3 workload, %s, FP64 oracle"
                       % (pick, args.n, args.op)},
            "cpu_baseline": {"value": value, "unit": "voxel-iterations/s", "cores": cpu_cores(), "kind": "oracle",
                             "sample": "%d single iterations of a %d^3 random-sphere cell" % (K, pick)},
            "e2e": {"value": value, "unit": "voxel-iterations/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=600)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gfp", choices=["gfp", "reference"])
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--op", default="AFB_R")
    ap.add_argument("--prec", default="MIXED", choices=["MIXED", "FP64"])
    ap.add_argument("--ttt", type=int, default=1, help="also time full solves to eta = 1e-8 (mixed and FP64)")
    ap.add_argument("--ttt-maxit", type=int, default=3000)
    ap.add_argument("--tune", type=int, default=1, help="run the tile autotuner before timing")
    ap.add_argument("--tiles", default="", help="x lines,y columns,z columns (negative z: TMA z-pass)")
    ap.add_argument("--experiment", default="", help="conv3d: iterations vs contrast for the paper's 3D cell; batch: batched homogenization; "
                    "schemes128: all schemes on the 128^3 smooth cube")
    ap.add_argument("--conv-tol", type=float, default=1e-8)
    ap.add_argument("--conv-rule", default="residual", choices=["residual", "increment"])
    ap.add_argument("--conv-interface", default="sharp", choices=["sharp", "smooth"])
    ap.add_argument("--conv-maxit-f", type=int, default=3000)
    ap.add_argument("--conv-chi", default="1e-3,1e-2,1e-1,10,1e2,1e3", help="contrasts of conv3d")
    ap.add_argument("--conv-f-chi", default="", help="contrasts at which conv3d runs F (default: all)")
    ap.add_argument("--batch-count", type=int, default=32)
    ap.add_argument("--schemes-maxit-slow", type=int, default=3000, help="iteration cap of F and HC in schemes128")
    ap.add_argument("--schemes-chi", default="1e-3,1e-1,10,1e3", help="contrasts of schemes128")
    ap.add_argument("--schemes-ops", default="F,CD,ACD,HC,AHC,AFB_R,DGO", help="schemes of schemes128")
    ap.add_argument("--batch-maxit", type=int, default=20000)
    ap.add_argument("--oracle-n", type=int, default=128, help="grid of the CPU-baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--passes-only", type=int, default=0,
                    help="only time K iterations pass by pass (gfp_time_passes) and print them (profiling case)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank != 0:
            return
        line = reference_arm(args)
        print(json.dumps(line))
        return
    if args.passes_only:
        print(json.dumps(passes_only(args)))
        return
    if args.experiment == "conv3d":
        convergence_experiment(args)
        return
    if args.experiment == "batch":
        rank, world, local = dist_setup()
        if world > 1:
            out = batch_sharded_experiment(args, rank, world, local)
            if rank == 0:
                print(json.dumps(out))
            return
        print(json.dumps(batch_experiment(args)))
        return
    if args.experiment == "schemes128":
        schemes128_experiment(args)
        return
    rank, world, local = dist_setup()
    line = run_gfp(args, rank, world, local)
    if rank != 0:
        return
    if not args.no_cpu_baseline and world == 1:
        # about 10-30 s of oracle work: single iterations of the workload's cell at --oracle-n until 10 s
        v, dt = oracle_sample(args.oracle_n, args.op, 1)
        its, total = 1, dt
        while total < 10.0 and total + dt < 30.0:
            total += oracle_sample(args.oracle_n, args.op, 1)[1]
            its += 1
        line["cpu_baseline"] = {"value": args.oracle_n ** 3 * its / total, "unit": "voxel-iterations/s",
                                "cores": cpu_cores(), "kind": "oracle",
                                "sample": "%d single iterations of the same workload at %d^3 (%.1f s)"
                                          % (its, args.oracle_n, total)}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
