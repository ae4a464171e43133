"""Benchmark: time-to-1e-8 per map with the two-level preconditioner (vs M_BD).

Workload (default): 256x256 patch (65536 pixels, I/Q/U), 128 detectors x
2^20 samples at 100 Hz, back-and-forth raster, HWP angle U[0, pi), Gaussian
sky, 1/f noise with f_knee U[0.1, 2] Hz per detector, banded Toeplitz
inverse-noise weight with half-bandwidth 2048 over 64 stationary intervals,
coarse space of k = 32 Ritz vectors.  Synthetic, seeded (seed = rank).

The scan (pointing, M_BD and the k-vector coarse space) is set up once and
kept resident, as the paper's "simplified" reuse of one deflation basis for
many maps does (Sect. 7); its one-time cost is reported beside the result.
One step = one map from a timeline resident in HBM: b = P^T W d and two-level
PCG to a relative residual of 1e-8 (float32 operator, float64 refinement).
`value` is device seconds per map for the whole job (max over ranks of the
timed region divided by all maps solved).  The M_BD solve of the same map is
timed beside it.  The `e2e` figure is the same call through the C ABI with a
host timeline and a host map (copies inside the timed region).

--impl reference times the FP64 oracle on the host cores on a bounded sample
of the same workload and scales it to the same metric.
"""
from __future__ import annotations

import argparse
import json
import os
import queue
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-to-1e-8 residual per map (2-level vs M_BD), A·x samples/s, p99 latency"
UNIT = "s/map"
# ncu: k_filter_half<float, 0, 512, 9216> moved 141.3 MB read + 3.0 MB written for 1.68e7 samples
NCU_DRAM_BYTES_PER_SAMPLE_HALF_F32 = (141.282304e6 + 2.973184e6) / 16777216


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="c2")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--k", type=int, default=32)
    ap.add_argument("--m-max", type=int, default=120)
    ap.add_argument("--eps-arn", type=float, default=1e-6)
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--max-iter", type=int, default=1000)
    ap.add_argument("--no-bd", action="store_true", help="skip the M_BD comparison solve")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-fp64", action="store_true", help="skip the MM_FP64 solve of the same map")
    ap.add_argument("--no-wide", action="store_true", help="skip the solve with every resolved Ritz pair")
    ap.add_argument("--inner-tol", type=float, default=2e-6)
    ap.add_argument("--coarse", default="lanczos", choices=["lanczos", "arnoldi"],
                    help="coarse space from the Lanczos vectors of a first M_BD run, or from a separate Arnoldi run")
    ap.add_argument("--poly-order", type=int, default=1, help="templates mode: subscan polynomial order")
    ap.add_argument("--fp64-products", type=int, default=2, choices=[1, 2],
                    help="templates mode, fp64: operator products in native float64 (1) or double-float (2, default)")
    ap.add_argument("--stokes", type=int, default=1, choices=[0, 1, 2],
                    help="templates mode: 1 Q/U maps from d^-, 2 I maps from d^+, 0 I/Q/U")
    ap.add_argument("--mode", default="solve", choices=["solve", "mc", "serve", "apply", "scale", "templates",
                                                       "subsets", "coarse"],
                    help="solve: c2 maps on a resident scan; mc: batched Monte Carlo (c3); serve: request stream; "
                         "apply: A x alone (profiling); coarse: M_2l on a batch, tensor-core vs float64 coarse "
                         "products")
    ap.add_argument("--n-det", type=int, default=0, help="apply mode: detectors kept from the config (0: all)")
    ap.add_argument("--half-bw", type=int, default=-1, help="apply mode: band half-width override")
    ap.add_argument("--filter", type=int, default=0, help="apply mode: 0 autotuned, 1 direct band, 2 FFT")
    ap.add_argument("--fft-len", type=int, default=0, help="apply mode: forced transform length (0: autotuned)")
    ap.add_argument("--apply-precision", default="f32", choices=["f32", "f64", "df"])
    ap.add_argument("--apply-rhs", type=int, default=1, help="apply mode: right-hand sides per product")
    ap.add_argument("--half", type=int, default=1, choices=[0, 1],
                    help="apply mode: allow whole blocks as half-length complex transforms")
    ap.add_argument("--n-rhs", type=int, default=64)
    ap.add_argument("--n-subsets", type=int, default=16, help="subsets mode: data subsets of one patch")
    ap.add_argument("--subset-cap", type=int, default=100, help="subsets mode: PCG iteration cap (as the paper's)")
    ap.add_argument("--mc-m-max", type=int, default=300, help="mc mode: Arnoldi steps of the shared basis")
    ap.add_argument("--mc-eps-arn", type=float, default=1e-12, help="mc mode: Arnoldi tolerance")
    ap.add_argument("--requests", type=int, default=500, help="serve mode: requests in the Poisson stream")
    ap.add_argument("--load", type=float, default=0.7, help="serve mode: offered load / sequential M_BD rate")
    ap.add_argument("--cap-requests", type=int, default=200, help="serve mode: requests of the capacity run")
    ap.add_argument("--seq-requests", type=int, default=24, help="serve mode: requests timed alone for the baseline")
    ap.add_argument("--coarse-nx", type=int, default=512, help="coarse mode: square patch side")
    ap.add_argument("--coarse-k", type=int, default=64, help="coarse mode: coarse-space dimension")
    return ap.parse_args()


# ---------------- helpers ----------------
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = max(smax, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def fft_passes(L):
    """Radix sequence of the library's planner for L = 2^a 3^b: 9 or 3, then 16s, then 8/4/2."""
    rs, rest = [], L
    if rest % 9 == 0:
        rs.append(9)
        rest //= 9
    elif rest % 3 == 0:
        rs.append(3)
        rest //= 3
    while rest % 16 == 0:
        rs.append(16)
        rest //= 16
    if rest in (2, 4, 8):
        rs.append(rest)
    return rs


# real flops per point of one pass (butterfly + pass twiddles), as the kernel computes them
FLOPS_PER_POINT = {16: 266 / 16, 9: 168 / 9, 8: 102 / 8, 4: 34 / 4, 3: 28 / 3, 2: 10 / 2}


def fft_flops_per_point(L):
    return sum(FLOPS_PER_POINT[r] for r in fft_passes(L))


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ---------------- reference arm: the oracle on the host ----------------
def cpu_oracle_sample(cfg_name, seed, n_products, budget_s=20.0):
    """Time the FP64 oracle's A x on a prefix of blocks, scaled to a full solve.

    Returns (seconds per map estimate, sample description, cores).
    """
    import oracle as O
    import synth
    cfg = dict(synth.CONFIGS[cfg_name])
    # a bounded sample: 2 detectors of the same geometry
    nd = min(2, cfg["n_det"])
    full_samples = cfg["n_det"] * cfg["n_t"]
    cfg["n_det"] = nd
    scan = synth.make_scan(seed=seed, **cfg)
    blocks_per_det = cfg["n_int"]
    # keep a handful of blocks so one product takes a few seconds
    nb = max(1, min(scan.n_blocks, 4))
    n_keep = int(scan.block_off[nb])
    prob = O.Problem(scan.pix[:n_keep], scan.psi[:n_keep], scan.block_off[:nb + 1], scan.band,
                     scan.block_band[:nb], scan.n_pix)
    x = np.random.default_rng(seed).standard_normal((scan.n_pix, 3))
    O.apply_A(prob, x)                                   # warm-up
    reps, t0 = 0, time.perf_counter()
    while True:
        O.apply_A(prob, x)
        reps += 1
        if time.perf_counter() - t0 > budget_s / 2 or reps >= 20:
            break
    per_product = (time.perf_counter() - t0) / reps
    per_sample = per_product / n_keep
    est = per_sample * full_samples * n_products
    desc = (f"oracle A x (numpy, FP64, direct band) on {nb} blocks = {n_keep} samples, "
            f"{reps} reps; scaled by samples to the full workload ({full_samples}) and by "
            f"{n_products} products with A per map (the GPU solve's count)")
    return est, desc, 1


# ---------------- the oracle's full c1 solves on the host cores ----------------
_ORACLE_SUB = {}


def _oracle_worker_init(sub):
    _ORACLE_SUB["prob"] = sub


def _oracle_worker_apply(x):
    import oracle as O
    return O.apply_A(_ORACLE_SUB["prob"], x)


def _oracle_c1_problem(seed=0):
    """c1 problem as the oracle sees it after pixel selection, its M_BD and b (noisy timeline)."""
    import oracle as O
    import synth
    scan = synth.scan_from_config("c1", seed=seed)
    d = synth.make_tod(scan, synth.make_sky(scan.n_pix, seed), synth.make_noise(scan, seed))
    prob = O.Problem.from_scan(scan)
    blocks, hits = O.bd_blocks(prob)
    good = O.select_pixels(blocks, hits, 1e-3)
    prob = prob.with_pix(O.flag_samples(prob.pix, good))
    blocks, _ = O.bd_blocks(prob)
    return prob, O.bd_inverse(blocks, good), O.rhs(prob, d).reshape(-1)


def _oracle_solves(prob, mbd, b, apply_A, k=16, m_max=40):
    """The oracle's M_BD PCG and its two-level PCG (Arnoldi coarse space) to 1e-8; returns seconds."""
    import oracle as O
    A = lambda v: apply_A(v.reshape(-1, 3)).reshape(-1)  # noqa: E731
    M = lambda v: O.bd_apply(mbd, v).reshape(-1)  # noqa: E731
    t0 = time.perf_counter()
    _, ibd = O.pcg(A, M, b, tol=1e-8, max_iter=1000)[:2]
    t_bd = time.perf_counter() - t0
    t0 = time.perf_counter()
    W, H, m = O.arnoldi(lambda v: M(A(v)), M(b), m_max, 1e-12)
    Z, _ = O.ritz_basis(W, H, m, k)
    AZ, _, L = O.coarse_space(A, Z)
    _, i2 = O.pcg(A, lambda v: O.m2l_apply(v, M, Z, AZ, L), b, tol=1e-8, max_iter=1000)[:2]
    t_2l = time.perf_counter() - t0
    return t_bd, ibd["iters"], t_2l, i2["iters"]


def cpu_oracle_c1(reps=3, budget_s=90.0):
    """Measured, not extrapolated: the FP64 oracle's full c1 solves (M_BD, and M_2l including its
    Arnoldi coarse space) on one host core and on every host core.  The all-core run splits the
    stationary blocks over worker processes (A is a sum over blocks, Sect. 3, Eq. linearsystem) and
    sums their oracle products; best of `reps`."""
    import multiprocessing as mp

    import oracle as O
    prob, mbd, b = _oracle_c1_problem()
    cores = os.cpu_count() or 1
    out = {"workload": "c1: 32x32 patch, 8 det x 32768 samples, lambda 512, 8 intervals; PCG to 1e-8; "
                       "M_2l with k=16 Ritz vectors of a 40-step Arnoldi run (its cost included)",
           "nproc": cores}
    t_start = time.perf_counter()
    best = None
    for _ in range(reps):
        r = _oracle_solves(prob, mbd, b, lambda x: O.apply_A(prob, x))
        best = r if best is None else tuple(min(a, c) if i % 2 == 0 else a for i, (a, c) in enumerate(zip(best, r)))
        if time.perf_counter() - t_start > budget_s / 2:
            break
    out["one_core"] = {"m_bd_s": best[0], "m_bd_iters": best[1], "m_2l_s": best[2], "m_2l_iters": best[3],
                       "cores": 1}
    # all cores: contiguous block ranges per worker
    nb = len(prob.block_off) - 1
    nw = max(1, min(cores, nb))
    cuts = np.linspace(0, nb, nw + 1).astype(int)
    subs = []
    for w in range(nw):
        b0, b1 = cuts[w], cuts[w + 1]
        o0, o1 = int(prob.block_off[b0]), int(prob.block_off[b1])
        subs.append(O.Problem(prob.pix[o0:o1], prob.psi[o0:o1], prob.block_off[b0:b1 + 1] - o0, prob.band,
                              prob.block_band[b0:b1], prob.n_pix))
    ctx = mp.get_context("spawn")
    pools = [ctx.Pool(1, initializer=_oracle_worker_init, initargs=(sub,)) for sub in subs]
    try:
        def par_apply(x):
            parts = [pl.apply_async(_oracle_worker_apply, (x,)) for pl in pools]
            return sum(p.get() for p in parts)
        par_apply(np.zeros((prob.n_pix, 3)))   # workers up
        best = None
        for _ in range(reps):
            r = _oracle_solves(prob, mbd, b, par_apply)
            best = r if best is None else tuple(min(a, c) if i % 2 == 0 else a for i, (a, c) in enumerate(zip(best, r)))
            if time.perf_counter() - t_start > budget_s:
                break
    finally:
        for pl in pools:
            pl.terminate()
    out["all_cores"] = {"m_bd_s": best[0], "m_bd_iters": best[1], "m_2l_s": best[2], "m_2l_iters": best[3],
                        "cores": nw}
    return out


def workload_config(args, world):
    """The `config` object of the default bench line (both arms)."""
    return {"workload": f"{args.config}: 256x256 patch, 128 det x 2^20 samples, lambda 2048, "
                        f"64 intervals, k={args.k}; one step = one map (b = P^T W d + two-level PCG "
                        f"to {args.tol:g}) on a resident scan whose pointing, M_BD and coarse space "
                        f"were built once (the coarse space from an M_BD run on another sky and noise "
                        f"realisation of the same scan)",
            "precision": args.precision, "l2": "inputs (1.1 GB pointing + timeline) exceed L2",
            "replicas": world}


def run_reference(args, world, rank):
    if rank != 0:
        return
    t0 = time.time()
    products = 70   # two-level PCG products per map measured on the GPU arm (67), plus b and the residuals
    est, desc, cores = cpu_oracle_sample(args.config, 0, products, budget_s=20.0 / max(1, args.steps))
    line = {"impl": "reference", "metric": METRIC, "value": est, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": est * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args, world),
            "cpu_baseline": {"value": est, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": est, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": time.time() - t0}
    print(json.dumps(line), flush=True)


# ---------------- our arm ----------------
def main():
    args = parse()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    if args.mode == "mc":
        return run_mc(args, world, rank, local)
    if args.mode == "serve":
        return run_serve(args, world, rank, local)
    if args.mode == "apply":
        return run_apply(args, world, rank, local)
    if args.mode == "scale":
        return run_scale(args, world, rank, local)
    if args.mode == "templates":
        return run_templates(args, world, rank, local)
    if args.mode == "subsets":
        return run_subsets(args, world, rank, local)
    if args.mode == "coarse":
        return run_coarse(args, world, rank, local)
    import torch
    import synth
    import __graft_entry__ as G
    G.build()
    from paper_1801_08937_gb300 import mapmaker as M

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    seed = rank
    t_gen = time.time()
    scan = synth.scan_from_config(args.config, seed=seed)
    # the coarse space is harvested from an M_BD run on one realisation of the scan's data (sky and
    # noise); the timed maps are another realisation, so the basis is not tailored to their solution
    tod_h = synth.make_tod(scan, synth.make_sky(scan.n_pix, seed), synth.make_noise(scan, seed))
    tod = synth.make_tod(scan, synth.make_sky(scan.n_pix, seed + 7919), synth.make_noise(scan, seed + 7919))
    t_gen = time.time() - t_gen
    prec = M.MM_FP32_MIXED if args.precision == "mixed" else M.MM_FP64
    tod_np = tod.astype(np.float32 if prec == M.MM_FP32_MIXED else np.float64)
    stream = torch.cuda.current_stream()
    dev = torch.device("cuda", local)
    pix_d = torch.from_numpy(scan.pix).to(dev)
    psi_d = torch.from_numpy(scan.psi).to(dev)
    tod_d = torch.from_numpy(tod_np).to(dev)
    tod_h_d = torch.from_numpy(tod_h.astype(tod_np.dtype)).to(dev)
    x_d = torch.empty((1, scan.n_pix, 3), dtype=torch.float64, device=dev)
    ctx = M.Context(local, stream.cuda_stream, prec)
    if prec == M.MM_FP32_MIXED:
        ctx.set_option("inner_tol", args.inner_tol)

    info_last = {}

    def setup_scan(pointing=(pix_d, psi_d), tod_in=tod_h_d):
        """One-time per scan: pointing, M_BD and the coarse space (from a first M_BD run by default)."""
        ctx.setup_pointing(pointing[0], pointing[1], scan.block_off, scan.block_band, scan.band, scan.n_pix,
                           n_det=scan.n_det)
        ctx.build_bd(1e-3)
        if args.coarse == "lanczos":
            ctx.set_option("harvest", args.m_max)
            ctx.solve(tod_in, M.MM_PRECOND_BD, tol=args.tol, max_iter=args.max_iter, out=x_d)
            ctx.set_option("harvest", 0)
            return ctx.build_coarse_from_solve(k=args.k)
        b = ctx.rhs(tod_in)
        return ctx.build_coarse(b[0], m_max=args.m_max, eps_arn=args.eps_arn, k=args.k)

    def step(precond=M.MM_PRECOND_2L, tod_in=tod_d, out=x_d):
        """One map: b = P^T W d and PCG to tol on the resident scan."""
        x, info = ctx.solve(tod_in, precond, tol=args.tol, max_iter=args.max_iter, out=out)
        info_last["info"] = info[0]
        return x

    def timed(fn, reps):
        torch.cuda.synchronize()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(reps):
            fn()
        a1.record(stream)
        torch.cuda.synchronize()
        return a0.elapsed_time(a1) / reps

    setup_ms = timed(setup_scan, 1)
    k_used = ctx.get_coarse()[1].shape[0]
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # ---- timed region: K two-level solves on the resident scan ----
    ctx.set_option("time_filter", 1)
    ctx.get_option("filter_ms")
    launches0 = ctx.get_option("kernel_launches")
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    n_filter = ctx.get_option("filter_launches")
    filter_ms = ctx.get_option("filter_ms")
    launches = int(ctx.get_option("kernel_launches") - launches0)
    ctx.set_option("time_filter", 0)
    info2l = dict(info_last["info"])
    from paper_1801_08937_gb300 import sharding as SH
    ms_max = SH.max_over_ranks(ms, dist)
    maps = args.steps * world
    value = ms_max / 1e3 / maps

    # ---- the dominant kernel: float32 fused gather/filter/scatter, A x alone ----
    L = int(ctx.get_option("plan_fft_len"))
    whole = int(ctx.get_option("plan_whole"))
    lam = scan.half_bw
    n_work = 0
    T = L // 2 if whole == 2 else L          # complex points per transform
    if L:
        blen = scan.n_t // scan.n_int
        segs_per_block = 1 if whole else -(-blen // (L - 2 * lam))
        n_work = scan.n_blocks if whole == 2 else -(-(scan.n_blocks * segs_per_block) // 2)
    xin = torch.randn((1, scan.n_pix, 3), dtype=torch.float64, device=dev)
    yout = torch.empty_like(xin)
    for _ in range(3):
        ctx.apply_A(xin, out=yout)
    ctx.set_option("time_filter", 1)
    ctx.get_option("filter_ms")
    reps = 20
    for _ in range(reps):
        ctx.apply_A(xin, out=yout)
    ax_ms = ctx.get_option("filter_ms") / reps
    ctx.set_option("time_filter", 0)
    # forward + inverse transform, plus the spectrum step (2 flop per point; 8 per point for the
    # paired real-spectrum step of half-length transforms)
    flops_per_launch = n_work * (2 * fft_flops_per_point(T) * T + (8 if whole == 2 else 2) * T) if L else 0.0
    bytes_per_launch = 8.0 * scan.n_samples
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    achieved_gbs = bytes_per_launch / (ax_ms * 1e-3) / 1e9 if ax_ms > 0 else 0.0
    achieved_tf = flops_per_launch / (ax_ms * 1e-3) / 1e12 if ax_ms > 0 else 0.0
    # DRAM bytes (read + write) per sample of this kernel, from an ncu capture of the same kernel on
    # 16 of the 128 detectors (1.68e7 samples, inputs larger than L2); traffic scales with samples
    traffic = None
    if prec == M.MM_FP32_MIXED and whole == 2 and L == 18432:
        traffic = NCU_DRAM_BYTES_PER_SAMPLE_HALF_F32 * scan.n_samples
    # measured CUDA-core FMA rates (the arithmetic view's denominators), clocks sampled meanwhile
    fma_clk = ClockSampler(local)
    fma_clk.start()
    fp32_peak = M.fma_peak(local, False, 1.0) / 1e12
    fp64_peak = M.fma_peak(local, True, 0.5) / 1e12
    fma_clocks = fma_clk.stop()
    alu_peak = fp32_peak if prec == M.MM_FP32_MIXED else fp64_peak
    # the HBM view is the headline: 8 B/sample of pointing per product (pix + psi), the north-star
    # roofline of A x; the arithmetic view (transform flops against the measured FMA rate) beside it
    roofline = {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved_gbs / hbm_peak if hbm_peak else None, "traffic": traffic,
                "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs: copy bandwidth, burst)",
                "algorithmic_bytes": "8 B/sample (pix + psi) x %d samples per launch" % scan.n_samples,
                "traffic_note": ("dram__bytes_read.sum + dram__bytes_write.sum per sample from one ncu capture "
                                 "(16-detector cut), scaled by samples to this launch") if traffic else None,
                "kernel": "%s<%s> (gather + FFT Toeplitz + scatter)"
                          % ("k_filter_half" if whole == 2 else "k_filter_fft",
                             "float" if prec == M.MM_FP32_MIXED else "double"),
                "avg_launch_ms": ax_ms, "fft_len": L,
                "fft_radices": fft_passes(T) if L else None, "whole_blocks": bool(whole),
                "half_length_transform": whole == 2,
                "alu_view": {"achieved_tflops": achieved_tf, "peak_tflops": alu_peak,
                             "frac": achieved_tf / alu_peak if alu_peak else None,
                             "flops_per_launch": flops_per_launch,
                             "peak_source": "measured: mm_fma_peak (%s FMA chains on every SM, ~1 s)"
                                            % ("float32" if prec == M.MM_FP32_MIXED else "float64"),
                             "fp32_fma_tflops": fp32_peak, "fp64_fma_tflops": fp64_peak,
                             "clocks_during_peak": fma_clocks},
                "step_filter_ms": filter_ms / max(1, args.steps), "step_filter_launches": n_filter / max(1, args.steps)}

    # ---- M_BD per map on the same resident scan ----
    bd = None
    if not args.no_bd:
        bd_ms = timed(lambda: step(M.MM_PRECOND_BD), max(1, min(args.steps, 2)))
        ibd = dict(info_last["info"])
        bd = {"time_to_tol_s": bd_ms / 1e3, "iters": ibd["iters"], "status": ibd["status"],
              "true_rel_res": ibd["true_rel_res"], "refinements": ibd["refinements"]}

    # ---- the same map with a larger coarse space from the same Lanczos harvest: k = 64 asked, the
    # Ritz selection keeps the pairs the harvest resolves; then the configured k again ----
    wide = None
    if not args.no_wide and args.coarse == "lanczos" and args.k < 64:
        try:
            k_wide = ctx.build_coarse_from_solve(k=64)
            step()
            wide_ms = timed(step, max(1, min(args.steps, 3)))
            iw = dict(info_last["info"])
            wide = {"k": k_wide, "time_to_tol_s": wide_ms / 1e3, "iters": iw["iters"], "status": iw["status"],
                    "true_rel_res": iw["true_rel_res"], "refinements": iw["refinements"],
                    "note": "k = 64 asked of the same harvest as the headline's k; not the configured k"}
        finally:
            ctx.build_coarse_from_solve(k=args.k)

    # ---- the same map in MM_FP64 (the configured precision of this workload): every operator product
    # in double-float arithmetic (about 44 bits), float64 vectors, dots and coarse space ----
    fp64 = None
    if not args.no_fp64 and prec == M.MM_FP32_MIXED:
        c64 = M.Context(local, stream.cuda_stream, M.MM_FP64)
        c64.set_option("fp64_products", 2)
        tod64 = torch.from_numpy(tod).to(dev)
        tod64_h = torch.from_numpy(tod_h).to(dev)
        x64 = torch.empty_like(x_d)

        def setup64():
            c64.setup_pointing(pix_d, psi_d, scan.block_off, scan.block_band, scan.band, scan.n_pix,
                               n_det=scan.n_det)
            c64.build_bd(1e-3)
            c64.set_option("harvest", args.m_max)
            c64.solve(tod64_h, M.MM_PRECOND_BD, tol=args.tol, max_iter=args.max_iter, out=x64)
            c64.set_option("harvest", 0)
            c64.build_coarse_from_solve(k=args.k)

        setup64_ms = timed(setup64, 1)
        res64 = {}
        for name, pc in (("two_level", M.MM_PRECOND_2L), ("m_bd", M.MM_PRECOND_BD)):
            def one(pc=pc):
                _, inf = c64.solve(tod64, pc, tol=args.tol, max_iter=args.max_iter, out=x64)
                res64["info"] = inf[0]
            ms64 = timed(one, 2)
            i64 = res64["info"]
            res64[name] = {"time_to_tol_s": ms64 / 1e3, "iters": i64["iters"], "status": i64["status"],
                           "true_rel_res": i64["true_rel_res"]}
        fp64 = {"context": "MM_FP64, fp64_products = 2 (double-float products, float64 vectors)",
                "setup_once_s": setup64_ms / 1e3, "two_level": res64["two_level"], "m_bd": res64["m_bd"]}
        if not args.no_wide and args.k < 64:
            # every Ritz pair the harvest resolves (here the harvested run is the whole M_BD solve)
            k64w = c64.build_coarse_from_solve(k=64)

            def one_w():
                _, inf = c64.solve(tod64, M.MM_PRECOND_2L, tol=args.tol, max_iter=args.max_iter, out=x64)
                res64["info"] = inf[0]
            one_w()
            msw = timed(one_w, 2)
            iw = res64["info"]
            fp64["two_level_all_resolved_ritz"] = {"k": k64w, "time_to_tol_s": msw / 1e3, "iters": iw["iters"],
                                                   "status": iw["status"], "true_rel_res": iw["true_rel_res"]}
        c64.close()
        del tod64, tod64_h, x64

    # ---- c1 (plain M_BD, FP64): the oracle's full solves measured on the host cores, and the GPU ----
    c1 = None
    if rank == 0 and world == 1 and not args.no_cpu:
        c1 = {"oracle": cpu_oracle_c1()}
        scan1 = synth.scan_from_config("c1", seed=0)
        d1 = torch.from_numpy(synth.make_tod(scan1, synth.make_sky(scan1.n_pix, 0),
                                             synth.make_noise(scan1, 0))).to(dev)
        g1 = M.Context(local, stream.cuda_stream, M.MM_FP64)
        g1.setup_scan(scan1)
        g1.build_bd(1e-3)
        r1 = {}

        def solve1(pc):
            _, inf = g1.solve(d1, pc, tol=1e-8, max_iter=1000)
            r1["info"] = inf[0]
        bd1 = timed(lambda: solve1(M.MM_PRECOND_BD), 5)
        it_bd1 = r1["info"]["iters"]
        cs1 = timed(lambda: g1.build_coarse(None, m_max=40, eps_arn=1e-12, k=16), 1)
        tl1 = timed(lambda: solve1(M.MM_PRECOND_2L), 5)
        c1["gpu"] = {"m_bd_s": bd1 / 1e3, "m_bd_iters": it_bd1, "m_2l_s": (tl1 + cs1) / 1e3,
                     "m_2l_iters": r1["info"]["iters"], "m_2l_coarse_setup_s": cs1 / 1e3,
                     "context": "MM_FP64 (native float64 products), mean of 5"}
        g1.close()

    # ---- end to end through the C ABI with host buffers ----
    e2e = None
    if not args.no_e2e:
        pin_tod = torch.from_numpy(tod_np).pin_memory()
        out_h = torch.empty((1, scan.n_pix, 3), dtype=torch.float64).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        step(M.MM_PRECOND_2L, tod_in=pin_tod, out=out_h)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        e2e = {"value": wall, "unit": UNIT, "h2d_bytes_per_step": int(scan.n_samples * tod_np.itemsize),
               "d2h_bytes_per_step": int(scan.n_pix * 3 * 8),
               "note": "ctx.solve on host timeline and host map (pinned); scan resident"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        products = info2l["iters"] + 2 + info2l["refinements"]
        est, desc, cores = cpu_oracle_sample(args.config, 0, products)
        cpu = {"value": est, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc,
               "method": "extrapolated from a timed sample (the full c2 oracle solve would take hours); "
                         "measured full solves at c1 are in the c1 object"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if prec == M.MM_FP32_MIXED else "f64",
            "data": "synthetic",
            "config": workload_config(args, world),
            "two_level": {"iters": info2l["iters"], "true_rel_res": info2l["true_rel_res"],
                          "refinements": info2l["refinements"], "k": k_used, "status": info2l["status"],
                          "setup_once_s": setup_ms / 1e3, "coarse_from": args.coarse, "m_max": args.m_max,
                          "eps_arn": args.eps_arn if args.coarse == "arnoldi" else None},
            "m_bd": bd,
            "two_level_all_resolved_ritz": wide,
            "apply_A": {"samples_per_s": scan.n_samples / (ax_ms * 1e-3) if ax_ms > 0 else None,
                        "kernel_ms": ax_ms,
                        "hbm_frac": (8.0 * scan.n_samples / (ax_ms * 1e-3) / 1e9) / hbm_peak if ax_ms else None},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "fp64": fp64,
            "c1": c1,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk,
            "gen_s": t_gen,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()


# ---------------- template filters (the paper's ground-based filtering) ----------------
def run_templates(args, world, rank, local):
    """The paper's filters (Sect. 4, 5.1) on the config's scan geometry without a half-wave plate: white
    noise, polarisation maps from the differenced timeline, subscan Legendre polynomials of order
    --poly-order and the azimuth-bin ground template in F = F_B W^-1 F_G W^-1 F_B.  Per map: M_2l (k Ritz
    vectors from the Lanczos sequence of a first M_BD run) against M_BD; the filtered A x alone against
    the HBM roofline (pix, psi and azimuth bin: 12 B/sample)."""
    import torch
    import synth
    import __graft_entry__ as G
    G.build()
    from paper_1801_08937_gb300 import mapmaker as M
    # the filters leave a near-null space of slowly varying Q/U patterns (hundreds of modes at c1): the
    # coarse space needs the largest k and well converged Ritz vectors; untouched defaults become those
    if args.k == 32:
        args.k = 256
    if args.coarse == "lanczos" and args.m_max == 120:
        args.coarse, args.m_max = "arnoldi", 1000
    if args.eps_arn == 1e-6:
        args.eps_arn = 1e-12
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    t_gen = time.time()
    over = {"n_det": args.n_det} if args.n_det else {}
    scan = synth.scan_from_config(args.config, seed=rank, half_bw=0, f_knee=0.0, hwp=False, **over)
    sub_off, az, n_bins = synth.make_templates(scan)
    def realisation(s_):
        sky = synth.make_sky(scan.n_pix, s_)
        if args.stokes == 1:
            sky[:, 0] = 0.0
        elif args.stokes == 2:
            sky[:, 1:] = 0.0
        return torch.from_numpy(synth.make_tod(scan, sky, synth.make_noise(scan, s_)).astype(np.float32)).to(dev)

    # the basis comes from one realisation of the data, the timed maps are another
    tod_h = realisation(rank + 7919)
    tod = realisation(rank)
    az_d = torch.from_numpy(az).to(dev)
    t_gen = time.time() - t_gen
    out = torch.empty((1, scan.n_pix, 3), dtype=torch.float64, device=dev)
    prec = M.MM_FP32_MIXED if args.precision == "mixed" else M.MM_FP64
    if prec == M.MM_FP64:
        tod = tod.double()
        tod_h = tod_h.double()
    ctx = M.Context(local, stream.cuda_stream, prec)
    ctx.set_option("inner_tol", args.inner_tol)

    def timed(fn):
        torch.cuda.synchronize()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        r = fn()
        a1.record(stream)
        torch.cuda.synchronize()
        return a0.elapsed_time(a1) / 1e3, r

    def setup():
        ctx.setup_scan(scan)
        ctx.set_templates(args.poly_order, sub_off, az_d, n_bins, args.stokes)
        if prec == M.MM_FP64:
            ctx.set_option("fp64_products", args.fp64_products)
        dropped = ctx.build_bd(1e-3)
        if args.coarse == "arnoldi":
            return dropped, ctx.build_coarse(ctx.rhs(tod_h)[0], m_max=args.m_max, eps_arn=args.eps_arn, k=args.k)
        ctx.set_option("harvest", args.m_max)
        ctx.solve(tod_h, M.MM_PRECOND_BD, tol=args.tol, max_iter=args.max_iter, out=out)
        ctx.set_option("harvest", 0)
        return dropped, ctx.build_coarse_from_solve(k=args.k)

    res = {}
    if args.steps > 0:
        t_setup, (dropped, k) = timed(setup)
    else:   # A x alone
        ctx.setup_scan(scan)
        ctx.set_templates(args.poly_order, sub_off, az_d, n_bins, args.stokes)
        if prec == M.MM_FP64:
            ctx.set_option("fp64_products", args.fp64_products)
        t_setup, dropped, k = 0.0, ctx.build_bd(1e-3), 0
    for name, pc in ((("two_level", M.MM_PRECOND_2L), ("m_bd", M.MM_PRECOND_BD)) if args.steps > 0 else ()):
        ctx.solve(tod, pc, tol=args.tol, max_iter=args.max_iter, out=out)
        tot, info = 0.0, None
        for _ in range(args.steps):
            t, (_, info) = timed(lambda: ctx.solve(tod, pc, tol=args.tol, max_iter=args.max_iter, out=out))
            tot += t
        res[name] = {"time_per_map_s": tot / args.steps, "iters": info[0]["iters"], "status": info[0]["status"],
                     "true_rel_res": info[0]["true_rel_res"], "refinements": info[0]["refinements"]}
    x = torch.randn((1, scan.n_pix, 3), dtype=torch.float64, device=dev)
    y = torch.empty_like(x)
    for _ in range(3):
        ctx.apply_A(x, out=y)
    ctx.set_option("time_filter", 1)
    ctx.get_option("filter_ms")
    reps = 20
    for _ in range(reps):
        ctx.apply_A(x, out=y)
    ax_ms = ctx.get_option("filter_ms") / reps
    ctx.set_option("time_filter", 0)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    gbs = 12.0 * scan.n_samples / (ax_ms * 1e-3) / 1e9
    line = {"mode": "templates", "config": f"{args.config} geometry, no half-wave plate, white noise, "
                                            f"{['I/Q/U', 'd^- (Q/U)', 'd^+ (I)'][args.stokes]} maps, "
                                            f"polynomial order {args.poly_order} per subscan, {n_bins} azimuth bins",
            "precision": args.precision, "coarse_from": args.coarse, "m_max": args.m_max,
            "samples": scan.n_samples, "subscans": int(len(sub_off) - 1), "pixels_dropped": dropped, "k": k,
            "setup_once_s": t_setup, "two_level": res.get("two_level"), "m_bd": res.get("m_bd"),
            "fp64_products": ["float64", "double-float"][args.fp64_products - 1] if prec == M.MM_FP64 else None,
            "apply_A": {"kernel": "k_filter_tmpl<%s>" % (("double", "df")[args.fp64_products - 1] if prec == M.MM_FP64
                                                         else "float"), "ms": ax_ms, "samples_per_s": scan.n_samples / (ax_ms * 1e-3),
                        "hbm_gbs_12B_per_sample": gbs, "hbm_frac_of_measured": gbs / hbm},
            "gen_s": t_gen}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()


# ---------------- divide and conquer: active vs simplified coarse spaces (Sect. 7) ----------------
def run_subsets(args, world, rank, local):
    """The paper's divide-and-conquer comparison on the GPU: several data subsets of one patch (c1
    geometry, other detector offsets, raster phases and noise per subset) are each solved with M_BD,
    with M_2l whose basis is built on that subset (the "active" approach, Arnoldi to eps_Arn 1e-6 and
    1e-12), and with M_2l whose basis comes from the first subset only (the "simplified" approach,
    mm_get_coarse / mm_set_coarse, Arnoldi to 1e-12), every solve capped at a fixed number of
    iterations; reports the median final residual, iterations and time with the set-up included."""
    import torch
    import synth
    import __graft_entry__ as G
    G.build()
    from paper_1801_08937_gb300 import mapmaker as M
    torch.cuda.set_device(local)
    k = 25   # the paper's dim Z
    cfg = dict(synth.CONFIGS[args.config if args.config != "c2" else "c1"])
    subs = []
    t_gen = time.time()
    for i in range(args.n_subsets):
        scan = synth.make_scan(seed=2000 + i + 1000 * rank, **cfg)
        d = synth.make_tod(scan, synth.make_sky(scan.n_pix, 7 + rank), synth.make_noise(scan, 2000 + i))
        subs.append((scan, d))
    t_gen = time.time() - t_gen

    def tmark():
        torch.cuda.synchronize()
        return time.perf_counter()

    res = {name: {"res": [], "iters": [], "s": []} for name in ("m_bd", "active_1e-6", "simplified", "active_1e-12")}
    Z0 = None
    for i, (scan, d) in enumerate(subs):
        c = M.Context(local, None, M.MM_FP64)
        c.setup_scan(scan)
        c.build_bd(1e-3)
        t0 = tmark()
        _, inf = c.solve(d, M.MM_PRECOND_BD, tol=args.tol, max_iter=args.subset_cap)
        t1 = tmark()
        res["m_bd"]["res"].append(inf[0]["true_rel_res"])
        res["m_bd"]["iters"].append(inf[0]["iters"])
        res["m_bd"]["s"].append(t1 - t0)
        for name, eps in (("active_1e-6", 1e-6), ("active_1e-12", 1e-12)):
            t0 = tmark()
            c.build_coarse(None, m_max=args.mc_m_max, eps_arn=eps, k=k)
            _, inf = c.solve(d, M.MM_PRECOND_2L, tol=args.tol, max_iter=args.subset_cap)
            t1 = tmark()
            res[name]["res"].append(inf[0]["true_rel_res"])
            res[name]["iters"].append(inf[0]["iters"])
            res[name]["s"].append(t1 - t0)
            if i == 0 and eps == 1e-12:
                Z0 = c.get_coarse()[0]
        t0 = tmark()
        if i == 0:
            c.build_coarse(None, m_max=args.mc_m_max, eps_arn=1e-12, k=k)   # the one basis, built once
        else:
            c.set_coarse(Z0)
        _, inf = c.solve(d, M.MM_PRECOND_2L, tol=args.tol, max_iter=args.subset_cap)
        t1 = tmark()
        res["simplified"]["res"].append(inf[0]["true_rel_res"])
        res["simplified"]["iters"].append(inf[0]["iters"])
        res["simplified"]["s"].append(t1 - t0)
        c.close()
    table = {}
    for name, r in res.items():
        rr = np.array(r["res"])
        table[name] = {"median_true_rel_res": float(np.median(rr)),
                       "spread_16_84": [float(np.percentile(rr, 16)), float(np.percentile(rr, 84))],
                       "iters_mean": float(np.mean(r["iters"])), "reached_tol": int(np.sum(rr <= args.tol)),
                       "time_total_s": float(np.sum(r["s"])), "time_per_subset_s": float(np.mean(r["s"]))}
    if rank == 0:
        print(json.dumps({"mode": "subsets", "metric": "final residual and time per subset (Sect. 7, Table 2 layout)",
                          "workload": f"{args.n_subsets} subsets of one {cfg['nx']}x{cfg['ny']} patch, "
                                      f"{cfg['n_det']} det x {cfg['n_t']} samples, lambda {cfg['half_bw']}; "
                                      f"PCG to {args.tol:g}, at most {args.subset_cap} iterations; k = {k}; "
                                      f"Arnoldi up to {args.mc_m_max} steps; MM_FP64",
                          "results": table, "gen_s": t_gen}), flush=True)


# ---------------- mixed precision at scale (c4) ----------------
def run_scale(args, world, rank, local):
    """c4: 512x512 patch, 1024 det x 2^20 samples.  Mixed-precision two-level map
    (coarse space k=64 from a first M_BD run) against the float64 GPU path,
    and sampled rows of A x against the oracle on a 1/64 subset (16 detectors)."""
    import torch
    import oracle as O
    import synth
    import __graft_entry__ as G
    G.build()
    from paper_1801_08937_gb300 import mapmaker as M
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    t_gen = time.time()
    scan = synth.scan_from_config("c4", seed=rank)
    tod = synth.make_tod(scan, synth.make_sky(scan.n_pix, rank), synth.make_noise(scan, rank))
    # the coarse space is harvested from another realisation of the data than the timed map
    tod_h = synth.make_tod(scan, synth.make_sky(scan.n_pix, rank + 7919), synth.make_noise(scan, rank + 7919))
    t_gen = time.time() - t_gen
    pix_d = torch.from_numpy(scan.pix).to(dev)
    psi_d = torch.from_numpy(scan.psi).to(dev)

    def timed(fn):
        torch.cuda.synchronize()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        out = fn()
        a1.record(stream)
        torch.cuda.synchronize()
        return a0.elapsed_time(a1) / 1e3, out

    res = {}
    maps = {}
    for name, prec in (("mixed", M.MM_FP32_MIXED), ("fp64", M.MM_FP64)):
        ctx = M.Context(local, stream.cuda_stream, prec)
        tod_d = torch.from_numpy(tod.astype(np.float32 if prec == M.MM_FP32_MIXED else np.float64)).to(dev)
        out = torch.empty((1, scan.n_pix, 3), dtype=torch.float64, device=dev)
        ctx.setup_pointing(pix_d, psi_d, scan.block_off, scan.block_band, scan.band, scan.n_pix, n_det=scan.n_det)
        ctx.build_bd(1e-3)
        # first use of each plan shape runs the autotuner: do it before timing
        ctx.rhs(tod_d)
        ctx.apply_A(out, out=torch.empty_like(out))
        if name == "mixed":
            ctx.set_option("inner_tol", args.inner_tol)
            t_bd, (_, ibd) = timed(lambda: ctx.solve(tod_d, M.MM_PRECOND_BD, tol=args.tol, max_iter=args.max_iter,
                                                     out=out))
            # coarse space, once per scan: k = 64 Ritz vectors need a Lanczos sequence longer than 64, so
            # the harvested M_BD run is carried to a tighter inner tolerance than the timed one
            # (all Ritz pairs of a 64-step sequence: longer float32 Lanczos sequences lose orthogonality
            # and their k = 64 smallest Ritz vectors deflate less)
            m_h = 64
            ctx.set_option("inner_tol", 1e-13)
            ctx.set_option("harvest", m_h)
            tod_hd = torch.from_numpy(tod_h.astype(np.float32)).to(dev)
            t_h, _ = timed(lambda: ctx.solve(tod_hd, M.MM_PRECOND_BD, tol=min(args.tol, 1e-12), max_iter=args.max_iter,
                                             out=out))
            del tod_hd
            ctx.set_option("harvest", 0)
            ctx.set_option("inner_tol", args.inner_tol)
            t_c, k = timed(lambda: ctx.build_coarse_from_solve(k=64))
            harvested = int(ctx.get_option("harvested"))
            t_c += t_h
            t_2l, (_, i2l) = timed(lambda: ctx.solve(tod_d, M.MM_PRECOND_2L, tol=args.tol, max_iter=args.max_iter,
                                                     out=out))
            res[name] = {"m_bd_s": t_bd, "m_bd_iters": ibd[0]["iters"], "coarse_s": t_c, "k": k,
                         "coarse_from": f"Lanczos vectors of an M_BD run ({harvested} kept)",
                         "two_level_s": t_2l, "two_level_iters": i2l[0]["iters"],
                         "true_rel_res": i2l[0]["true_rel_res"]}
        else:
            t_bd, (_, ibd) = timed(lambda: ctx.solve(tod_d, M.MM_PRECOND_BD, tol=args.tol, max_iter=args.max_iter,
                                                     out=out))
            res[name] = {"m_bd_s": t_bd, "m_bd_iters": ibd[0]["iters"], "true_rel_res": ibd[0]["true_rel_res"]}
        maps[name] = out.cpu().numpy()[0]
        ctx.close()
        del tod_d
        torch.cuda.empty_cache()
    err = float(np.linalg.norm(maps["mixed"] - maps["fp64"]) / np.linalg.norm(maps["fp64"]))
    # 1/64 subset: 16 detectors of the same scan, sampled rows of A x against the oracle
    sub = synth.scan_from_config("c4", seed=rank, n_det=16)
    prob = O.Problem.from_scan(sub)
    rng = np.random.default_rng(9)
    pixels = [int(p) for p in rng.integers(0, sub.n_pix, 6)]
    x = rng.standard_normal((sub.n_pix, 3))
    ref = O.apply_A_rows(prob, x, pixels)
    ctx = M.Context(local, stream.cuda_stream, M.MM_FP32_MIXED)
    ctx.setup_scan(sub)
    y = ctx.apply_A(torch.from_numpy(x[None]).to(dev)).cpu().numpy()[0]
    ctx.close()
    sub_err = float(np.linalg.norm(y[pixels] - ref) / np.linalg.norm(ref))
    line = {"mode": "scale", "config": "c4: 512x512 patch, 1024 det x 2^20 samples, lambda 2048, 64 intervals, k=64",
            "samples": scan.n_samples, "mixed": res["mixed"], "fp64": res["fp64"],
            "map_rel_err_mixed_vs_fp64": err, "subset_Ax_rows_rel_err_vs_oracle": sub_err, "gen_s": t_gen}
    if rank == 0:
        print(json.dumps(line), flush=True)


# ---------------- A x alone (profiling) ----------------
def run_apply(args, world, rank, local):
    """mm_apply_A on the config's scan (optionally fewer detectors), timed with the filter's CUDA events."""
    import torch
    import synth
    import __graft_entry__ as G
    G.build()
    from paper_1801_08937_gb300 import mapmaker as M
    torch.cuda.set_device(local)
    over = {"n_det": args.n_det} if args.n_det else {}
    if args.half_bw >= 0:
        over["half_bw"] = args.half_bw
    scan = synth.scan_from_config(args.config, seed=rank, **over)
    prec = M.MM_FP64 if args.apply_precision == "f64" else M.MM_FP32_MIXED
    ctx = M.Context(local, torch.cuda.current_stream().cuda_stream, prec)
    if args.filter:
        ctx.set_option("filter", args.filter)
    if args.fft_len:
        ctx.set_option("filter", 2)
        ctx.set_option("fft_len", args.fft_len)
    if args.apply_precision == "df":
        ctx.set_option("apply_precision", 2)
    ctx.set_option("half_transform", args.half)
    ctx.setup_scan(scan)
    nrhs = max(1, args.apply_rhs)
    x = torch.randn((nrhs, scan.n_pix, 3), dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    for _ in range(max(1, args.warmup)):
        ctx.apply_A(x, out=y)
    ctx.set_option("time_filter", 1)
    ctx.get_option("filter_ms")
    for _ in range(args.steps):
        ctx.apply_A(x, out=y)
    ms = ctx.get_option("filter_ms") / args.steps
    if rank == 0:
        peaks = {}
        try:
            peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        except Exception:
            pass
        hbm = float(peaks.get("hbm_gbs", 6800.0))
        # algorithmic bytes: each sample's pix and psi once per launch, whatever the right-hand sides
        gbs = 8.0 * scan.n_samples / (ms * 1e-3) / 1e9
        print(json.dumps({"mode": "apply", "config": args.config, "n_det": scan.n_det, "half_bw": scan.half_bw,
                          "samples": scan.n_samples, "n_rhs": nrhs, "precision": args.apply_precision,
                          "fft_len": int(ctx.get_option("plan_fft_len")),
                          "plan_whole": int(ctx.get_option("plan_whole")), "filter_ms": ms,
                          "samples_per_s": nrhs * scan.n_samples / (ms * 1e-3), "hbm_gbs_8B_per_sample": gbs,
                          "hbm_frac_of_measured": gbs / hbm}), flush=True)
    ctx.close()


# ---------------- M_2l on a batch: tensor-core vs float64 coarse products ----------------
def run_coarse(args, world, rank, local):
    """M_2l R for n_rhs right-hand sides on a large square patch with a k-vector coarse space
    (Sect. 3.2, Eq. m2l): the coarse products Z^T R, Z U, AZ U on the tensor cores (tc_coarse 2)
    and in float64 on the CUDA cores (tc_coarse 0), each timed with CUDA events on the
    context's stream over --steps calls after --warmup calls.  Inputs (Z, AZ, R: 3 x 400 MB at the
    default 512 x 512, k = 64, 64 right-hand sides) are larger than L2."""
    import numpy as np
    import torch
    import synth
    import __graft_entry__ as G
    G.build()
    from paper_1801_08937_gb300 import mapmaker as M
    torch.cuda.set_device(local)
    nx, k, nrhs = args.coarse_nx, args.coarse_k, args.n_rhs
    scan = synth.make_scan(nx=nx, ny=nx, n_det=16, n_t=1 << 18, n_int=4, half_bw=16, f_knee=1.0, seed=72 + rank)
    stream = torch.cuda.current_stream()
    ctx = M.Context(local, stream.cuda_stream, M.MM_FP64)
    ctx.setup_scan(scan)
    ctx.build_bd()
    rng = np.random.default_rng(72 + rank)
    ctx.set_coarse(rng.standard_normal((k, scan.n_pix, 3)))
    x = torch.from_numpy(rng.standard_normal((nrhs, scan.n_pix, 3))).cuda()
    y = torch.empty_like(x)
    res = {}
    clk = ClockSampler(local)
    clk.start()
    for name, tc in (("tensor_core", 2), ("float64", 0)):
        ctx.set_option("tc_coarse", tc)
        for _ in range(max(3, args.warmup)):
            ctx.apply_precond(M.MM_PRECOND_2L, x, out=y)
        l0 = ctx.get_option("kernel_launches")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            ctx.apply_precond(M.MM_PRECOND_2L, x, out=y)
        e1.record(stream)
        torch.cuda.synchronize()
        res[name] = {"ms_per_call": e0.elapsed_time(e1) / args.steps,
                     "launches_per_call": (ctx.get_option("kernel_launches") - l0) / args.steps}
    clocks = clk.stop()
    ctx.close()
    if rank != 0:
        return
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    n4 = 4 * scan.n_pix
    # algorithmic bytes: R, Z, AZ read and M_2l R written once (stored 4 doubles per pixel), M_BD's
    # six doubles per pixel; the tensor-core path reads R and Z a second time
    alg = (2 * nrhs + 2 * k) * n4 * 8 + 48 * scan.n_pix
    moved = (3 * nrhs + 3 * k) * n4 * 8 + 48 * scan.n_pix
    t = res["tensor_core"]["ms_per_call"] * 1e-3
    flops = 3 * 2 * 2 * k * nrhs * n4   # Z^T R, Z U, AZ U; three TF32 products each
    print(json.dumps({"mode": "coarse", "n_pix": scan.n_pix, "k": k, "n_rhs": nrhs, **res,
                      "speedup_vs_float64": res["float64"]["ms_per_call"] / res["tensor_core"]["ms_per_call"],
                      "algorithmic_bytes": alg, "bytes_moved_by_design": moved,
                      "hbm_gbs_algorithmic": alg / t / 1e9, "hbm_frac_of_measured": alg / t / 1e9 / hbm,
                      "tf32_tflops": flops / t / 1e12, "inputs": "larger than L2", "clocks": clocks}), flush=True)


# ---------------- batched Monte Carlo (c3) ----------------
def run_mc(args, world, rank, local):
    """64 right-hand sides of uneven length on the c1 geometry, one launch per
    PCG iteration for all of them, iterations replayed from a CUDA graph; the
    coarse space comes from the master scan once (simplified approach)."""
    import torch
    import synth
    import __graft_entry__ as G
    G.build()
    from paper_1801_08937_gb300 import mapmaker as M
    torch.cuda.set_device(local)
    seed = rank
    scan = synth.scan_from_config("c3", seed=seed)
    lens = synth.mc_lengths(args.n_rhs, 1 << 19, 1 << 20, seed)
    t_gen = time.time()
    tods = np.empty((args.n_rhs, scan.n_samples), dtype=np.float32)
    for i in range(args.n_rhs):
        s_i = 1000 + i + 100000 * seed
        tods[i] = synth.make_tod(scan, synth.make_sky(scan.n_pix, s_i), synth.make_noise(scan, s_i))
    # the shared basis comes from a realisation that is not one of the timed maps
    s_b = 1000 + args.n_rhs + 100000 * seed
    tod_basis = synth.make_tod(scan, synth.make_sky(scan.n_pix, s_b), synth.make_noise(scan, s_b)).astype(np.float32)
    t_gen = time.time() - t_gen
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)      # graphs are captured on a created stream
    torch.cuda.set_stream(stream)
    tod_d = torch.from_numpy(tods).to(dev)
    ctx = M.Context(local, stream.cuda_stream, M.MM_FP32_MIXED)
    ctx.set_option("graphs", 1)
    ctx.set_option("check_every", 8)

    def timed(fn, reps=1):
        torch.cuda.synchronize()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        out = None
        for _ in range(reps):
            out = fn()
        a1.record(stream)
        torch.cuda.synchronize()
        return a0.elapsed_time(a1) / reps, out

    out = torch.empty((args.n_rhs, scan.n_pix, 3), dtype=torch.float64, device=dev)

    def setup():
        # the paper's simplified approach (Sect. 7): Ritz vectors of one subset's M_BD A from an Arnoldi
        # run converged to eps_Arn = 1e-12, reused for every map
        ctx.setup_scan(scan)
        ctx.build_bd(1e-3)
        b = ctx.rhs(torch.from_numpy(tod_basis[None]).to(dev))
        return ctx.build_coarse(b[0], m_max=args.mc_m_max, eps_arn=args.mc_eps_arn, k=args.k)

    setup_ms, k_used = timed(setup)

    def batched(precond=M.MM_PRECOND_2L, lengths=lens):
        return ctx.solve(tod_d, precond, tol=args.tol, max_iter=args.max_iter, rhs_len=lengths, out=out)[1]

    for _ in range(max(1, args.warmup)):
        batched()
    launches0 = ctx.get_option("kernel_launches")
    ms, infos = timed(batched, args.steps)
    launches = int(ctx.get_option("kernel_launches") - launches0) // max(1, args.steps)
    its = [i["iters"] for i in infos]
    ok = sum(1 for i in infos if i["status"] == "MM_OK")
    n_2l = sum(1 for i in infos if i["precond_used"] == "M_2l")
    ms_bd, infos_bd = timed(lambda: batched(M.MM_PRECOND_BD), max(1, args.steps))
    # the paper's Monte Carlo case: every map on the same (full-length) operator A, other noise and sky
    batched(M.MM_PRECOND_2L, None)
    ms_sh, inf_sh = timed(lambda: batched(M.MM_PRECOND_2L, None), max(1, args.steps))
    ms_shbd, inf_shbd = timed(lambda: batched(M.MM_PRECOND_BD, None), max(1, args.steps))
    # the same with the coarse products on the tensor cores whatever the map size (the default
    # keeps maps this small on the CUDA cores in float64)
    ctx.set_option("tc_coarse", 2)
    batched(M.MM_PRECOND_2L, None)
    ms_shtc, inf_shtc = timed(lambda: batched(M.MM_PRECOND_2L, None), max(1, args.steps))
    ctx.set_option("tc_coarse", 1)
    # single right-hand side solves of the same maps, one at a time
    n_single = min(4, args.n_rhs)
    one = torch.empty((1, scan.n_pix, 3), dtype=torch.float64, device=dev)
    single = {}
    for name, pc in (("m_bd", M.MM_PRECOND_BD), ("two_level", M.MM_PRECOND_2L)):
        tot, iters = 0.0, []
        for i in range(n_single):
            t, inf = timed(lambda: ctx.solve(tod_d[i:i + 1], pc, tol=args.tol, max_iter=args.max_iter,
                                             rhs_len=lens[i:i + 1], out=one)[1])
            tot += t
            iters.append(inf[0]["iters"])
        single[name] = {"time_per_map_s": tot / n_single / 1e3, "iters_mean": float(np.mean(iters))}
    value = ms / 1e3 / args.n_rhs
    line = {"metric": METRIC + " [batched Monte Carlo]", "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": f"c3: {args.n_rhs} RHS on a 32x32 patch, 8 det x 2^20 master scan, per-RHS "
                                   f"lengths U[2^19, 2^20] per detector, lambda 512, 4096-sample intervals, "
                                   f"shared coarse space k={k_used}, CUDA graph of 8 iterations",
                       "samples_per_batched_Ax": int(np.sum(lens) * scan.n_det)},
            "batched": {"iters_mean": float(np.mean(its)), "iters_max": int(np.max(its)), "converged": ok,
                        "kernel_launches_per_batch": launches, "rhs_with_m2l": n_2l,
                        "rhs_falling_back_to_m_bd": args.n_rhs - n_2l,
                        "note": "a basis deflates maps of the length it was built from; shorter prefixes "
                                "run M_BD (option coarse_fallback)"},
            "batched_m_bd": {"time_per_map_s": ms_bd / 1e3 / args.n_rhs,
                             "iters_mean": float(np.mean([i["iters"] for i in infos_bd]))},
            "shared_A": {"workload": "the paper's Monte Carlo case: the same %d maps' noise and sky on the "
                                     "full-length master scan (one operator A for all)" % args.n_rhs,
                         "two_level_time_per_map_s": ms_sh / 1e3 / args.n_rhs,
                         "two_level_iters_mean": float(np.mean([i["iters"] for i in inf_sh])),
                         "m_bd_time_per_map_s": ms_shbd / 1e3 / args.n_rhs,
                         "m_bd_iters_mean": float(np.mean([i["iters"] for i in inf_shbd])),
                         "coarse_products": ("float64 CUDA cores (tc_coarse 1 keeps maps under 16384 pixels "
                                             "there)" if scan.n_pix < 16384 else "tensor cores (tcgen05, TF32 pairs)"),
                         "two_level_tensor_core_coarse_time_per_map_s": ms_shtc / 1e3 / args.n_rhs,
                         "two_level_tensor_core_coarse_iters_mean": float(np.mean([i["iters"] for i in inf_shtc])),
                         "converged": sum(1 for i in inf_sh if i["status"] == "MM_OK")},
            "single_rhs": single, "setup_once_s": setup_ms / 1e3, "gen_s": t_gen}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()


# ---------------- serving (c5) ----------------
def run_serve(args, world, rank, local):
    """Poisson stream of map requests: patches 64^2..512^2, 16..1024 detectors x 2^18..2^20 samples,
    30% of the requests on one of the eight most recently used scans (their resident M_BD and
    coarse space reused; requests on a busy scan fold into its next multi-RHS solve).  Scans and
    timelines are generated on the device when a request arrives (synth.device); the client asks the
    server for memory back before it generates, so a request never waits on a full device."""
    import torch
    import __graft_entry__ as G
    G.build()
    from synth.device import make_scan_device, make_tod_device
    from paper_1801_08937_gb300 import mapmaker as M
    from paper_1801_08937_gb300 import serving as S
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    rng = np.random.default_rng(5 + rank)
    patches, dets, lengths = [64, 128, 256, 512], [16, 32, 64, 128, 256, 512, 1024], [1 << 18, 1 << 19, 1 << 20]
    n_req = args.requests
    reqs, n_scans, order = [], 0, []
    for j in range(n_req):
        recent = list(dict.fromkeys(reversed(order)))[:8]
        if recent and rng.random() < 0.3:
            key = recent[int(rng.integers(len(recent)))]
        else:
            key = (int(rng.choice(patches)), int(rng.choice(dets)), int(rng.choice(lengths)), n_scans)
            n_scans += 1
        order.append(key)
        reqs.append((key, 9000 + j))
    lam = 512
    scans = {}

    def headroom(need):
        """Free device memory for the client's own arrays (server scans are released if needed)."""
        for _ in range(3000):
            free = torch.cuda.mem_get_info(local)[0]
            if free >= need + (4 << 30):
                return
            torch.cuda.empty_cache()
            srv_now = holder.get("srv")
            if srv_now is not None:
                srv_now.release_idle(need + (8 << 30))
            time.sleep(0.01)

    def scan_of(key, keep):
        if key not in scans:
            nx, nd, nt, i = key
            headroom(12 * nd * nt)
            scans[key] = make_scan_device(torch, dev, nx, nd, nt, nt // 16384, lam, seed=2000 + i)
        for k in [k for k in scans if k not in keep]:   # the client keeps the recent scans only
            del scans[k]
        return scans[key]

    def spec(sc):
        return S.ScanSpec(sc.pix, sc.psi, sc.block_off, sc.block_band, sc.band, sc.n_pix, sc.n_det)

    def make_request(j):
        key, seed = reqs[j]
        keep = set(list(dict.fromkeys(reversed(order[:j + 1])))[:8])
        sc = scan_of(key, keep)
        headroom(24 * sc.n_samples)
        tod = make_tod_device(torch, sc, seed)
        torch.cuda.current_stream().synchronize()
        return S.MapRequest("scan%d" % key[3], spec(sc), tod, M.MM_PRECOND_2L, tol=args.tol, max_iter=args.max_iter)

    holder = {}
    kw = dict(m_max=40, k=16, eps_arn=1e-6)
    gen_stream = torch.cuda.Stream(device=dev)
    sizes = np.array([k[1] * k[2] for k, _ in reqs], dtype=np.float64)

    def producer(seq, q):
        """Requests generated ahead of their submission on a stream of their own (the queue bounds
        how many wait), so generation overlaps the server's work instead of delaying arrivals."""
        try:
            torch.cuda.set_device(local)
            with torch.cuda.stream(gen_stream):
                for j in seq:
                    q.put(make_request(j))
        except BaseException as ex:   # reported by the consumer
            q.put(ex)

    def take(q):
        r = q.get(timeout=600)
        if isinstance(r, BaseException):
            raise r
        return r

    def run_stream(seq, depth):
        q = queue.Queue(maxsize=depth)
        th = threading.Thread(target=producer, args=(seq, q), daemon=True)
        th.start()
        return q, th

    # sequential M_BD baseline: a random sample of the stream's requests, alone and one at a time, each
    # with its scan's set-up; its time per sample scales to the stream's mix of sizes
    seq_idx = sorted(rng.choice(n_req, size=min(args.seq_requests, n_req), replace=False).tolist())
    seq_t, seq_samples = 0.0, 0
    for j in seq_idx:
        r = make_request(j)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c = M.Context(local, None, M.MM_FP32_MIXED)
        sp = r.scan
        c.setup_pointing(sp.pix, sp.psi, sp.block_off, sp.block_band, sp.band, sp.n_pix, n_det=sp.n_det)
        c.build_bd(1e-3)
        c.solve(r.tod[None], M.MM_PRECOND_BD, tol=args.tol, max_iter=args.max_iter)
        c.close()
        torch.cuda.synchronize()
        seq_t += time.perf_counter() - t0
        seq_samples += sp.n_samples
        del r, c
    scans.clear()
    torch.cuda.empty_cache()
    s_per_sample = seq_t / seq_samples
    seq_s = s_per_sample * float(sizes.mean())       # sequential M_BD seconds per map of this mix
    rate = args.load / seq_s
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n_req))
    srv = S.MapServer(device=local, precision=M.MM_FP32_MIXED, iters_per_tick=4, max_active=24, max_batch=16,
                      coarse="harvest", reserve_bytes=8 << 30, **kw).start()
    holder["srv"] = srv
    q, th = run_stream(range(n_req), 8)
    futs, late = [], 0
    t_start = time.perf_counter()
    for j in range(n_req):
        r = take(q)
        delay = t_start + arrivals[j] - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        elif delay < -0.05:
            late += 1
        r.arrival = time.perf_counter()
        futs.append(srv.submit(r))
        del r
    res = [f.result(timeout=1800) for f in futs]
    wall = time.perf_counter() - t_start
    th.join()
    st = srv.stats()
    srv.stop()
    holder.clear()
    scans.clear()
    torch.cuda.empty_cache()
    ok = sum(1 for r in res if r.info["status"] == "MM_OK")
    # capacity: a fresh server kept busy by a closed loop of 24 outstanding requests
    n_cap = min(n_req, args.cap_requests)
    srv2 = S.MapServer(device=local, precision=M.MM_FP32_MIXED, iters_per_tick=4, max_active=24, max_batch=16,
                       coarse="harvest", reserve_bytes=8 << 30, **kw).start()
    holder["srv"] = srv2
    q, th = run_stream(range(n_cap), 8)
    t1 = time.perf_counter()
    futs2, res2 = [], []
    for j in range(n_cap):
        while len(futs2) - len(res2) >= 24:
            res2.append(futs2[len(res2)].result(timeout=1800))
        r = take(q)
        r.arrival = time.perf_counter()
        futs2.append(srv2.submit(r))
        del r
    while len(res2) < len(futs2):
        res2.append(futs2[len(res2)].result(timeout=1800))
    cap_s = time.perf_counter() - t1
    th.join()
    cap = n_cap / cap_s
    st2 = srv2.stats()
    srv2.stop()
    holder.clear()
    line = {"metric": METRIC + " [serving]", "value": st["p99_s"], "unit": "s (p99 latency)", "n_gpus": world,
            "steps": n_req, "warmup": 0, "ms_per_step": wall / n_req * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic (generated on the device)",
            "config": {"workload": f"{n_req} Poisson requests at {args.load}x sequential M_BD capacity, patches "
                                   "64^2..512^2, 16..1024 det x 2^18..2^20 samples, lambda 512, 30% of requests on "
                                   "one of the 8 most recent scans",
                       "unique_scans": n_scans},
            "serving": {"p50_s": st["p50_s"], "p99_s": st["p99_s"], "maps_per_s": n_req / wall,
                        "converged": ok, "cache_hits": st["cache_hits"], "evictions": st["evictions"],
                        "max_concurrent": st["max_concurrent"], "batched_requests": st["batched_requests"],
                        "largest_batch": st["largest_batch"], "oom_requeued": st["oom_requeued"],
                        "late_arrivals_over_50ms": late, "samples_per_s": float(sizes.sum()) / wall},
            "saturated": {"maps_per_s": cap, "requests": n_cap, "outstanding": 24,
                          "samples_per_s": float(sizes[:n_cap].sum()) / cap_s,
                          "converged": sum(1 for r in res2 if r.info["status"] == "MM_OK"),
                          "batched_requests": st2["batched_requests"], "largest_batch": st2["largest_batch"],
                          "p50_s": st2["p50_s"], "p99_s": st2["p99_s"]},
            "sequential_m_bd": {"maps_per_s": 1.0 / seq_s, "s_per_map": seq_s, "samples_per_s": 1.0 / s_per_sample,
                                "n": len(seq_idx), "note": "time per sample of a random sample of the stream's "
                                "requests (set-up + M_BD solve, one at a time), scaled to the stream's mean size"},
            "mean_samples_per_request": float(sizes.mean()), "offered_rate_per_s": rate}
    if rank == 0:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
