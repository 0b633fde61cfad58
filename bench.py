"""Benchmark: filter-sweep HBM throughput of filter diagonalization on GB300.

Workload (one GPU): the narrow-band stencil matrix, a periodic 3D Anderson
model with L = 128 (2,097,152 rows, 7 nonzeros per row, hopping -1, on-site
disorder uniform in [-1, 1], seed 1), nb = 64 vectors per SpMMV block,
Chebyshev degree 500, N_s = 384 search vectors (6 blocks; the paper uses
N_s = 384 for N_t = 100, Table 6), window [-0.05, 0.05].

One step = one outer FD iteration through the C ABI in the FP32-filter form
the workload names: every 64-wide bundle is rounded to FP32, filtered with
500 fused FP32 steps and widened back; then Cholesky-QR (2 passes),
Rayleigh-Ritz (SpMMV, Gram, Jacobi, rotations) and the residual norms run in
FP64 and are read back to the host.
value = algorithmic filter bytes per step (Eq. EstimateT, kappa = 5) / step
time: the sweep's HBM throughput with the orthogonalisation and Rayleigh-Ritz
time charged to it.  The all-FP64 form of the same step is reported under
"f64_form"; its fused step is bound by GB300's FP64 rate, not by HBM.  The
inputs (6.4 GB block, 0.5 GB matrix) exceed the 129 MB L2, so no flush is
needed between steps.

`--impl reference` times the FP64 CPU oracle (scipy CSR SpMMV + NumPy) on a
bounded sample of the same workload on the host cores.
"""
import argparse
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

L = 128
SPEC = f"anderson3d:L={L},W=2,seed=1"
NB, DEGREE, NS = 64, 500, 384
WINDOW = (-0.05, 0.05)
METRIC = "filter-sweep HBM GB/s vs peak; time to k eigenpairs at residual<=1e-9"
UNIT = "GB/s"
WORKLOAD = {"workload": "anderson3d L=128 (2,097,152 rows) stencil, nb=64, degree=500, N_s=384, "
                        "one FD outer iteration (filter + CholQR2 + Rayleigh-Ritz + residuals)",
            "rows": L ** 3, "nnz_per_row": 7, "nb": NB, "degree": DEGREE, "ns": NS,
            "window": list(WINDOW), "l2_policy": "inputs larger than L2 (6.4 GB block)"}


# GB300 FP64 peak (nominal 1.25 TFLOP/s; an FMA-loop probe on this machine measured 1.20)
FP64_TFLOPS = 1.25
# DRAM bytes (read + write) of one generic FP32 step of this workload, from one ncu
# capture of `bench.py --kernel-only f32` (profiles/k_cheb_step_f32_stencil_L128_nb64.md),
# with the kernel shape it was taken on and the SHA-256 of the step kernel's sources
# at that time: when the sources differ, the figure is stale and is reported as null
TRAFFIC_F32 = {"bytes": 1.762341888e9 + 1.0270528e9, "kernel": "k_cheb_step<float,64,GENERIC>",
               "rows": 2097152, "nnz": 14680064, "nb": 64,
               "sources_sha256": "ca2c354e272c5d65b724693c96f91916002584102c602b2b76fa213a5c67b8c7"}
STEP_SOURCES = ["paper_2209_01974_gb300/csrc/fd_step.cuh", "paper_2209_01974_gb300/csrc/fd_filter.cu"]


def step_sources_sha256():
    import hashlib
    h = hashlib.sha256()
    for f in STEP_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def traffic_record(D, nnz, nb):
    """The captured DRAM bytes per launch if they belong to this kernel shape and
    to the step kernel's current sources, else None with the reason."""
    t = TRAFFIC_F32
    if (t["rows"], t["nnz"], t["nb"]) != (D, nnz, nb):
        return None, "traffic captured on another shape"
    if t["sources_sha256"] != step_sources_sha256():
        print("bench: roofline.traffic is stale (the step kernel's sources changed since the ncu "
              "capture); reporting null", file=sys.stderr)
        return None, "step kernel changed since the ncu capture"
    return t["bytes"], f"ncu dram__bytes_read.sum + dram__bytes_write.sum of {t['kernel']}, one launch"


def filter_bytes(D, nnz, nb, n, Sx):
    """Algorithmic bytes of one degree-n filter on an nb-wide block (Eq. traffic, kappa = 5)."""
    mat = nnz * (Sx + 4.0)
    vec = nb * D * Sx
    total = (mat + 2 * vec) + (mat + (4 if n > 2 else 3) * vec)
    total += max(0, n - 3) * (mat + 5 * vec) + (mat + 4 * vec if n >= 3 else 0)
    return total


def generic_step_bytes(D, nnz, nb, Sx):
    return nnz * (Sx + 4.0) + 5 * nb * D * Sx


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = "clocks.sm,clocks.max.sm,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown," \
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown," \
             "clocks_event_reasons.sw_power_cap"

    def __init__(self, index):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                     timeout=5).stdout.strip()
                if out:
                    self.samples.append([x.strip() for x in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4)
                          if len(s) > 3 + i and s[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


# --------------------------------------------------------------------------- oracle leg
def oracle_sample(n_steps=3, cores_note=True):
    """Time the FP64 oracle's filter (scipy CSR) on one 64-wide block for n_steps steps."""
    from oracle import chebyshev as ch
    from oracle import matrices as mat
    import fd_inputs
    csr = mat.build(SPEC)
    A = mat.to_scipy(csr)
    D, nnz = A.shape[0], A.nnz
    V0 = fd_inputs.random_block(D, NB, 0)
    alpha, beta = ch.scale_params(-7.01, 7.01)
    mu = ch.filter_coeffs(alpha * WINDOW[0] + beta, alpha * WINDOW[1] + beta, n_steps)
    t0 = time.perf_counter()
    ch.cheb_filter(A, V0, mu, alpha, beta)
    dt = time.perf_counter() - t0
    byts = filter_bytes(D, nnz, NB, n_steps, 8.0)
    return byts / dt / 1e9, dt, byts


# ---- the oracle on every host core: the 64 columns of the block split over a
# spawned process pool (the filter is independent per column), each worker
# running the oracle's Alg. 2 unchanged on its column slice
_W = {}


def _oracle_worker_init():
    from oracle import chebyshev as ch
    from oracle import matrices as mat
    _W["A"] = mat.to_scipy(mat.build(SPEC))
    _W["ch"] = ch


def _oracle_worker_filter(job):
    import fd_inputs
    c0, c1, n_steps = job
    A, ch = _W["A"], _W["ch"]
    V = fd_inputs.random_block(A.shape[0], NB, 0)[:, c0:c1]
    alpha, beta = ch.scale_params(-7.01, 7.01)
    mu = ch.filter_coeffs(alpha * WINDOW[0] + beta, alpha * WINDOW[1] + beta, n_steps)
    t0 = time.perf_counter()
    ch.cheb_filter(A, V, mu, alpha, beta)
    return time.perf_counter() - t0


def host_cpu():
    """(logical cores available to this process, CPU model string)."""
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Vendor ID") and ":" in line:
                model = (model + " " + line.split(":", 1)[1].strip()).strip()
    except Exception:
        pass
    return cores, model or "unknown"


class OraclePool:
    """The oracle's filter over every host core (spawned workers, so it is safe
    after CUDA has been initialised)."""

    def __init__(self, cores):
        import multiprocessing as mp
        self.cores = cores
        self.pool = mp.get_context("spawn").Pool(cores, initializer=_oracle_worker_init)

    def sample(self, n_steps=3):
        """Wall time of the degree-n_steps oracle filter of the 64-wide block, the
        columns split over the workers; returns (GB/s, seconds, bytes)."""
        k = min(self.cores, NB)
        cuts = [round(i * NB / k) for i in range(k + 1)]
        jobs = [(cuts[i], cuts[i + 1], n_steps) for i in range(k)]
        t0 = time.perf_counter()
        self.pool.map(_oracle_worker_filter, jobs)
        dt = time.perf_counter() - t0
        D = L ** 3
        byts = filter_bytes(D, 7 * D, NB, n_steps, 8.0)
        return byts / dt / 1e9, dt, byts

    def close(self):
        self.pool.close()
        self.pool.join()


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    cores, model = host_cpu()
    pool = OraclePool(cores)
    for _ in range(args.warmup):
        pool.sample(3)
    times, tot_bytes = [], 0.0
    for _ in range(args.steps):
        gbs, dt, byts = pool.sample(3)
        times.append(dt)
        tot_bytes += byts
    pool.close()
    value = tot_bytes / sum(times) / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": WORKLOAD,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "cpu_model": model,
                             "kind": "oracle",
                             "sample": "oracle Alg. 2 filter (scipy CSR SpMMV), degree 3 on one 64-wide "
                                       f"block of the L=128 stencil, columns split over {cores} spawned "
                                       "processes, per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# --------------------------------------------------------------------------- ranks
def max_over_ranks(value, world, device="cpu"):
    """Largest value over all ranks (the job's time is its slowest replica's)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def job_throughput(bytes_per_rank_step, steps, world, max_ms):
    """Whole-job GB/s of `world` independent replicas (weak scaling): all ranks'
    algorithmic bytes over the slowest rank's time."""
    return world * bytes_per_rank_step * steps / (max_ms * 1e-3) / 1e9


# --------------------------------------------------------------------------- GPU leg
def run_gpu(args):
    import torch
    import torch.distributed as dist

    import paper_2209_01974_gb300 as fd

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    stream = torch.cuda.current_stream(dev)
    ctx = fd.fd_create(local, stream.cuda_stream)
    A = fd.fd_build_matrix(ctx, SPEC)
    info = A.info
    D, nnz = info["D"], info["nnz"]
    lam_l, lam_r = fd.fd_spectral_bounds(ctx, A, 20, 0)
    alpha, beta = 2.0 / (lam_r - lam_l), -(lam_r + lam_l) / (lam_r - lam_l)
    mu = fd.fd_filter_coeffs(alpha * WINDOW[0] + beta, alpha * WINDOW[1] + beta, DEGREE)
    gen = torch.Generator(device=dev).manual_seed(1234 + rank)
    V = torch.randn((D, NS), dtype=torch.float64, device=dev, generator=gen)
    AV = torch.empty_like(V)
    W1 = torch.empty((D, NB), dtype=torch.float64, device=dev)
    W2 = torch.empty_like(W1)
    V32 = torch.empty((D, NB), dtype=torch.float32, device=dev)
    W132 = torch.empty_like(V32)
    W232 = torch.empty_like(V32)
    fd.fd_orthonormalize(ctx, V)
    sweep_bytes32 = (NS // NB) * filter_bytes(D, nnz, NB, DEGREE, 4.0)
    sweep_bytes64 = (NS // NB) * filter_bytes(D, nnz, NB, DEGREE, 8.0)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]

    def step(prec, times=None):
        if times is not None:
            ev[0].record(stream)
        for j in range(0, NS, NB):
            if prec == "f32":
                fd.fd_copy_block(ctx, V[:, j:j + NB], V32)
                fd.fd_filter(ctx, A, V32, mu, alpha, beta, W132, W232)
                fd.fd_copy_block(ctx, V32, V[:, j:j + NB])
            else:
                fd.fd_filter(ctx, A, V[:, j:j + NB], mu, alpha, beta, W1, W2)
        if times is not None:
            ev[1].record(stream)
        fd.fd_orthonormalize(ctx, V)
        th, rho = fd.fd_rayleigh_ritz(ctx, A, V, AV)
        if times is not None:
            ev[2].record(stream)
            ev[2].synchronize()
            times.append((ev[0].elapsed_time(ev[1]), ev[0].elapsed_time(ev[2])))
        return th, rho

    def timed(prec, steps, warmup):
        for _ in range(warmup):
            step(prec)
        barrier()
        l0 = ctx.kernel_launches
        times = []
        with ClockSampler(local) as clk:
            t0 = torch.cuda.Event(enable_timing=True)
            t1 = torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            for _ in range(steps):
                step(prec, times)
            t1.record(stream)
            barrier()
        total = max_over_ranks(t0.elapsed_time(t1), world, dev)
        return total, times, ctx.kernel_launches - l0, clk.summary()

    total_ms, times, launches, clocks = timed("f32", args.steps, args.warmup)
    ms_per_step = total_ms / args.steps
    value = job_throughput(sweep_bytes32, args.steps, world, total_ms)
    filt_ms = sum(t[0] for t in times)
    achieved = sweep_bytes32 * args.steps / (filt_ms * 1e-3) / 1e9

    # all-FP64 form of the same step (FP64-ALU bound on GB300), over as many steps
    k64 = args.steps
    total64, times64, _, _ = timed("f64", k64, 1)
    filt64 = sum(t[0] for t in times64)
    flops64 = (NS // NB) * DEGREE * (2.0 * nnz * NB + 6.0 * NB * D)
    f64_form = {"value": job_throughput(sweep_bytes64, k64, world, total64), "unit": UNIT,
                "ms_per_step": total64 / k64, "steps": k64,
                "filter_gbs": sweep_bytes64 * k64 / (filt64 * 1e-3) / 1e9,
                "roofline": {"bound": "alu", "achieved": flops64 * k64 / (filt64 * 1e-3) / 1e12,
                             "peak": FP64_TFLOPS, "unit": "TFLOP/s",
                             "frac": flops64 * k64 / (filt64 * 1e-3) / 1e12 / FP64_TFLOPS,
                             "peak_source": "nominal GB300 FP64 rate of the profiling recipe "
                                            "(an FMA-loop probe measured 1.20)"}}

    # e2e: the same step with the search block copied in from pinned host memory and
    # the Ritz values / residuals read back, all inside the timed region
    host = V.cpu().pin_memory()
    e2e_ms = []
    for _ in range(max(1, min(args.steps, 3))):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        V.copy_(host, non_blocking=True)
        step("f32")
        e1.record(stream)
        e1.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
    e2e_val = world * sweep_bytes32 / (statistics.mean(e2e_ms) * 1e-3) / 1e9

    # time to solution: 20 eigenpairs of the 8-site Hubbard chain (config 1), and
    # 32 eigenpairs of the L = 48, W = 16 Anderson model in every form
    A1 = fd.fd_build_matrix(ctx, "hubbard:n_sites=8,n_up=4,n_dn=4,t=1,U=4,bc=open")
    tts = {}
    for prec in ("f64", "f32"):
        th, rho, res = fd.fd_solve(ctx, A1, -0.5, 0.5, 20, 32, 100, 1e-9, precision=prec)
        tts[prec] = {"seconds": res["t_total"], "iterations": res["iterations"],
                     "n_spmmv": res["n_spmmv"], "max_resid": float(rho.max())}
    A1.free()
    tts48 = {} if args.no_tts else time_to_solution(ctx, args.tts_forms_bench.split(","))
    c3 = {} if args.no_config3 else config3_sweep(ctx)

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peak = peaks.get("hbm_gbs")
    peak_note = "of measured" if peak else "of fallback"
    peak = peak or 6800.0
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cores, model = host_cpu()
        gbs1, dt1, _ = oracle_sample(3)
        pool = OraclePool(cores)
        pool.sample(3)                      # warm-up: workers built their matrix
        gbs, dt, _ = pool.sample(3)
        pool.close()
        cpu = {"value": gbs, "unit": UNIT, "cores": cores, "cpu_model": model, "kind": "oracle",
               "sample": f"oracle Alg. 2 filter (scipy CSR SpMMV), degree 3 on one 64-wide block of the "
                         f"L=128 stencil, columns split over {cores} spawned processes: {dt:.2f} s",
               "one_core": {"value": gbs1, "unit": UNIT, "seconds": dt1}}
    traffic, traffic_note = traffic_record(D, nnz, NB)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "dtype_detail": "FP32 filter sweeps; FP64 Cholesky-QR, Rayleigh-Ritz, residuals",
                "data": "synthetic", "config": WORKLOAD,
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak, "traffic": traffic, "traffic_source": traffic_note,
                             "peak_source": peak_note,
                             "kernel": "k_cheb_step<float,64> (fused SpMMV + recurrence + "
                                       "accumulation), averaged over the filter phase",
                             "bytes_per_generic_launch": generic_step_bytes(D, nnz, NB, 4.0)},
                "f64_form": f64_form,
                "cpu_baseline": cpu,
                "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": D * NS * 8,
                        "d2h_bytes_per_step": 2 * NS * 8},
                "gpu_launches": launches,
                "clocks": clocks,
                "phases_ms_per_step": {"filter": filt_ms / args.steps,
                                       "ortho_rr": sum(t[1] - t[0] for t in times) / args.steps},
                "time_to_solution": {"workload": "hubbard 8 sites 4+4 open, 20 eigenpairs nearest "
                                                 "[-0.5,0.5], nb=32, degree>=100, tol 1e-9", **tts},
                "time_to_solution_anderson48": tts48,
                "config3_hubbard14": c3}
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


TTS_SPEC = "anderson3d:L=48,W=16,seed=3"
# form: (precision, learned constants, intervals, finishing sweeps of the FP32 form)
TTS_FORMS = {"f64": ("f64", False, "ritz", "f64"), "f64_lehmann": ("f64", False, "lehmann", "f64"),
             "f32": ("f32", False, "ritz", "f64"), "f32_lehmann": ("f32", False, "lehmann", "f64"),
             "f64_learned": ("f64", True, "ritz", "f64"), "f32_learned": ("f32", True, "ritz", "f64"),
             "f32_learned_lehmann": ("f32", True, "lehmann", "f64"),
             "ff": ("ff", False, "ritz", "f64"), "f32_ff": ("f32", False, "ritz", "ff"),
             "f32_ff_learned": ("f32", True, "ritz", "ff")}


def time_to_solution(ctx, forms, spec=TTS_SPEC, nt=32, nb=32, half_width=0.002, max_outer=40,
                     n_max=100000):
    """Time to nt eigenpairs at residual <= 1e-9 of the L = 48, W = 16 Anderson
    model (110,592 rows) nearest 0, per form: plain FP64 (Ritz or Lehmann
    intervals), FP32 sweeps with an FP64 finish, and the learned filter
    parameters; eigenvalues compared with the first form's."""
    import paper_2209_01974_gb300 as fd
    from paper_2209_01974_gb300 import predictor
    A = fd.fd_build_matrix(ctx, spec)
    params = predictor.load()
    out = {"workload": f"{spec} ({A.D} rows), {nt} eigenpairs nearest 0 (window +-{half_width}), "
                       f"nb={nb}, degree >= 100, tol 1e-9, max_outer {max_outer}, n_max {n_max}"}
    ref = None
    for name in forms:
        prec, learned, iv, finish = TTS_FORMS[name]
        th, rho, res, pred = predictor.solve_with(ctx, params if learned else None, A, -half_width, half_width,
                                                  nt, nb, 100, 1e-9, seed=0, precision=prec,
                                                  max_outer=max_outer, n_max=n_max, intervals=iv,
                                                  finish=finish)
        th = np.sort(th)
        if ref is None and res["converged"]:
            ref = th
        out[name] = {"converged": res["converged"], "seconds": res["t_total"], "iterations": res["iterations"],
                     "n_spmmv": res["n_spmmv"], "n_spmmv_f32": res["n_spmmv_f32"],
                     "n_spmmv_ff": res["n_spmmv_ff"],
                     "final_degree": res["final_degree"], "max_resid": float(rho.max()),
                     "max_abs_dtheta_vs_first_converged": (float(np.abs(th - ref).max())
                                                           if ref is not None and res["converged"] else None),
                     "params": pred}
    A.free()
    return out


def config3_sweep(ctx, degree=50, reps=3):
    """The 14-site Hubbard ring (11,778,624 rows) fused step at nb = 32, 64, 128:
    the matrix-free operator in FP32, FP64 and float-float, and the stored matrix in FP32;
    per-step time of degree-`degree` filters and the step's algorithmic GB/s."""
    import torch

    import paper_2209_01974_gb300 as fd
    out = {"workload": "hubbard ring 14 sites 7+7 periodic, degree-50 filters on one nb-wide block"}
    peak = (json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs")
            if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else None) or 6800.0
    for label, spec, cases in (("kron", KERNEL_WORKLOADS["hubbard14kron"], [("f32", 32), ("f32", 64),
                                                                          ("f32", 128), ("f64", 64),
                                                                          ("ff", 64)]),
                               ("stored", KERNEL_WORKLOADS["hubbard14"], [("f32", 64)])):
        A = fd.fd_build_matrix(ctx, spec)
        D, nnz = A.D, A.info["nnz"]
        lo, hi = fd.fd_spectral_bounds(ctx, A)
        al, be = 2 / (hi - lo), -(hi + lo) / (hi - lo)
        mu = fd.fd_filter_coeffs(al * 9.0 + be, al * 9.5 + be, degree)
        for prec, nb in cases:
            dt = torch.float32 if prec == "f32" else torch.float64
            es = 4.0 if prec == "f32" else 8.0
            V = torch.randn((D, nb), dtype=dt, device="cuda")
            if prec == "ff":  # float-float pairs split from the FP64 block
                Vff = torch.empty((D, nb, 2), dtype=torch.float32, device="cuda")
                fd.fd_copy_block(ctx, V, Vff)
                V = Vff
            W1, W2 = torch.empty_like(V), torch.empty_like(V)
            fd.fd_filter(ctx, A, V, mu, al, be, W1, W2)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                fd.fd_filter(ctx, A, V, mu, al, be, W1, W2)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps / degree
            gbs = generic_step_bytes(D, 0 if label == "kron" else nnz, nb, es) / ms / 1e6
            out[f"{label}_{prec}_nb{nb}"] = {"ms_per_step": ms, "gbs": gbs, "frac_of_measured_peak": gbs / peak}
            del V, W1, W2
            torch.cuda.empty_cache()
        A.free()
    return out


KERNEL_WORKLOADS = {
    "stencil": SPEC,
    "hubbard14": "hubbard:n_sites=14,n_up=7,n_dn=7,t=1,U=4,bc=periodic",
    "hubbard14kron": "hubbard:n_sites=14,n_up=7,n_dn=7,t=1,U=4,bc=periodic,kron=1",
    "hubbard12": "hubbard:n_sites=12,n_up=6,n_dn=6,t=1,U=4,bc=periodic",
    "hubbard12kron": "hubbard:n_sites=12,n_up=6,n_dn=6,t=1,U=4,bc=periodic,kron=1",
    "roadgraph": "roadgraph:side=2000,q=0.3,seed=0",
    "anderson48": TTS_SPEC,
}


def run_ozaki_probe(D=524288, ns=NS):
    """Profiling driver of the dense steps: Cholesky-QR of a D x ns FP64 block with
    the tensor-core (Ozaki) products and with FP64 arithmetic, timed; 1.5 GB."""
    import torch

    import paper_2209_01974_gb300 as fd
    ctx = fd.fd_create(0)
    g = torch.Generator(device="cuda").manual_seed(5)
    V0 = torch.randn((D, ns), dtype=torch.float64, device="cuda", generator=g)
    out = {}
    for mode in ("ozaki", "fp64"):
        fd.fd_set_gemm_mode(ctx, mode)
        V = V0.clone()
        fd.fd_orthonormalize(ctx, V)
        torch.cuda.synchronize()
        V = V0.clone()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fd.fd_orthonormalize(ctx, V)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        # two passes of Gram (D ns^2 symmetric) + triangular rotation (D ns^2 / 2)
        flops = 2 * (D * ns * ns + D * ns * ns)
        out[mode] = {"ms": ms, "fp64_equiv_tflops": flops / ms / 1e9}
    print(json.dumps({"kernel_only": "cholqr2", "D": D, "ns": ns, **out}))
    return 0


def run_kernel_only(prec, workload="stencil", nb=NB, degree=12, reps=5):
    """Profiling driver: one nb-wide block of a workload matrix (the L=128 stencil by
    default; the 14-site Hubbard ring, stored or matrix-free; the 4M-node road graph),
    degree-`degree` filters in FP32, FP64 or float-float; used for the ncu captures summarised
    under profiles/.  The matrix-free workloads read no matrix: their algorithmic
    bytes per step are the five vector passes alone."""
    import torch

    import paper_2209_01974_gb300 as fd
    dt = torch.float32 if prec == "f32" else torch.float64  # float-float blocks are split from FP64
    ctx = fd.fd_create(0)
    A = fd.fd_build_matrix(ctx, KERNEL_WORKLOADS[workload])
    D, nnz = A.D, A.info["nnz"]
    lo, hi = fd.fd_spectral_bounds(ctx, A)
    al, be = 2 / (hi - lo), -(hi + lo) / (hi - lo)
    mu = fd.fd_filter_coeffs(al * WINDOW[0] + be, al * WINDOW[1] + be, degree)
    V = torch.randn((D, nb), dtype=dt, device="cuda")
    if prec == "ff":  # float-float pairs (D x nb x 2 float32) split from an FP64 block
        Vff = torch.empty((D, nb, 2), dtype=torch.float32, device="cuda")
        fd.fd_copy_block(ctx, V, Vff)
        V = Vff
    W1, W2 = torch.empty_like(V), torch.empty_like(V)
    for _ in range(2):
        fd.fd_filter(ctx, A, V, mu, al, be, W1, W2)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fd.fd_filter(ctx, A, V, mu, al, be, W1, W2)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps / degree
    es = 4.0 if prec == "f32" else 8.0
    mat_nnz = 0 if "kron=1" in KERNEL_WORKLOADS[workload] else nnz
    print(json.dumps({"kernel_only": prec, "workload": workload, "rows": D, "nnz": nnz, "nb": nb,
                      "degree": degree, "ms_per_step": ms,
                      "gbs_generic_bytes": generic_step_bytes(D, mat_nnz, nb, es) / ms / 1e6}))
    return 0


def run_batched(args):
    """64 independent 3D Anderson instances (L = 16 + floor(33 u), W = 2 + 14 u from
    SplitMix64 streams 5 / 6, seeds 0..63), 16 eigenpairs nearest E = 0, nb = 16,
    degree >= 200, residual <= 1e-9: one batched solve (persistent filter launch
    per outer iteration, CUDA graph, autotuned nb / C / CTA shape) against the same
    instances solved one by one, in the precision form --precision, with each
    instance's learned filter constants when --learned."""
    import torch

    import paper_2209_01974_gb300 as fd
    from fd_inputs import anderson_instance
    from paper_2209_01974_gb300 import predictor
    n = args.instances
    specs = []
    for s in range(n):
        L, W = anderson_instance(s)
        specs.append(f"anderson3d:L={L},W={float(W)!r},seed={s}")
    ctx = fd.fd_create(0)
    t0 = time.perf_counter()
    tune = fd.fd_tune_batched(ctx, specs, 16, 20)
    t_tune = time.perf_counter() - t0
    if args.tune_only:  # the autotuner's probes alone (the profiling driver of k_batched_filter)
        print(json.dumps({"phase": "tuner", "instances": n, "rows_total": sum(anderson_instance(s)[0] ** 3
                                                                              for s in range(n)),
                          "tuner": tune, "tuner_seconds": t_tune}))
        return 0
    mats = [fd.fd_build_matrix(ctx, sp, C=tune["C"]) for sp in specs]
    nb = tune["nb"]
    ns = nb * -(-64 // nb)
    probs, preds = [], []
    params = predictor.load() if args.learned else None
    for s, m in enumerate(mats):
        p = {"c_n": 0.0, "m_l": 0.0, "m_r": 0.0}
        if params is not None:
            f = fd.fd_filter_features(ctx, m, -0.01, 0.01, 16, nb, ns, s)
            p = fd.fd_predict_filter_params(ctx, params, f)
        preds.append(p)
        probs.append((-0.01, 0.01, 16, s, p["c_n"], p["m_l"], p["m_r"]))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out, res = fd.fd_solve_batched(ctx, mats, probs, nb, 200, 1e-9, raise_noconv=False,
                                   cta_warps=tune["cta_warps"], max_outer=args.max_outer,
                                   n_max=args.n_max, precision=args.precision, finish=args.finish,
                                   verbose=int(args.verbose))
    t_batched = time.perf_counter() - t0
    rows = sum(m.D for m in mats)
    head = {"phase": "batched", "precision": args.precision, "finish": args.finish,
            "learned": bool(args.learned),
            "max_outer": args.max_outer, "n_max": args.n_max, "rows_total": rows, "tuner": tune,
            "tuner_seconds": t_tune, "batched_seconds": t_batched,
            "converged_batched": sum(r["converged"] for r in res),
            "n_spmmv_batched": int(sum(r["n_spmmv"] for r in res)),
            "n_spmmv_f32_batched": int(sum(r["n_spmmv_f32"] for r in res)),
            "n_spmmv_ff_batched": int(sum(r["n_spmmv_ff"] for r in res)),
            "used_graph": res[0]["used_graph"]}
    print(json.dumps(head), flush=True)
    if args.no_sequential:
        return 0
    t0 = time.perf_counter()
    seq, seq_th = [], []
    for m, (a, b, nt, sd, cn, ml, mr) in zip(mats, probs):
        extra = {"c_n": cn, "m_l": ml, "m_r": mr} if params is not None else {}
        th, rho, r = fd.fd_solve(ctx, m, a, b, nt, nb, 200, 1e-9, seed=sd, raise_noconv=False,
                                 max_outer=args.max_outer, n_max=args.n_max, precision=args.precision,
                                 finish=args.finish, **extra)
        seq.append(r)
        seq_th.append(th)
    t_seq = time.perf_counter() - t0
    both = [i for i in range(n) if res[i]["converged"] and seq[i]["converged"]]
    dth = max((float(np.abs(out[i][0] - seq_th[i]).max()) for i in both), default=None)
    line = {"workload": f"batched: {n} Anderson instances L 16..48, W 2..16, 16 pairs at E=0 (window "
                        "+-0.01), nb from tuner, degree >= 200, tol 1e-9",
            "precision": args.precision, "finish": args.finish, "learned": bool(args.learned),
            "max_outer": args.max_outer, "n_max": args.n_max,
            "rows_total": rows, "tuner": tune, "tuner_seconds": t_tune,
            "batched_seconds": t_batched, "sequential_seconds": t_seq,
            "speedup": t_seq / t_batched,
            "converged_batched": sum(r["converged"] for r in res),
            "converged_sequential": sum(r["converged"] for r in seq),
            "n_spmmv_batched": int(sum(r["n_spmmv"] for r in res)),
            "n_spmmv_f32_batched": int(sum(r["n_spmmv_f32"] for r in res)),
            "n_spmmv_ff_batched": int(sum(r["n_spmmv_ff"] for r in res)),
            "used_graph": res[0]["used_graph"],
            "max_abs_dtheta_batched_vs_sequential": dth,
            "max_resid_batched": float(max((o[1][np.isfinite(o[1])].max() for o in out
                                             if np.isfinite(o[1]).any()), default=0.0))}
    print(json.dumps(line))
    return 0


def pick_interior_window(mu, lam_l, lam_r, lo_frac=0.3, hi_frac=0.7, grid=4001):
    """Centre of the lowest Jackson-damped KPM density between the given fractions
    of the spectrum (a sparse region keeps the required degree moderate)."""
    n = len(mu) - 1
    N = n + 1
    k = np.arange(n + 1)
    a = np.pi / (N + 1)
    g = ((N - k + 1) * np.cos(a * k) + np.sin(a * k) / np.tan(a)) / (N + 1)
    x = np.linspace(-1 + 2 * lo_frac, -1 + 2 * hi_frac, grid)
    T = np.cos(np.outer(np.arccos(x), k))
    c = g * mu
    c[1:] *= 2.0
    dos = (T @ c) / (np.pi * np.sqrt(1 - x * x))
    xc = x[np.argmin(dos)]
    return 0.5 * (lam_r - lam_l) * xc + 0.5 * (lam_r + lam_l)


def run_learned_eval(args):
    """The trained filter-parameter predictor against the plain heuristic on the
    road-like graph Laplacian: 64 eigenpairs at the sparsest interior point of its
    KPM density, FP32 sweeps with FP64 finish, residual <= 1e-9."""
    import paper_2209_01974_gb300 as fd
    from paper_2209_01974_gb300 import predictor
    ctx = fd.fd_create(0)
    spec = f"roadgraph:side={args.side},q=0.3,seed=0"
    A = fd.fd_build_matrix(ctx, spec)
    lo, hi = fd.fd_spectral_bounds(ctx, A)
    al, be = 2 / (hi - lo), -(hi + lo) / (hi - lo)
    mu = fd.fd_kpm_moments(ctx, A, 256, 16, 0, al, be)
    tau = pick_interior_window(mu, lo, hi)
    params = predictor.load()
    rows = {}
    for name, p in (("heuristic", None), ("learned", params)):
        th, rho, res, pred = predictor.solve_with(ctx, p, A, tau - 1e-3, tau + 1e-3, 64, 64, 100, 1e-9,
                                                  seed=0, precision="f32", max_outer=args.max_outer,
                                                  n_max=args.n_max)
        rows[name] = {"converged": res["converged"], "iterations": res["iterations"],
                      "n_spmmv": res["n_spmmv"], "final_degree": res["final_degree"],
                      "seconds": res["t_total"], "max_resid": float(rho.max()), "params": pred}
    print(json.dumps({"workload": f"{spec} ({A.D} nodes), 64 eigenpairs nearest {tau:.6f}, nb=64, "
                                  "FP32 sweeps + FP64 finish, tol 1e-9", **rows}))
    return 0


def run_chi(args):
    """Communication metrics chi_1..3 (Sec. 3.1) of the workload matrices for
    N_p = 2 .. 64, computed on the GPU from the sparsity pattern (Tables 2, 7)."""
    import paper_2209_01974_gb300 as fd
    ctx = fd.fd_create(0)
    specs = {"Hubbard14 (Table 2)": "hubbard:n_sites=14,n_up=7,n_dn=7,t=1,U=4,bc=open",
             "SpinChain24 pattern (Table 7)": "hubbard:n_sites=24,n_up=12,n_dn=0,t=1,U=4,bc=open",
             "Anderson L=128 stencil": "anderson3d:L=128,W=2,seed=1",
             "road graph 4.2M": "roadgraph:side=2048,q=0.3,seed=0"}
    out = {}
    for name, spec in specs.items():
        A = fd.fd_build_matrix(ctx, spec, C=64, sigma=1)
        rows = []
        t0 = time.perf_counter()
        for n_p in (2, 4, 8, 16, 32, 64):
            c1, c2, c3, _, _ = fd.fd_comm_metrics(ctx, A, n_p)
            rows.append({"N_p": n_p, "chi_1": round(c1, 4), "chi_2": round(c2, 4), "chi_3": round(c3, 4)})
        out[name] = {"spec": spec, "D": A.D, "seconds_all_N_p": time.perf_counter() - t0, "rows": rows}
        A.free()
    print(json.dumps({"chi": out}))
    return 0


def run_tts(args):
    """Time to N_t eigenpairs at residual <= 1e-9 of a mid-size matrix for the
    forms named in --tts-forms (see time_to_solution)."""
    import paper_2209_01974_gb300 as fd
    ctx = fd.fd_create(0)
    out = time_to_solution(ctx, args.tts_forms.split(","), spec=args.tts_spec, nt=args.tts_nt,
                           nb=args.nb if args.nb != NB else 32, half_width=args.tts_half_width,
                           max_outer=args.max_outer, n_max=args.n_max)
    print(json.dumps({"tts": out}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle sample")
    ap.add_argument("--kernel-only", choices=["f32", "f64", "ff", "cholqr2"], default=None,
                    help="profiling driver: degree-12 filters on one nb-wide block")
    ap.add_argument("--workload", choices=sorted(KERNEL_WORKLOADS), default="stencil")
    ap.add_argument("--nb", type=int, default=NB)
    ap.add_argument("--degree", type=int, default=12, help="filter degree of --kernel-only")
    ap.add_argument("--batched", action="store_true",
                    help="batched-instances measurement (64 Anderson problems) instead of the bench")
    ap.add_argument("--instances", type=int, default=64)
    ap.add_argument("--precision", default="f64", choices=["f64", "f32", "ff"],
                    help="precision form of --batched")
    ap.add_argument("--finish", default="f64", choices=["f64", "ff"],
                    help="--batched: finishing sweeps of the FP32 form (FP64 or float-float)")
    ap.add_argument("--learned", action="store_true", help="--batched: each instance's learned constants")
    ap.add_argument("--verbose", action="store_true", help="--batched / --tts: per-iteration log on stderr")
    ap.add_argument("--tune-only", action="store_true",
                    help="--batched: run the autotuner's probes and stop")
    ap.add_argument("--no-sequential", action="store_true",
                    help="--batched: time the batched solve only, not the one-by-one solves")
    ap.add_argument("--max-outer", type=int, default=40)
    ap.add_argument("--n-max", type=int, default=100000)
    ap.add_argument("--learned-eval", action="store_true",
                    help="predictor vs heuristic on the road-like graph Laplacian")
    ap.add_argument("--side", type=int, default=400)
    ap.add_argument("--chi", action="store_true",
                    help="communication metrics of the workload matrices (Sec. 3.1)")
    ap.add_argument("--tts", action="store_true",
                    help="time to solution of the FP64, FP32 and learned forms on a mid-size matrix")
    ap.add_argument("--tts-spec", default="anderson3d:L=48,W=16,seed=3")
    ap.add_argument("--tts-nt", type=int, default=32)
    ap.add_argument("--tts-half-width", type=float, default=0.002)
    ap.add_argument("--tts-forms", default="f64,f32,f32_learned")
    ap.add_argument("--tts-forms-bench", default="f64,f64_lehmann,f32,f32_ff,f32_learned,f32_ff_learned",
                    help="forms of the time-to-solution block of the default bench line")
    ap.add_argument("--no-tts", action="store_true", help="skip the L=48 time-to-solution block")
    ap.add_argument("--no-config3", action="store_true", help="skip the 14-site Hubbard ring sweep")
    args = ap.parse_args()
    if args.chi:
        return run_chi(args)
    if args.tts:
        return run_tts(args)
    if args.learned_eval:
        return run_learned_eval(args)
    if args.batched:
        return run_batched(args)
    if args.kernel_only == "cholqr2":
        return run_ozaki_probe()
    if args.kernel_only:
        return run_kernel_only(args.kernel_only, args.workload, args.nb, args.degree)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
