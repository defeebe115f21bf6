"""Throughput of per-pixel sparse recovery of a 2.5x compressed hyperspectral cube.

One step = the whole hot path over one cube: measurement Y = X A^T + E (Eq. 1) and
recovery of every pixel with each of the paper's five algorithms (FISTA, ADMM, gOMP,
BIHT, CoSaMP; Section II-A), all through the C ABI of libcs_hsi.so.

Workload: 512 x 512 pixels, N = 200 bands, M = 80 measurements (2.5x), Gaussian Phi,
DCT-II Psi, power-law spectra |x_k| = k^-1.5 with random signs, N(0, 1e-3) noise;
FISTA 300 iterations (lambda = 1e-3), ADMM 300 iterations (rho = 1, lambda = 1e-3),
gOMP kappa = 20, G = 4; BIHT kappa = 20, mu = 0.1; CoSaMP kappa = 20; eps = 1e-8.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
    python bench.py --only ALGO [--pixels P]     # one algorithm on P pixels, twice (profiling)

Prints one JSON line.  value = recovered spectra per second over the whole job
(pixels x algorithms per step / step time).  The FP64 oracle (CPU) is timed on a
bounded pixel sample on the host cores and its outputs on that sample give the
accuracy of the GPU results (relative L2).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

M, N, SIDE = 80, 200, 512
P = SIDE * SIDE
LAM, ITERS, RHO, KAPPA, G, MU, EPS = 1e-3, 300, 1.0, 20, 4, 0.1, 1e-8
NOISE_VAR, SEED = 1e-3, 1
ALGOS = ["fista", "admm", "gomp", "biht", "cosamp"]
METRIC = "recovered spectra/s at rel-L2<=1e-3 vs FP64 oracle, mixed vs FP32; % roofline"
UNIT = "spectra/s"
SM_COUNT, SM_MAX_MHZ = 152, 2070.0
# Plain-ALU peaks derived from unit counts x clock (see the design notes):
# FP32: 128 FMA lanes per SM; FP64: 1.25 TFLOP/s for the chip at the maximum clock.
FP32_PEAK_TFLOPS = SM_COUNT * 128 * 2 * SM_MAX_MHZ * 1e6 / 1e12
FP64_PEAK_TFLOPS = 1.25
KERNEL_FILES = {"fista": "fista_tc.cu", "admm": "admm_tc.cu", "measure": "convex_f32.cu",
                "gomp": "greedy.cu", "biht": "greedy.cu", "cosamp": "greedy.cu",
                "sparsify": "sparsify.cu"}


def config(extra=None):
    c = {"workload": f"cube {SIDE}x{SIDE} x N={N}, M={M}; power-law spectra + N(0,1e-3) noise; "
                     f"measure + FISTA({ITERS}) + ADMM({ITERS}) + gOMP(k={KAPPA},G={G}) + "
                     f"BIHT(k={KAPPA}) + CoSaMP(k={KAPPA})",
         "pixels": P, "bands": N, "measurements": M, "algorithms": ALGOS,
         "spectra_per_step": P * len(ALGOS),
         "precision": "FISTA and ADMM split-BF16 tensor cores (mixed; FP32 runs timed "
                      "beside them); greedy FP32 correlation certified against FP64 + FP32 "
                      "Cholesky with FP64 refinement",
         "l2": "flushed between timed steps (256 MiB write)"}
    if extra:
        c.update(extra)
    return c


# ----------------------------------------------------------------------------- oracle leg
def oracle_sample(n_pix, threads, X_true, E, Phi):
    """Runs the FP64 oracle on the first n_pix pixels of the cube; returns outputs and time."""
    import oracle as orc
    A = orc.dictionary(Phi)
    L = orc.lipschitz(A)
    Y = orc.measure(A, X_true[:n_pix], E[:n_pix]).astype(np.float32)
    out, t0 = {}, time.perf_counter()
    out["fista"] = orc.fista(A, Y, L, LAM, EPS, ITERS, threads=threads)[0]
    out["admm"] = orc.admm(A, Y, RHO, LAM, EPS, ITERS, threads=threads)[0]
    out["gomp"] = orc.gomp(A, Y, KAPPA, G, EPS, threads=threads)
    out["biht"] = orc.biht(A, Y, KAPPA, MU, EPS, 100, threads=threads)
    out["cosamp"] = orc.cosamp(A, Y, KAPPA, EPS, 100, threads=threads)
    secs = time.perf_counter() - t0
    return out, secs, Y


# ----------------------------------------------------------------------------- ranks
def rank_seed(rank):
    """Each rank recovers its own cube (pixels are independent: weak scaling)."""
    return SEED + rank


def max_over_ranks(t_ms, dist=None, device="cpu"):
    """The job's step time: the slowest rank's (every rank's cube must be done)."""
    if dist is None:
        return t_ms
    import torch
    tt = torch.tensor([t_ms], device=device, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def job_value(t_ms, world):
    """Recovered spectra per second over the whole job: every rank's pixels, five
    algorithms each, in the slowest rank's step time."""
    return P * len(ALGOS) * world / (t_ms * 1e-3)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def sample_inputs(n_pix):
    from paper_2401_14762_gb300 import synthetic as sy
    Phi = sy.gaussian_phi(M, N, SEED)
    X = sy.powerlaw_coeffs(n_pix, N, SEED)
    E = sy.noise(n_pix, M, NOISE_VAR, SEED)
    return Phi, X, E


def run_reference(args):
    """The oracle as it stands, on the host cores, each step a bounded pixel sample."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n_pix = 2048
    cores = host_cores()
    Phi, X, E = sample_inputs(n_pix)
    for _ in range(args.warmup):
        oracle_sample(32, cores, X, E, Phi)
    times = []
    for _ in range(args.steps):
        _, secs, _ = oracle_sample(n_pix, cores, X, E, Phi)
        times.append(secs)
    t = sum(times) / len(times)
    value = n_pix * len(ALGOS) / t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config({"sample_pixels": n_pix}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"first {n_pix} pixels of the cube, all five algorithms"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = str(device_index)
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(device_index).uuid)
            self.dev = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
        except Exception:
            vis = os.environ.get("CUDA_VISIBLE_DEVICES")
            if vis:
                self.dev = vis.split(",")[device_index]
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.dev, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- GPU leg
def kernel_hash(name):
    src = os.path.join(ROOT, "paper_2401_14762_gb300", "csrc", KERNEL_FILES[name])
    return hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]


def measured_traffic(name):
    """Per-launch DRAM bytes from the committed ncu summary, if taken on this kernel source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path))[name]
    except Exception:
        return None
    if rec.get("source_sha256_16") != kernel_hash(name):
        return None
    return rec.get("dram_bytes_per_launch")


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def run_gpu(args):
    import torch

    from paper_2401_14762_gb300 import build, cs
    from paper_2401_14762_gb300 import synthetic as sy

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    build.build()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    # inputs of this rank's cube (pixels are independent: weak scaling over ranks)
    seed = rank_seed(rank)
    Phi = sy.gaussian_phi(M, N, SEED)
    Xt = sy.powerlaw_coeffs_torch(P, N, seed, dev)
    E = sy.noise_torch(P, M, NOISE_VAR, seed, dev)
    t0 = time.perf_counter()
    ctx = cs.cs_create(M, N, Phi=Phi, admm_rho=RHO, stream=stream.cuda_stream)
    setup_ms = (time.perf_counter() - t0) * 1e3
    Y = torch.empty((P, M), device=dev)
    outs = {a: torch.empty((P, N), device=dev) for a in ALGOS}
    iters = {a: torch.zeros(P, device=dev, dtype=torch.int32) for a in ALGOS}
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    conv = {a: torch.zeros(P, dtype=torch.uint8, device=dev) for a in ALGOS}
    opts = {a: cs.make_opts(eps=EPS, max_iters=100, mu=MU, iters_out=iters[a],
                            converged_out=conv[a]) for a in ALGOS}
    # FISTA runs on the tensor cores (split-BF16, mixed precision); its plain FP32 run is
    # timed beside it for the mixed-vs-FP32 comparison
    opts["fista"] = cs.make_opts(eps=EPS, prec=cs.CS_BF16, iters_out=iters["fista"],
                                 converged_out=conv["fista"])
    opts["admm"] = cs.make_opts(eps=EPS, prec=cs.CS_BF16, iters_out=iters["admm"],
                                converged_out=conv["admm"])
    fista32_out = torch.empty((P, N), device=dev)
    fista32_opts = cs.make_opts(eps=EPS)
    admm32_out = torch.empty((P, N), device=dev)

    work = {}

    def step(ev=None):
        def mark(k):
            if ev is not None:
                ev[k].record(stream)
        mark("start")
        cs.cs_measure(ctx, Xt, Y, E)
        mark("measure")
        cs.cs_recover_fista(ctx, Y, outs["fista"], LAM, ITERS, opts["fista"])
        mark("fista")
        cs.cs_recover_admm(ctx, Y, outs["admm"], RHO, LAM, ITERS, opts["admm"])
        mark("admm")
        cs.cs_recover_gomp(ctx, Y, outs["gomp"], KAPPA, G, opts["gomp"])
        mark("gomp")
        if ev is None:
            work["gomp"] = cs.cs_get_work(ctx)
        cs.cs_recover_biht(ctx, Y, outs["biht"], KAPPA, opts["biht"])
        mark("biht")
        if ev is None:
            work["biht"] = cs.cs_get_work(ctx)
        cs.cs_recover_cosamp(ctx, Y, outs["cosamp"], KAPPA, opts["cosamp"])
        mark("cosamp")
        if ev is None:
            work["cosamp"] = cs.cs_get_work(ctx)

    for _ in range(args.warmup):
        step()
    cs.cs_sync(ctx)
    names = ["start", "measure"] + ALGOS
    per = {k: [] for k in names[1:]}
    step_ms = []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        wall0 = time.perf_counter()
        for _ in range(args.steps):
            flush.fill_(1)  # evict L2 between steps (outside the timed events)
            ev = {k: torch.cuda.Event(enable_timing=True) for k in names}
            step(ev)
            torch.cuda.synchronize()
            prev = "start"
            for k in names[1:]:
                per[k].append(ev[prev].elapsed_time(ev[k]))
                prev = k
            step_ms.append(ev["start"].elapsed_time(ev["cosamp"]))
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
    if dist:
        dist.barrier()
    cs.cs_sync(ctx)
    # the FP32 FISTA and ADMM kernels alone, same input, for the mixed-vs-FP32 comparison
    f32_ms, a32_ms = [], []
    for _ in range(2):
        for call, out, ms in ((lambda o: cs.cs_recover_fista(ctx, Y, o, LAM, ITERS, fista32_opts),
                               fista32_out, f32_ms),
                              (lambda o: cs.cs_recover_admm(ctx, Y, o, RHO, LAM, ITERS,
                                                            cs.make_opts(eps=EPS)),
                               admm32_out, a32_ms)):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            call(out)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
    # CoSaMP and BIHT stop at a repeated iterate (an exact shortcut: same X and iteration
    # counts); their every-iteration runs are timed once beside the step for reference
    full_ms = {}
    for a in ("biht", "cosamp"):
        flush.fill_(1)
        tmp = torch.empty((P, N), device=dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        o = cs.make_opts(eps=EPS, max_iters=100, mu=MU, cycle_skip=False)
        call = cs.cs_recover_biht if a == "biht" else cs.cs_recover_cosamp
        e0.record(stream)
        call(ctx, Y, tmp, KAPPA, o)
        e1.record(stream)
        torch.cuda.synchronize()
        full_ms[a] = (e0.elapsed_time(e1), bool(torch.equal(tmp, outs[a])))
        del tmp
    t_step = max_over_ranks(sum(step_ms) / len(step_ms), dist, dev)
    value = job_value(t_step, world)
    kern_ms = {k: sum(v) / len(v) for k, v in per.items()}

    # ---- end to end: pinned host buffers through the same C calls; the library copies
    # every input in and every result out inside the timed region
    Xh = Xt.cpu().pin_memory()
    Eh = E.cpu().pin_memory()
    Yh = torch.empty((P, M)).pin_memory()
    outh = {a: torch.empty((P, N)).pin_memory() for a in ALGOS}
    e2e_ms = []
    # one untimed pass first: it allocates the library's staging buffers, a one-off
    for rep in range(1 + max(1, min(args.steps, 3))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cs.cs_measure(ctx, Xh, Yh, Eh)
        cs.cs_recover_fista(ctx, Yh, outh["fista"], LAM, ITERS,
                            cs.make_opts(eps=EPS, prec=cs.CS_BF16))
        cs.cs_recover_admm(ctx, Yh, outh["admm"], RHO, LAM, ITERS,
                           cs.make_opts(eps=EPS, prec=cs.CS_BF16))
        cs.cs_recover_gomp(ctx, Yh, outh["gomp"], KAPPA, G, cs.make_opts(eps=EPS))
        cs.cs_recover_biht(ctx, Yh, outh["biht"], KAPPA, cs.make_opts(eps=EPS, mu=MU))
        cs.cs_recover_cosamp(ctx, Yh, outh["cosamp"], KAPPA, cs.make_opts(eps=EPS))
        if rep > 0:
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_t = statistics.median(e2e_ms)  # wall clock: the median is robust to host noise
    push = run_pushbroom(cs, ctx, Yh, outh) if rank == 0 else None
    h2d = P * N * 4 + P * M * 4 + len(ALGOS) * P * M * 4
    d2h = P * M * 4 + len(ALGOS) * P * N * 4

    line = None
    if rank == 0:
        its = {a: iters[a].double().sum().item() for a in ALGOS}
        # roofline of the dominant kernel (algorithmic flops per launch / event time)
        flops = {"fista": 4.0 * M * N * its["fista"],
                 "admm": (4.0 * M * N + 2.0 * M * M) * its["admm"],
                 "measure": 2.0 * M * N * P}
        flops.update(work)  # greedy: algorithmic flops counted by the kernels (warm-up run)
        dom = max(kern_ms, key=kern_ms.get)
        pk = peaks()
        ach = flops[dom] / (kern_ms[dom] * 1e-3) / 1e12
        roof = {"kernel": dom, "bound": "alu", "achieved": ach, "peak": FP32_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": ach / FP32_PEAK_TFLOPS,
                "traffic": measured_traffic(dom),
                "peak_kind": "derived FP32 FMA peak: 152 SMs x 128 lanes x 2 x 2070 MHz",
                "work": "algorithmic flops of the method (correlation, Cholesky least squares "
                        "per support, residual) counted by the kernel"}
        kernels = {}
        for k, ms in kern_ms.items():
            ent = {"ms": ms, "share": ms / t_step}
            if k in flops:
                ach = flops[k] / (ms * 1e-3) / 1e12
                ent.update(tflops=ach, frac_fp32_peak=ach / FP32_PEAK_TFLOPS)
            if k in its:
                ent["mean_iters"] = its[k] / P
            kernels[k] = ent

        # accuracy against the oracle on a sample, and the CPU baseline
        n_s = 6144  # about 10 s of oracle time on 16 host cores
        cores = host_cores()
        Phi_s, Xs, Es = Phi, Xt[:n_s].double().cpu().numpy(), E[:n_s].double().cpu().numpy()
        ref, secs, Ys = oracle_sample(n_s, cores, Xs, Es, Phi_s)
        # the GPU recovers the oracle's own measurements of the sample (same FP32 Y on both
        # sides), with the step's options; the step itself measures on the GPU, and a
        # measurement that differs in its last bit can send a greedy pixel at a near-tie
        # down another trajectory: a property of the input, not of the recovery
        Yd = torch.from_numpy(Ys).to(dev)
        Xa = torch.empty((n_s, N), device=dev)
        calls = {
            "fista": lambda o: cs.cs_recover_fista(ctx, Yd, o, LAM, ITERS,
                                                   cs.make_opts(eps=EPS, prec=cs.CS_BF16)),
            "admm": lambda o: cs.cs_recover_admm(ctx, Yd, o, RHO, LAM, ITERS,
                                                 cs.make_opts(eps=EPS, prec=cs.CS_BF16)),
            "gomp": lambda o: cs.cs_recover_gomp(ctx, Yd, o, KAPPA, G, cs.make_opts(eps=EPS)),
            "biht": lambda o: cs.cs_recover_biht(ctx, Yd, o, KAPPA, cs.make_opts(eps=EPS, mu=MU)),
            "cosamp": lambda o: cs.cs_recover_cosamp(ctx, Yd, o, KAPPA, cs.make_opts(eps=EPS)),
            "fista_fp32": lambda o: cs.cs_recover_fista(ctx, Yd, o, LAM, ITERS, cs.make_opts(eps=EPS)),
            "admm_fp32": lambda o: cs.cs_recover_admm(ctx, Yd, o, RHO, LAM, ITERS,
                                                      cs.make_opts(eps=EPS)),
        }
        import oracle as orc
        Psi = orc.dct2_psi(N)
        acc, psnr = {}, {}
        for a, call in calls.items():
            call(Xa)
            cs.cs_sync(ctx)
            g = Xa.double().cpu().numpy()
            key = a.replace("_fp32", "")
            r = ref[key] if key in ("fista", "admm") else ref[key][0]
            acc[a] = float(np.linalg.norm(g - r) / np.linalg.norm(r))
            # PSNR of each recovery against the true spectra (band domain f = Psi x)
            pg, po = orc.psnr(g, Xs, Psi), orc.psnr(r, Xs, Psi)
            psnr[a] = {"gpu_db": pg, "oracle_db": po, "delta_db": abs(pg - po)}
        # Table I's columns (Section III) on this synthetic cube: PSNR against the true
        # spectra over the whole cube, iterations, the ratio of pixels that met Delta < eps
        # (the iteration cap stands in for the paper's wall-clock cap), recovery time
        # orthonormal DCT-II synthesis matrix (the library's default Psi), built here
        kk = torch.arange(N, dtype=torch.float64, device=dev)
        C = torch.cos(math.pi * (2 * kk[None, :] + 1) * kk[:, None] / (2 * N)) * math.sqrt(2 / N)
        C[0] /= math.sqrt(2)
        Psi_d = C.T
        F_true = Xt.double() @ Psi_d.T
        peak = F_true.abs().max()
        table1 = {}
        for a in ALGOS:
            mse = ((outs[a].double() @ Psi_d.T - F_true) ** 2).mean()
            it_a = iters[a].double()
            table1[a] = {"psnr_db": float(10 * torch.log10(peak * peak / mse)),
                         "iters_mean": float(it_a.mean()), "iters_min": int(it_a.min()),
                         "iters_max": int(it_a.max()),
                         "converged_ratio": float((conv[a] == 1).double().mean()),
                         "recovery_ms": kern_ms[a]}
        del F_true
        f32 = sum(f32_ms) / len(f32_ms)
        kernels["fista_fp32"] = {"ms": f32, "tflops": flops["fista"] / (f32 * 1e-3) / 1e12,
                                 "frac_fp32_peak": flops["fista"] / (f32 * 1e-3) / 1e12 /
                                 FP32_PEAK_TFLOPS}
        kernels["fista"]["precision"] = "split-BF16 tcgen05 (3 MMAs per product), FP32 acc"
        a32 = sum(a32_ms) / len(a32_ms)
        kernels["admm_fp32"] = {"ms": a32, "tflops": flops["admm"] / (a32 * 1e-3) / 1e12,
                                "frac_fp32_peak": flops["admm"] / (a32 * 1e-3) / 1e12 /
                                FP32_PEAK_TFLOPS}
        kernels["admm"]["precision"] = "split-BF16 tcgen05 (3 MMAs per product), FP32 acc"
        kernels["admm"]["speedup_vs_fp32"] = a32 / kern_ms["admm"]
        # tensor-pipe view of the two tcgen05 kernels: MMA flops issued per pixel-iteration
        # (3 split MMAs per product over the 16-padded shapes) against the measured BF16
        # GEMM peak, sustained (both kernels run hundreds of iterations back to back)
        Mp, Np = (M + 15) // 16 * 16, (N + 15) // 16 * 16
        mma = {"fista": 3 * 2 * (2 * Mp * Np), "admm": 3 * 2 * (2 * Mp * Np + Mp * Mp)}
        bf16 = pk.get("bf16_tflops_sustained")
        for a, per in mma.items():
            rate = per * its[a] / (kern_ms[a] * 1e-3) / 1e12
            kernels[a]["mma_tflops"] = rate
            kernels[a]["frac_bf16_sustained_of_measured"] = rate / bf16 if bf16 else None
        for a, (ms, same) in full_ms.items():
            kernels[a]["every_iteration_ms"] = ms
            kernels[a]["every_iteration_bitwise_equal"] = same
        kernels["fista"]["speedup_vs_fp32"] = f32 / kern_ms["fista"]
        cpu_value = n_s * len(ALGOS) / secs
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic",
                "config": config({"setup_ms": setup_ms, "wall_ms_per_step": wall * 1e3 / args.steps}),
                "roofline": roof,
                "cpu_baseline": {"value": cpu_value, "unit": UNIT, "cores": cores, "kind": "oracle",
                                 "sample": f"first {n_s} pixels of the cube, all five algorithms, "
                                           f"{secs:.1f} s"},
                "e2e": {"value": P * len(ALGOS) / (e2e_t * 1e-3), "unit": UNIT,
                        "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
                # measure, FISTA momentum table + FISTA, ADMM, and for each of gOMP, BIHT
                # and CoSaMP its cube-descriptor upload + the recovery kernel
                "gpu_launches": 10 * args.steps,
                "clocks": clk.summary(),
                "kernels": kernels,
                "accuracy_rel_l2_vs_oracle": acc,
                "psnr_vs_truth": psnr,
                "table1": table1,
                "pushbroom": push,
                "accuracy_inputs": f"the oracle's FP32 measurements of the first {n_s} pixels, "
                                   "recovered by both sides with the step's options",
                "peaks_file": {k: pk.get(k) for k in ("hbm_gbs", "bf16_tflops")}}
    if line is not None:
        line["sparsify"] = run_sparsify(cs, ctx, Xt, dev, stream, flush)
    cs.cs_destroy(ctx)
    if rank == 0 and not args.no_batch:
        line["batch"] = run_batch(cs, sy, dev, stream, flush)
    if line is not None:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_pushbroom(cs, ctx, Yh, outh, lines=64):
    """Pushbroom mode (Section II): each recovery of the cube from pinned host memory,
    once as one host-pointer call (copy in, recover, copy out) and once streamed in
    chunks of `lines` sensor lines with copies overlapping the recoveries
    (cs_recover_stream).  Wall-clock per call, after one untimed call of each."""
    chunk = lines * SIDE
    calls = {
        "fista": (cs.CS_ALGO_FISTA, dict(lam=LAM, iters=ITERS),
                  cs.make_opts(eps=EPS, prec=cs.CS_BF16),
                  lambda o: cs.cs_recover_fista(ctx, Yh, o, LAM, ITERS,
                                                cs.make_opts(eps=EPS, prec=cs.CS_BF16))),
        "admm": (cs.CS_ALGO_ADMM, dict(lam=LAM, rho=RHO, iters=ITERS),
                 cs.make_opts(eps=EPS, prec=cs.CS_BF16),
                 lambda o: cs.cs_recover_admm(ctx, Yh, o, RHO, LAM, ITERS,
                                              cs.make_opts(eps=EPS, prec=cs.CS_BF16))),
        "gomp": (cs.CS_ALGO_GOMP, dict(kappa=KAPPA, G=G), cs.make_opts(eps=EPS),
                 lambda o: cs.cs_recover_gomp(ctx, Yh, o, KAPPA, G, cs.make_opts(eps=EPS))),
        "biht": (cs.CS_ALGO_BIHT, dict(kappa=KAPPA), cs.make_opts(eps=EPS, mu=MU),
                 lambda o: cs.cs_recover_biht(ctx, Yh, o, KAPPA, cs.make_opts(eps=EPS, mu=MU))),
        "cosamp": (cs.CS_ALGO_COSAMP, dict(kappa=KAPPA), cs.make_opts(eps=EPS),
                   lambda o: cs.cs_recover_cosamp(ctx, Yh, o, KAPPA, cs.make_opts(eps=EPS))),
    }
    out = {"chunk_pixels": chunk, "lines_per_chunk": lines}
    for a, (code, prm, opts, whole) in calls.items():
        o = outh[a]
        res = {}
        for mode in ("whole", "stream"):
            for rep in range(2):
                t0 = time.perf_counter()
                if mode == "whole":
                    whole(o)
                else:
                    cs.cs_recover_stream(ctx, code, Yh, o, chunk, opts=opts, **prm)
                if rep:
                    res[mode + "_ms"] = (time.perf_counter() - t0) * 1e3
        out[a] = res
    out["stream_spectra_per_s"] = len(calls) * Yh.shape[0] / (
        sum(out[a]["stream_ms"] for a in calls) * 1e-3)
    out["whole_spectra_per_s"] = len(calls) * Yh.shape[0] / (
        sum(out[a]["whole_ms"] for a in calls) * 1e-3)
    return out


def run_sparsify(cs, ctx, Xt, dev, stream, flush, T=0.1):
    """The sparsification pre-processing of Section II (outside the step): the cube's
    spectra f = Psi x + white noise (std 0.01), T = 0.1 as in the paper's experiments.
    One FP32 transform per pixel (2 N^2 flops) with FP64-certified decisions; the
    algorithmic traffic is F in, X out and kappa out."""
    import torch
    P_, N_ = Xt.shape
    kk = torch.arange(N_, dtype=torch.float64, device=dev)
    C = torch.cos(math.pi * (2 * kk[None, :] + 1) * kk[:, None] / (2 * N_)) * math.sqrt(2 / N_)
    C[0] /= math.sqrt(2)
    g = torch.Generator(device=dev)
    g.manual_seed(SEED)
    F = (Xt.double() @ C + 0.01 * torch.randn((P_, N_), generator=g, device=dev,
                                             dtype=torch.float64)).float()
    X = torch.empty_like(F)
    kap = torch.empty(P_, dtype=torch.int16, device=dev)
    rec = torch.zeros(1, dtype=torch.int64, device=dev)
    for _ in range(3):
        cs.cs_sparsify(ctx, F, X, T, 1, kap, rec)
    ms = []
    for _ in range(5):
        flush.fill_(1)
        rec.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        cs.cs_sparsify(ctx, F, X, T, 1, kap, rec)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    cs.cs_sync(ctx)
    t = statistics.median(ms)
    flops = 2.0 * N_ * N_ * P_
    nbytes = P_ * (8 * N_ + 2)
    pk = peaks()
    return {"workload": f"{P_} spectra x N={N_}, power law + N(0, 1e-4) noise, T={T}, "
                        "sample std",
            "ms": t, "spectra_per_s": P_ / (t * 1e-3),
            "tflops": flops / (t * 1e-3) / 1e12,
            "frac_fp32_peak": flops / (t * 1e-3) / 1e12 / FP32_PEAK_TFLOPS,
            "gbs": nbytes / (t * 1e-3) / 1e9,
            "frac_hbm_of_measured": nbytes / (t * 1e-3) / 1e9 / pk["hbm_gbs"]
            if pk.get("hbm_gbs") else None,
            "traffic": measured_traffic("sparsify"),
            "algorithmic_bytes": nbytes,
            "pixels_decided_in_fp64": int(rec.item()),
            "zeroed_fraction": float((X == 0).double().mean()),
            "kappa_mean": float(kap.double().mean()),
            "l2": "flushed before each timed run"}


def run_batch(cs, sy, dev, stream, flush):
    """The batching workload: 64 cubes of uneven sizes (side U{64..512}), N in
    {120, 200, 224}, M = round(0.4 N), one Gaussian Phi per cube, exactly sparse pixels
    with per-pixel S ~ U{4..32}, noiseless.  gOMP (kappa = S per pixel, G = max(1,
    floor(S/5))) runs all cubes in one cs_recover_batch launch; FISTA (300 iterations,
    FP32) one launch per cube.  Timed once each after a warm-up on two cubes; the FP64
    oracle on 32 pixels of three cubes gives the accuracy."""
    import torch
    import oracle as orc
    recipe = sy.batch_recipe(SEED)
    cubes = []
    for i, r in enumerate(recipe):
        M_, N_, P_ = r["M"], r["N"], r["side"] * r["side"]
        Phi = sy.gaussian_phi(M_, N_, 1000 + i)
        ctx = cs.cs_create(M_, N_, Phi=Phi, stream=stream.cuda_stream)
        g = torch.Generator(device=dev)
        g.manual_seed(7919 * (i + 1))
        S = torch.randint(4, 33, (P_,), generator=g, device=dev)
        X = sy.sparse_coeffs_torch(P_, N_, S, 1000 + i, dev)
        Y = torch.empty((P_, M_), device=dev)
        cs.cs_measure(ctx, X, Y)
        cubes.append(dict(ctx=ctx, Phi=Phi, X=X, Y=Y, S=S.to(torch.int16), M=M_, N=N_, P=P_,
                          Xg=torch.empty((P_, N_), device=dev),
                          Xf=torch.empty((P_, N_), device=dev),
                          it=torch.empty(P_, device=dev, dtype=torch.int32)))
    total = sum(c["P"] for c in cubes)
    g_items = [dict(ctx=c["ctx"], Y=c["Y"], X=c["Xg"], kappa_per_pixel=c["S"],
                    iters_out=c["it"]) for c in cubes]
    f_items = [dict(ctx=c["ctx"], Y=c["Y"], X=c["Xf"]) for c in cubes]
    g_opts = cs.make_opts(eps=EPS)
    f_opts = cs.make_opts(eps=EPS, prec=cs.CS_FP32)
    cs.cs_recover_batch(g_items[:2], cs.CS_ALGO_GOMP, kappa=32, G=0, opts=g_opts)
    cs.cs_recover_batch(f_items[:2], cs.CS_ALGO_FISTA, lam=LAM, iters=ITERS, opts=f_opts)
    cs.cs_sync(cubes[0]["ctx"])
    times = {}
    for name, call in (("gomp", lambda: cs.cs_recover_batch(g_items, cs.CS_ALGO_GOMP, kappa=32,
                                                            G=0, opts=g_opts)),
                       ("fista", lambda: cs.cs_recover_batch(f_items, cs.CS_ALGO_FISTA, lam=LAM,
                                                             iters=ITERS, opts=f_opts))):
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        call()
        e1.record(stream)
        torch.cuda.synchronize()
        times[name] = e0.elapsed_time(e1)
    cs.cs_sync(cubes[0]["ctx"])
    # accuracy on 32 pixels of the first cube of each band count
    acc = {"gomp": [], "fista": []}
    cond = []  # the oracle FISTA output's sensitivity to a relative perturbation of y
    seen = set()
    for c in cubes:
        if c["N"] in seen:
            continue
        seen.add(c["N"])
        A = orc.dictionary(c["Phi"])
        Xs = c["X"][:32].double().cpu().numpy()
        Ys = orc.measure(A, Xs).astype(np.float32)
        S = c["S"][:32].cpu().numpy().astype(int)
        Xo = np.zeros_like(Xs)
        for k in np.unique(S):
            sel = S == k
            Xo[sel] = orc.gomp(A, Ys[sel], int(k), max(1, int(k) // 5), EPS)[0]
        Lf = orc.lipschitz(A)
        Xfo = orc.fista(A, Ys, Lf, LAM, EPS, ITERS)[0]
        pert = Ys.astype(np.float64) * (1.0 + 1e-7 * np.random.default_rng(5).standard_normal(Ys.shape))
        Xfp = orc.fista(A, pert, Lf, LAM, EPS, ITERS)[0]
        cond.append(float(np.linalg.norm(Xfp - Xfo) / np.linalg.norm(Xfo) / 1e-7))
        for key, ref, got in (("gomp", Xo, c["Xg"]), ("fista", Xfo, c["Xf"])):
            g = got[:32].double().cpu().numpy()
            acc[key].append(float(np.linalg.norm(g - ref) / np.linalg.norm(ref)))
    out = {"workload": "64 cubes, side U{64..512}, N in {120,200,224}, M=0.4N, one Phi per "
                       "cube, exactly sparse with per-pixel S ~ U{4..32}, noiseless",
           "cubes": len(cubes), "pixels": total,
           "gomp": {"ms": times["gomp"], "spectra_per_s": total / (times["gomp"] * 1e-3),
                    "launch": "one persistent cs_recover_batch launch over all cubes",
                    "mean_iters": float(sum(c["it"].double().sum().item() for c in cubes)) / total,
                    "rel_l2_vs_oracle_max": max(acc["gomp"])},
           "fista": {"ms": times["fista"], "spectra_per_s": total / (times["fista"] * 1e-3),
                     "launch": "one launch per cube (FP32 path)",
                     "rel_l2_vs_oracle_max": max(acc["fista"]),
                     # after 300 unconverged iterations the oracle's own output moves by
                     # kappa x a relative input change; FP32 rounding injected at every
                     # iteration then allows about 4 sqrt(K) kappa 2^-24
                     "oracle_conditioning_max": max(cond),
                     "fp32_tolerance_from_conditioning": 4 * np.sqrt(ITERS) * max(cond) * 2.0 ** -24},
           "accuracy_sample": "32 pixels of one cube per band count, FP64 oracle"}
    for c in cubes:
        cs.cs_destroy(c["ctx"])
    return out


def run_only(args):
    """One algorithm of the step on the first P pixels of the workload, called twice (the
    first call is a warm-up), for kernel profiles; prints nothing but a short status."""
    import torch

    from paper_2401_14762_gb300 import build, cs
    from paper_2401_14762_gb300 import synthetic as sy
    build.build()
    dev = torch.device("cuda", 0)
    n = args.pixels
    Phi = sy.gaussian_phi(M, N, SEED)
    Xt = sy.powerlaw_coeffs_torch(n, N, SEED, dev)
    E = sy.noise_torch(n, M, NOISE_VAR, SEED, dev)
    ctx = cs.cs_create(M, N, Phi=Phi, admm_rho=RHO, stream=torch.cuda.current_stream().cuda_stream)
    Y = torch.empty((n, M), device=dev)
    cs.cs_measure(ctx, Xt, Y, E)
    X = torch.empty((n, N), device=dev)
    mixed = cs.make_opts(eps=EPS, prec=cs.CS_BF16)
    calls = {
        "measure": lambda: cs.cs_measure(ctx, Xt, Y, E),
        "fista": lambda: cs.cs_recover_fista(ctx, Y, X, LAM, ITERS, mixed),
        "fista_fp32": lambda: cs.cs_recover_fista(ctx, Y, X, LAM, ITERS, cs.make_opts(eps=EPS)),
        "admm": lambda: cs.cs_recover_admm(ctx, Y, X, RHO, LAM, ITERS, mixed),
        "admm_fp32": lambda: cs.cs_recover_admm(ctx, Y, X, RHO, LAM, ITERS, cs.make_opts(eps=EPS)),
        "gomp": lambda: cs.cs_recover_gomp(ctx, Y, X, KAPPA, G, cs.make_opts(eps=EPS)),
        "biht": lambda: cs.cs_recover_biht(ctx, Y, X, KAPPA, cs.make_opts(eps=EPS, mu=MU)),
        "cosamp": lambda: cs.cs_recover_cosamp(ctx, Y, X, KAPPA, cs.make_opts(eps=EPS)),
        # the sparsification pre-processing on spectra f = Psi x (here X holds f)
        "sparsify": lambda: cs.cs_sparsify(ctx, F, X, 0.1, 1),
    }
    if args.only == "sparsify":
        kk = torch.arange(N, dtype=torch.float64, device=dev)
        C = torch.cos(math.pi * (2 * kk[None, :] + 1) * kk[:, None] / (2 * N)) * math.sqrt(2 / N)
        C[0] /= math.sqrt(2)
        g = torch.Generator(device=dev)
        g.manual_seed(SEED)
        F = (Xt.double() @ C + 0.01 * torch.randn((n, N), generator=g, device=dev,
                                                 dtype=torch.float64)).float()
    for _ in range(2):
        calls[args.only]()
    cs.cs_sync(ctx)
    torch.cuda.synchronize()
    print(f"ok {args.only} {n} pixels", flush=True)
    cs.cs_destroy(ctx)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--only", default=None,
                    choices=["measure", "fista", "fista_fp32", "admm", "admm_fp32", "gomp",
                             "biht", "cosamp", "sparsify"])
    ap.add_argument("--pixels", type=int, default=16384)
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the 64-cube batching measurement")
    args = ap.parse_args()
    if args.only:
        run_only(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
