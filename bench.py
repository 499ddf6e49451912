"""Benchmark of the exact RNS integer product (rns_reduce -> residue_gemm ->
crt_reconstruct) on the 4096 x 4096 (int64, |a| <= 2^20) by 4096 x 256
(512-bit) workload.

One step = one whole exact product C = A B through the C ABI (reduce both
operands, all residue products, CRT), inputs resident in HBM.  Prints one JSON
line (rank 0).  `--impl reference` times the CPU oracle instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Smith-form s/matrix and exact residue-GEMM TOPS, INT8-limb vs FP64-residue, bit-exact"
M_, K_, N_ = 4096, 4096, 256
A_BITS, B_WORDS, C_WORDS = 20, 8, 9
WORKLOAD = "rns_matmul: A 4096x4096 int64 uniform [-2^20,2^20] x B 4096x256 uniform signed 512-bit, exact C (9 words)"
EFF_OPS = 2 * M_ * N_ * K_  # effective integer-product operations per step


# DRAM bytes (read + write) of one launch of the residue-GEMM kernel on this
# workload, from a single-pass ncu capture of dram__bytes_read.sum and
# dram__bytes_write.sum.  Reported only while the kernel source (the kernel file
# and its PTX helpers) is the one the counters were taken on.
GEMM_TRAFFIC = {"source_sha256": "0e6a550177217bb6041c36171188832434f344c492dc98219add970f9cca330a",
                "bytes": 857_507_712 + 120_614_528}  # mean of two captured launches


def _gemm_traffic():
    import hashlib
    h = hashlib.sha256()
    try:
        for name in ("gemm_limb.cu", "tc_ptx.h"):  # the kernel and its PTX helpers
            h.update(open(os.path.join(ROOT, "paper_2605_19254_gb300", "csrc", name), "rb").read())
    except OSError:
        return None
    sha = h.hexdigest()
    return GEMM_TRAFFIC["bytes"] if GEMM_TRAFFIC["source_sha256"] == sha else None


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d.get("bf16_tflops"), d.get("hbm_gbs"), "measured"
    except Exception:
        return 1900.0, 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples (20 ms period), kept for the timed region."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.window = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def mark(self, t0, t1):
        self.window = (t0, t1)

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.05)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = []
        for ts, ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) >= 10:
                rows.append((ts, f))
        if self.window:  # samples that arrived during the timed region (+ one period of slack)
            inside = [r for r in rows if self.window[0] <= r[0] <= self.window[1] + 0.04]
            rows = inside if inside else rows[-2:]
        for ts, f in rows:
            try:
                sm.append(float(f[2]))
                mx = float(f[3])
            except ValueError:
                continue
            for nm, v in zip(names, f[6:10]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    from paper_2605_19254_gb300 import replicas

    e = replicas.rank_env()
    return e.world_size, e.rank, e.local_rank


def cpu_baseline(target_s: float = 12.0):
    """The oracle's schoolbook product on a bounded row sample of the workload."""
    import numpy as np

    import oracle
    from paper_2605_19254_gb300 import inputs

    oracle.build()
    A, B = inputs.rns_matmul_workload(0, M_, K_, N_, A_BITS, B_WORDS)
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    rows = max(1, cores)
    t0 = time.perf_counter()
    oracle.matmul(A[:rows], B, C_WORDS)
    dt = time.perf_counter() - t0
    # scale the sample to about target_s of CPU work
    rows2 = int(min(M_, max(rows, rows * target_s / max(dt, 1e-3))))
    rows2 = max(cores, rows2 // cores * cores)
    t0 = time.perf_counter()
    oracle.matmul(A[:rows2], B, C_WORDS)
    dt2 = time.perf_counter() - t0
    ops = 2 * rows2 * N_ * K_
    return {"value": ops / dt2 / 1e12, "unit": "TOPS", "cores": cores, "kind": "oracle",
            "sample": f"{rows2} of 4096 rows of C (x256 cols, K=4096), schoolbook big-integer product, "
                      f"{dt2:.2f} s"}


def paper_design_matmul(A, B, Wc, primes=None, rb=None):
    """Exact C = A B by the paper's own design (Section 3.1), on the host: residues
    modulo word-size primes below the bound K (p-1)^2 + (p-1) < 2^53, one float64
    GEMM per prime (exact under that bound; torch's CPU BLAS in place of the
    paper's dgemm), reduction of each product modulo p, and CRT back to integers.
    A: [M, K, Wa], B: [K, N, Wb] uint64 words -> [M, N, Wc] words.
    Reduction and CRT use the oracle's C routines; it is a baseline, not the path."""
    import numpy as np
    import torch

    import oracle

    K = A.shape[1]
    if primes is None:
        bits = 64 * A.shape[2] - 1 + 64 * B.shape[2] - 1 + int(np.ceil(np.log2(max(K, 2))))
        primes = oracle.basis(oracle.fp64_prime_cap(K) + 1, bits)
    ra = oracle.reduce(A, primes).astype(np.float64)
    if rb is None:
        rb = oracle.reduce(B, primes).astype(np.float64)
    prod = np.empty((len(primes), A.shape[0], B.shape[1]), dtype=np.int32)
    for i, p in enumerate(primes):
        c = torch.from_numpy(ra[i]) @ torch.from_numpy(rb[i])
        prod[i] = torch.remainder(c, float(p)).numpy().astype(np.int32)
    return oracle.crt(prod, primes, Wc)


def cpu_paper_design(target_s: float = 10.0):
    """paper_design_matmul on a bounded row sample of the workload, timed on the host
    cores.  B is reduced once (timed separately) and its share is pro-rated to the
    sampled rows, as one full product would reduce it once for all M rows."""
    import numpy as np
    import torch

    import oracle
    from paper_2605_19254_gb300 import inputs

    oracle.build()
    A, B = inputs.rns_matmul_workload(0, M_, K_, N_, A_BITS, B_WORDS)
    primes = oracle.basis(oracle.fp64_prime_cap(K_) + 1, A_BITS + 64 * B_WORDS - 1 + 12)
    t0 = time.perf_counter()
    rb = oracle.reduce(B, primes).astype(np.float64)
    t_b = time.perf_counter() - t0
    rows = 128
    t0 = time.perf_counter()
    paper_design_matmul(A[:rows], B, C_WORDS, primes, rb)
    dt = time.perf_counter() - t0
    rows2 = int(min(M_, max(rows, rows * target_s / max(dt, 1e-3))))
    rows2 = max(128, rows2 // 128 * 128)
    t0 = time.perf_counter()
    paper_design_matmul(A[:rows2], B, C_WORDS, primes, rb)
    dt2 = time.perf_counter() - t0 + t_b * rows2 / M_
    return {"value": 2 * rows2 * N_ * K_ / dt2 / 1e12, "unit": "TOPS", "cores": torch.get_num_threads(),
            "kind": "paper design on the host: float64 GEMM per prime",
            "sample": f"{rows2} of 4096 rows of C, {len(primes)} primes below 2^20.5 (K (p-1)^2 < 2^53): reduce of "
                      f"A's rows + {len(primes)} GEMMs + CRT, plus B's reduction ({t_b:.2f} s) pro-rated, {dt2:.2f} s"}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    from paper_2605_19254_gb300 import inputs
    oracle.build()
    A, B = inputs.rns_matmul_workload(0, M_, K_, N_, A_BITS, B_WORDS)
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    rows = max(cores, 2 * cores)
    for _ in range(args.warmup):
        oracle.matmul(A[:cores], B, C_WORDS)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.matmul(A[:rows], B, C_WORDS)
        times.append(time.perf_counter() - t0)
    per = statistics.mean(times)
    value = 2 * rows * N_ * K_ / per / 1e12
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "TOPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "throughput": "effective 2*M*N*K per second over the computed rows",
                       "sample_rows": rows},
            "cpu_baseline": {"value": value, "unit": "TOPS", "cores": cores, "kind": "oracle",
                             "sample": f"{rows} of 4096 rows of C per step (x256 cols, K=4096)"},
            "e2e": {"value": value, "unit": "TOPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run(args):
    import numpy as np
    import torch

    from paper_2605_19254_gb300 import build, inputs, replicas, smf

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0:
        build.build()
    if ws > 1:
        torch.distributed.barrier()
    build.build()

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    # replicas: one independent product per rank (weak scaling); split: the rows of
    # one product's A and C over the ranks, B replicated (strong scaling)
    split = ws > 1 and args.parallel == "split"
    A_np, B_np = inputs.rns_matmul_workload(0 if split else replicas.rank_seed(0, rank), M_, K_, N_, A_BITS,
                                            B_WORDS)
    m0, m1 = replicas.row_block(M_, ws, rank) if split else (0, M_)
    Mr = m1 - m0  # rows this rank computes
    A = torch.from_numpy(np.ascontiguousarray(A_np[m0:m1]).view(np.int64)).to(dev)
    B = torch.from_numpy(B_np.view(np.int64)).to(dev)
    C = torch.zeros((Mr, N_, C_WORDS), dtype=torch.int64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > L2 (129 MB)
    stream = torch.cuda.current_stream(dev)

    window = [None]

    def measure(form, steps, warmup, prof=False, fused=False):
        ctx = smf.Context(local, form)
        ctx.set_fused_crt(fused)
        wsb = ctx.rns_matmul_workspace(A, B, C, a_bits=A_BITS)
        work = torch.empty(wsb, dtype=torch.uint8, device=dev)
        for _ in range(warmup):
            ctx.rns_matmul(A, B, C, a_bits=A_BITS, workspace=work, stream=stream)
        ctx.status_sync(stream)
        if prof:
            ctx.profile_enable(True)
            ctx.profile_read()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        torch.cuda.synchronize(dev)
        barrier()
        t_wall = time.perf_counter()
        t_epoch0 = time.time()
        for s0, s1 in evs:
            flush.fill_(1)  # untimed: evict L2 between steps
            s0.record(stream)
            ctx.rns_matmul(A, B, C, a_bits=A_BITS, workspace=work, stream=stream)
            s1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        t_wall = time.perf_counter() - t_wall
        window[0] = (t_epoch0, time.time())
        ctx.status_sync(stream)
        ms = [a.elapsed_time(b) for a, b in evs]
        prof_d = ctx.profile_read() if prof else None
        ctx.destroy()
        return statistics.mean(ms), ms, prof_d, t_wall, wsb

    form_main = smf.SMF_FORM_INT8LIMB if args.form == "limb" else smf.SMF_FORM_FP64
    with ClockSampler(local) as clk:
        ms_main, ms_list, _, wall, wsb = measure(form_main, args.steps, args.warmup)
        clk.mark(*window[0])
    clocks = clk.summary()
    # per-kernel times (CUDA events on the launching stream) in a second pass
    _, _, prof, _, _ = measure(form_main, max(3, min(args.steps, 10)), 1, prof=True)
    ms_main = replicas.max_over_ranks(ms_main, ws, dev)

    # bit-exactness spot check of this run's output against nothing but itself is
    # not a check; the parity suite covers it.  Here: the FP64-residue form on the
    # same workload for the INT8-limb vs FP64 comparison.
    fp64 = None
    if rank == 0 and args.form == "limb" and not args.skip_fp64:
        ms_f, _, prof_f, _, _ = measure(smf.SMF_FORM_FP64, 2, 1, prof=True)
        gemm_f = prof_f["residue_gemm"][1] / max(1, prof_f["residue_gemm"][0])
        pctx = smf.Context(local, smf.SMF_FORM_FP64)
        fp64_peak = pctx.fp64_peak(stream)
        pb = pctx.basis_create(A_BITS + 64 * B_WORDS - 1 + 12, 1 << 26)
        L_f = len(pb.primes)
        pb.destroy()
        pctx.destroy()
        fp64_flops = 2 * Mr * N_ * K_ * L_f  # one fp64 fma per residue product term, per prime
        fp64 = {"value": 2 * Mr * N_ * K_ / (ms_f * 1e-3) / 1e12, "unit": "TOPS", "ms_per_step": ms_f,
                "residue_gemm_ms": gemm_f,
                "roofline": {"bound": "fp64", "kernel": "gemm_fp64_kernel", "unit": "TFLOP/s",
                             "achieved": fp64_flops / (gemm_f * 1e-3) / 1e12, "peak": fp64_peak,
                             "frac": fp64_flops / (gemm_f * 1e-3) / 1e12 / fp64_peak if fp64_peak else None,
                             "peak_kind": "measured FP64 FMA throughput (smf_fp64_peak: register-resident fma "
                                          "chains on every SM, CUDA events)", "primes": L_f}}

    # the residue product with the CRT in its epilogue (one kernel for both)
    fused = None
    if rank == 0 and args.form == "limb":
        ms_fz, _, _, _, _ = measure(form_main, args.steps, args.warmup, fused=True)
        _, _, prof_fz, _, _ = measure(form_main, max(3, min(args.steps, 10)), 1, prof=True, fused=True)
        fused = {"value": EFF_OPS / (ms_fz * 1e-3) / 1e12, "unit": "TOPS", "ms_per_step": ms_fz,
                 "kernel": "limb_gemm_crt_kernel", "per_kernel_ms": {
                     k: (v[1] / v[0] if v[0] else 0.0) for k, v in prof_fz.items()}}

    # end to end through the C ABI with pinned host buffers (copies timed)
    Ah = A.cpu().pin_memory()
    Bh = B.cpu().pin_memory()
    Ch = torch.zeros((Mr, N_, C_WORDS), dtype=torch.int64).pin_memory()
    ctx = smf.Context(local, form_main)
    work = torch.empty(ctx.rns_matmul_workspace(Ah, Bh, Ch, a_bits=A_BITS), dtype=torch.uint8, device=dev)
    for _ in range(2):
        ctx.rns_matmul(Ah, Bh, Ch, a_bits=A_BITS, workspace=work, stream=stream)
    ctx.status_sync(stream)
    e2e_steps = max(3, min(args.steps, 10))
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ctx.rns_matmul(Ah, Bh, Ch, a_bits=A_BITS, workspace=work, stream=stream)
    torch.cuda.synchronize(dev)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    ctx.status_sync(stream)
    ctx.destroy()
    e2e_s = replicas.max_over_ranks(e2e_s, ws, dev)

    if rank != 0:
        return
    # replicas: every rank's product counts; split: the ranks share one product
    job_ops = EFF_OPS if split else EFF_OPS * ws
    value = job_ops / (ms_main * 1e-3) / 1e12
    peak_tf, hbm, peak_kind = _peaks()
    gemm_n, gemm_ms = prof["residue_gemm"]
    gemm_avg = gemm_ms / max(1, gemm_n)
    bctx = smf.Context(local, form_main)
    bas = bctx.basis_create(A_BITS + 64 * B_WORDS - 1 + 12)  # |C| <= 4096 * 2^20 * 2^511
    L = len(bas.primes)
    h_small, h_big = min(bas.primes) // 2, max(bas.primes) // 2
    bas.destroy()
    bctx.destroy()

    def digits(h):  # balanced base-2^8 digits covering |x| <= h (top digit up to 128)
        t, lower, scale = 1, 0, 1
        while 128 * scale + lower < h:
            lower += 127 * scale
            scale *= 256
            t += 1
        return t

    TA = digits(1 << A_BITS) if (1 << A_BITS) <= h_small else digits(h_big)
    TB = digits(h_big)
    amax = (1 << A_BITS) if (1 << A_BITS) <= h_small else h_big

    def digit_bound(h, t, u):  # largest |digit u| of |x| <= h in t balanced digits
        if u < t - 1:
            return 128
        lower = sum(128 * 256 ** i for i in range(t - 1))
        return (h + lower) // 256 ** (t - 1)

    worst = max(sum(digit_bound(amax, TA, u) * digit_bound(h_big, TB, d - u)
                    for u in range(TA) if 0 <= d - u < TB) for d in range(TA + TB - 1))
    fold_products = (1 << 24) // worst // 64 * 64
    wide = (TA, TB) == (3, 3)
    gemm_kernel = "limb_gemm_wide_kernel (BN=64)" if wide else f"limb_gemm_kernel<{TA},{TB},48>"
    mma_n = 192 if wide else TB * 48
    if form_main == smf.SMF_FORM_INT8LIMB:
        flops = 2 * Mr * N_ * K_ * L * TA * TB  # digit-product MMA work of one launch
        roofline = {"bound": "tensor", "achieved": flops / (gemm_avg * 1e-3) / 1e12, "peak": peak_tf,
                    "unit": "TFLOP/s", "frac": None, "traffic": _gemm_traffic(),
                    "kernel": gemm_kernel, "peak_kind": f"bf16 dense burst ({peak_kind})"}
        roofline["frac"] = roofline["achieved"] / roofline["peak"]
    else:
        flops = 2 * Mr * N_ * K_ * L
        pctx = smf.Context(local, form_main)
        fpk = pctx.fp64_peak(stream)
        pctx.destroy()
        roofline = {"bound": "fp64", "achieved": flops / (gemm_avg * 1e-3) / 1e12, "peak": fpk,
                    "unit": "TFLOP/s", "frac": None, "traffic": None, "kernel": "gemm_fp64_kernel",
                    "peak_kind": "measured FP64 FMA throughput (smf_fp64_peak)"}
        roofline["frac"] = roofline["achieved"] / fpk if fpk else None
    # the reduce phase and the CRT: algorithmic HBM bytes over their measured time
    # (both are integer-issue bound; their issue-slot fractions come from ncu)
    red_ms = prof["reduce"][1] / max(1, prof["reduce"][0])
    crt_ms = prof["crt"][1] / max(1, prof["crt"][0])
    if form_main == smf.SMF_FORM_INT8LIMB:
        red_bytes = Mr * K_ * 8 + TA * Mr * K_ * 2 + K_ * N_ * B_WORDS * 8 + TB * L * K_ * N_ * 2
    else:
        red_bytes = Mr * K_ * 8 + Mr * K_ * 4 + K_ * N_ * B_WORDS * 8 + L * K_ * N_ * 4
    crt_bytes = L * Mr * N_ * 4 + Mr * N_ * C_WORDS * 8
    secondary = {
        name: {"ms": ms, "algorithmic_bytes": nbytes, "hbm_gbs": nbytes / (ms * 1e-3) / 1e9,
               "hbm_frac": nbytes / (ms * 1e-3) / 1e9 / hbm if hbm else None, "bound": "integer issue"}
        for name, ms, nbytes in (("reduce_phase", red_ms, red_bytes), ("crt", crt_ms, crt_bytes)) if ms > 0}
    out = {
        "metric": METRIC, "value": value, "unit": "TOPS", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_main, "higher_is_better": True,
        "scaling": "strong" if split else "weak",
        "vs_baseline": None, "dtype": "bf16-digits/fp32-acc -> exact int" if args.form == "limb" else "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "form": args.form,
                   "throughput": "effective exact integer-product ops 2*M*N*K per second (whole step)",
                   "primes": L, "digits": [TA, TB] if args.form == "limb" else None,
                   "engine": (f"tcgen05.mma kind::f16 M=128 N={mma_n}, 8-bit digits exact in bf16, fp32 TMEM "
                              f"accumulation per digit weight, drained every {fold_products} products")
                   if args.form == "limb" else "fp64 FMA, k-blocked",
                   "l2": "256 MB buffer written between timed steps (untimed)",
                   "parallelism": (f"row-block split x{ws}: each rank computes about {Mr} rows of A and C, B "
                                   "replicated, no exchange" if split else f"replicas x{ws}")},
        "per_kernel_ms": {k: (v[1] / v[0] if v[0] else 0.0) for k, v in prof.items()},
        "residue_gemm_tops": 2 * Mr * N_ * K_ * L / (gemm_avg * 1e-3) / 1e12,
        "roofline": roofline,
        "secondary_rooflines": secondary,
        "fused_crt": fused,
        "fp64_form": fp64,
        "e2e": {"value": job_ops / e2e_s / 1e12, "unit": "TOPS",
                "h2d_bytes_per_step": int(Ah.numel() * 8 + Bh.numel() * 8),
                "d2h_bytes_per_step": int(Ch.numel() * 8)},
        "gpu_launches": 4 * args.steps,
        "clocks": clocks,
        "wall_s_timed_region": wall,
    }
    out["base_convert"] = run_base_convert(dev, local, stream, flush, 50, hbm)
    out["padic_lift"] = run_lift(dev, local)
    out["largest_invariant_factor"] = run_lif(dev, local)
    if not args.skip_smith:
        out["smith_form"] = run_smith(dev, local, with_fp64=not args.skip_fp64)
        out["smith_serving"] = run_smith_serving(dev, local, with_fp64=not args.skip_fp64)
        out["smith_batched"] = run_smith_batch(dev, local)
    if not args.skip_serving and form_main == smf.SMF_FORM_INT8LIMB:
        out["serving"] = run_serving(dev, local, with_fp64=not args.skip_fp64)
    if not args.skip_batched and form_main == smf.SMF_FORM_INT8LIMB:
        out["batched"] = run_batched(dev, local, stream, flush, 20, 3, peak_tf, with_fp64=not args.skip_fp64)
    if not args.skip_cpu:
        out["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
        out["cpu_paper_design"] = cpu_paper_design(args.cpu_seconds)
    print(json.dumps(out), flush=True)


def run_base_convert(dev, local, stream, flush, steps, hbm_peak):
    """Conversion between RNS bases (Section 3.1) of the product's 4096 x 256
    residue matrix from its 23-prime basis to the next 23 primes below it."""
    import numpy as np
    import torch

    from paper_2605_19254_gb300 import inputs, smf

    ctx = smf.Context(local, smf.SMF_FORM_INT8LIMB)
    src = ctx.basis_create(A_BITS + 64 * B_WORDS - 1 + 12)
    dst = ctx.basis_create(A_BITS + 64 * B_WORDS - 1 + 12, min(src.primes))
    count = M_ * N_
    r = np.stack([inputs.uniform_int(7, f"cv{i}", (count,), 0, int(p) - 1) for i, p in enumerate(src.primes)])
    rin = torch.from_numpy(r.astype(np.int32)).to(dev)
    rout = torch.empty((len(dst.primes), count), dtype=torch.int32, device=dev)
    for _ in range(3):
        ctx.base_convert(src, dst, rin, rout, stream=stream)
    ctx.status_sync(stream)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for s0, s1 in evs:
        flush.fill_(1)
        s0.record(stream)
        ctx.base_convert(src, dst, rin, rout, stream=stream)
        s1.record(stream)
    torch.cuda.synchronize(dev)
    ctx.status_sync(stream)
    ms = statistics.mean(a.elapsed_time(b) for a, b in evs)
    nbytes = count * 4 * (len(src.primes) + len(dst.primes))
    out = {"workload": f"{count} entries (4096 x 256), {len(src.primes)} -> {len(dst.primes)} primes below 2^24",
           "ms": ms, "entries_per_s": count / (ms * 1e-3), "algorithmic_bytes": nbytes,
           "hbm_gbs": nbytes / (ms * 1e-3) / 1e9, "hbm_frac": nbytes / (ms * 1e-3) / 1e9 / hbm_peak if hbm_peak else None,
           "bound": "integer issue", "kernel": "convert_kernel<24>", "steps": steps}
    src.destroy()
    dst.destroy()
    ctx.destroy()
    return out


BATCH_COUNT, BATCH_R, BATCH_BWORDS = 512, 128, 8
BATCH_WORKLOAD = ("rns_matmul_grouped: 512 products A_i (n_i x n_i, n log-uniform in [32,1024], entries uniform "
                  "[-2^k,2^k], k alternating 7/20) x B_i (n_i x 128 signed 512-bit), one call")


def _digits(h):
    """Balanced base-2^8 digits covering |x| <= h (the top digit may reach 128)."""
    t, lower, scale = 1, 0, 1
    while 128 * scale + lower < h:
        lower += 127 * scale
        scale *= 256
        t += 1
    return t


def run_batched(dev, local, stream, flush, steps, warmup, peak_tf, with_fp64=True):
    """The batched workload through smf_rns_matmul_grouped (one launch per phase),
    against the same products one call at a time and the FP64-residue form."""
    import numpy as np
    import torch

    from paper_2605_19254_gb300 import inputs, smf

    batch = inputs.batched_workload(0, BATCH_COUNT, BATCH_R, BATCH_BWORDS)
    As, Bs, Cs, bits = [], [], [], []
    eff = 0
    for n, k, A, B in batch:
        Wc = (k + 64 * BATCH_BWORDS - 1 + int(np.ceil(np.log2(n))) + 2 + 63) // 64
        As.append(torch.from_numpy(A.view(np.int64)).to(dev))
        Bs.append(torch.from_numpy(B.view(np.int64)).to(dev))
        Cs.append(torch.zeros((n, BATCH_R, Wc), dtype=torch.int64, device=dev))
        bits.append(k)
        eff += 2 * n * n * BATCH_R
    del batch

    def timed(ctx, call, nsteps, nwarm, prof=False):
        for _ in range(nwarm):
            call(ctx)
        ctx.status_sync(stream)
        if prof:
            ctx.profile_enable(True)
            ctx.profile_read()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nsteps)]
        torch.cuda.synchronize(dev)
        for s0, s1 in evs:
            flush.fill_(1)  # untimed: evict L2 between steps
            s0.record(stream)
            call(ctx)
            s1.record(stream)
        torch.cuda.synchronize(dev)
        ctx.status_sync(stream)
        out = statistics.mean(a.elapsed_time(b) for a, b in evs)
        return out, (ctx.profile_read() if prof else None)

    ctx = smf.Context(local, smf.SMF_FORM_INT8LIMB)
    work = torch.empty(ctx.rns_matmul_grouped_workspace(As, Bs, Cs, a_bits=bits), dtype=torch.uint8, device=dev)

    def grouped(c):
        c.rns_matmul_grouped(As, Bs, Cs, a_bits=bits, workspace=work, stream=stream)

    ms, _ = timed(ctx, grouped, steps, warmup)
    _, prof = timed(ctx, grouped, max(3, min(steps, 10)), 1, prof=True)
    # the same batch as a plan: host work once, launches replayed as a CUDA
    # graph, digit counts and tile order chosen by the autotuner's measurements
    plan = ctx.group_plan(As, Bs, Cs, a_bits=bits, flags=smf.SMF_PLAN_AUTOTUNE, stream=stream)
    plan_info, plan_report = plan.info(), plan.report()
    ms_plan, _ = timed(ctx, lambda c: plan.launch(stream), steps, warmup)
    plan.destroy()
    # the same products one call at a time (a single product per launch sequence)
    wone = torch.empty(max(ctx.rns_matmul_workspace(a, b, c, a_bits=k) for a, b, c, k in zip(As, Bs, Cs, bits)),
                       dtype=torch.uint8, device=dev)

    def one_by_one(c):
        for a, b, cc, k in zip(As, Bs, Cs, bits):
            c.rns_matmul(a, b, cc, a_bits=k, workspace=wone, stream=stream)

    ms_loop, _ = timed(ctx, one_by_one, 3, 1)
    bas = ctx.basis_create(max(k + 64 * BATCH_BWORDS - 1 + int(np.ceil(np.log2(a.shape[0])))
                               for a, k in zip(As, bits)))
    primes = bas.primes
    bas.destroy()
    ctx.destroy()
    L = len(primes)
    h_small, h_big = min(primes) // 2, max(primes) // 2
    TB = _digits(h_big)
    flops = sum(2 * a.shape[0] * a.shape[0] * BATCH_R * L * TB *
                (_digits(1 << k) if (1 << k) <= h_small else _digits(h_big)) for a, k in zip(As, bits))
    gemm_ms = prof["residue_gemm"][1] / max(1, prof["residue_gemm"][0])
    per_kernel = {k: (v[1] / v[0] if v[0] else 0.0) for k, v in prof.items()}
    fp64 = None
    if with_fp64:
        fctx = smf.Context(local, smf.SMF_FORM_FP64)
        fwork = torch.empty(fctx.rns_matmul_grouped_workspace(As, Bs, Cs, a_bits=bits), dtype=torch.uint8, device=dev)

        def grouped_fp64(c):
            c.rns_matmul_grouped(As, Bs, Cs, a_bits=bits, workspace=fwork, stream=stream)

        ms_f, _ = timed(fctx, grouped_fp64, 2, 1)
        fctx.destroy()
        fp64 = {"value": eff / (ms_f * 1e-3) / 1e12, "unit": "TOPS", "ms_per_step": ms_f}
    return {
        "workload": BATCH_WORKLOAD, "metric": "effective exact integer-product TOPS (sum of 2 n_i^2 r per second)",
        "value": eff / (ms * 1e-3) / 1e12, "unit": "TOPS", "ms_per_step": ms, "steps": steps, "warmup": warmup,
        "products": len(As), "primes": L, "per_kernel_ms": per_kernel,
        "gpu_launches_per_step": 4,
        "roofline": {"bound": "tensor", "kernel": "limb_gemm_wide_kernel<grouped>",
                     "achieved": flops / (gemm_ms * 1e-3) / 1e12, "peak": peak_tf, "unit": "TFLOP/s",
                     "frac": flops / (gemm_ms * 1e-3) / 1e12 / peak_tf, "traffic": None,
                     "flops_per_launch": flops},
        "one_call_per_product": {"value": eff / (ms_loop * 1e-3) / 1e12, "unit": "TOPS", "ms_per_step": ms_loop},
        "graph_plan": {"value": eff / (ms_plan * 1e-3) / 1e12, "unit": "TOPS", "ms_per_step": ms_plan,
                       "padded_products": plan_info["padded"], "prefetched_products": plan_info["prefetched"],
                       "one_digit_kernel_products": plan_info["one_digit"],
                       "tile_order": plan_info["tile_order"],
                       "classes_tuned": plan_info["classes_tuned"], "tune_ms": plan_info["tune_ms"],
                       "autotune": plan_report.strip().splitlines()},
        "fp64_form": fp64,
    }


def run_lift(dev, local, n=1024, m=64, steps=16, reps=5):
    """p-adic lifting: `steps` steps of X_i = C R_i mod p, R_(i+1) = (R_i - A X_i)/p
    for a 20-bit A (n x n) and 40-bit B (n x m), limb form, one prime below 2^24."""
    import numpy as np
    import torch

    from paper_2605_19254_gb300 import inputs, smf

    ctx = smf.Context(local, smf.SMF_FORM_INT8LIMB)
    pb = ctx.basis_create(10)
    p = int(pb.primes[0])
    A = inputs.uniform_int(9, "LA", (n, n), -(1 << 20), 1 << 20)
    B = inputs.uniform_int(9, "LB", (n, m), -(1 << 40), 1 << 40)
    Ad = torch.from_numpy(A).to(dev)[..., None]
    # C = A^-1 mod p is an input of the call (the library's Gauss-Jordan over GF(p),
    # timed on its own here, outside the lifting's timed region)
    C = torch.empty((n, n), dtype=torch.int32, device=dev)
    inv_ws = torch.empty(ctx.inverse_mod_p_workspace(n), dtype=torch.uint8, device=dev)
    ctx.inverse_mod_p(pb, Ad, C, a_bits=20, workspace=inv_ws)
    ctx.status_sync()
    i0, i1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    i0.record()
    ctx.inverse_mod_p(pb, Ad, C, a_bits=20, workspace=inv_ws)
    i1.record()
    torch.cuda.synchronize(dev)
    ctx.status_sync()
    inv_ms = i0.elapsed_time(i1)
    Bd = torch.from_numpy(B).to(dev)[..., None]
    X = torch.empty((steps, n, m), dtype=torch.int32, device=dev)
    R = torch.empty((n, m, 1), dtype=torch.int64, device=dev)
    work = torch.empty(ctx.padic_lift_workspace(pb, Ad, Bd, a_bits=20, b_bits=40), dtype=torch.uint8, device=dev)
    for _ in range(2):
        ctx.padic_lift(pb, Ad, C, Bd, steps, X, R, a_bits=20, b_bits=40, workspace=work)
    ctx.status_sync()
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record()
    for _ in range(reps):
        ctx.padic_lift(pb, Ad, C, Bd, steps, X, R, a_bits=20, b_bits=40, workspace=work)
    s1.record()
    torch.cuda.synchronize(dev)
    ctx.status_sync()
    ms_step = s0.elapsed_time(s1) / reps / steps
    pb.destroy()
    ctx.destroy()
    return {"workload": f"A {n}x{n} (20-bit) x, B {n}x{m} (40-bit), {steps} steps, p = {p}",
            "ms_per_step": ms_step, "steps_per_s": 1e3 / ms_step, "inverse_mod_p_ms": inv_ms,
            "effective_tops": 4 * n * n * m / (ms_step * 1e-3) / 1e12,
            "note": "per step, 4 launches: C R mod p (residue product, one prime, K split); X_i and its digits "
                    "in the product basis; A X_i mod q_j (residue product, K split); A X_i by mixed radix, "
                    "(R - A X_i) / p and the digits of R mod p"}


# Phase 1 times the paper reports (Table 2, LIF column; Apple M4 Max, single run), seconds
PAPER_LIF_S = {1009: 2.424, 2003: 18.76, 5003: 168.6}


def run_lif(dev, local, sizes=(1009, 2003, 5003), m=32):
    """The largest invariant factor s_n (the paper's Phase 1) of its test
    matrices A_ij = i^j mod n: A^-1 mod p on the device, lifting of m random
    columns, host rational reconstruction.  One run per size, as the paper's
    breakdown is a single run; the library's own timers split the phases."""
    import torch

    from paper_2605_19254_gb300 import inputs, smf

    ctx = smf.Context(local, smf.SMF_FORM_INT8LIMB)
    out = []
    warm = torch.from_numpy(inputs.vandermonde_mod(53)[..., None].copy())
    ctx.largest_invariant_factor(warm, m=m, seed=1, a_bits=6)
    for n in sizes:
        A = torch.from_numpy(inputs.vandermonde_mod(n)[..., None].copy())
        bits = max(1, (n - 1).bit_length())
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        s, secs = ctx.largest_invariant_factor(A, m=m, seed=1, a_bits=bits)
        wall = time.perf_counter() - t0
        out.append({"n": n, "s_n_bits": s.bit_length(), "seconds": wall, "inverse_mod_p_s": secs[0],
                    "lifting_s": secs[1], "reconstruction_s": secs[2],
                    "paper_lif_s": PAPER_LIF_S.get(n)})
    ctx.destroy()
    return {"workload": f"largest invariant factor of A_ij = i^j mod n (the paper's test matrices), m = {m} random "
                        "right-hand sides, one prime below 2^24",
            "runs": out,
            "note": "paper_lif_s is the paper's Phase 1 time on an Apple M4 Max CPU: context, not a like-for-like "
                    "comparison; s_n at n = 1009 has 4083 bits in the paper"}


# Table 1 of the paper: Smith massager wall time on its test matrices A_ij = i^j mod n, Apple M4 Max CPU
PAPER_SMITH_S = {1009: 26.30, 2003: 134.4, 5003: 1744, 10007: 5399}


def run_smith(dev, local, with_fp64=True, with_large=True):
    """The Smith form (the paper's three phases) of its test matrices
    A_ij = i^j mod n at n = 1009, 2003, 5003, of the constructed n = 64
    workload U diag(s) V (both forms), and once of a dense random n = 10007
    matrix with entries in [-100, 100] (int32-sized).  One run each, timed
    on the host clock around the synchronous call; the library's own timers
    split the phases."""
    import math

    import numpy as np
    import torch

    from paper_2605_19254_gb300 import inputs, smf

    def one(ctx, A, bits, name, n):
        t = torch.from_numpy(np.ascontiguousarray(A)[..., None].copy())
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        s, secs, att = ctx.smith_form(t, seed=1, a_bits=bits)
        wall = time.perf_counter() - t0
        return {"matrix": name, "n": n, "seconds": wall, "phase1_s": secs[0], "phase2_s": secs[1],
                "phase3_s": secs[2], "attempts": att, "nontrivial_factors": sum(1 for v in s if v > 1),
                "factors_above_2^62": sum(1 for v in s if v.bit_length() > 62), "s_n_bits": s[-1].bit_length(),
                "log2_det": round(sum(math.log2(v) for v in s)),
                "paper_s": PAPER_SMITH_S.get(n) if name == "vandermonde_mod" else None}

    tail = [2, 6, 12, 60, 120, 840]
    A1 = np.array(inputs.smith_known_matrix(0, [1] * 58 + tail), dtype=np.int64)
    runs = {}
    for form, fname in ((smf.SMF_FORM_INT8LIMB, "limb"), (smf.SMF_FORM_FP64, "fp64")):
        if form == smf.SMF_FORM_FP64 and not with_fp64:
            continue
        ctx = smf.Context(local, form)
        ctx.smith_form(torch.from_numpy(inputs.vandermonde_mod(53)[..., None].copy()), seed=1, a_bits=6)  # warm-up
        out = [one(ctx, A1, int(np.abs(A1).max()).bit_length(), "constructed U diag(s) V", 64)]
        for n in (1009, 2003, 5003):
            if form == smf.SMF_FORM_FP64 and n > 2003:
                continue  # the FP64 form's lifting alone takes minutes here
            if n > 2003 and not with_large:
                continue
            out.append(one(ctx, inputs.vandermonde_mod(n), n.bit_length(), "vandermonde_mod", n))
        if form == smf.SMF_FORM_INT8LIMB and with_large:
            out.append(one(ctx, inputs.smith_dense_matrix(10007, 100, 0), 7, "dense random [-100, 100]", 10007))
        ctx.destroy()
        runs[fname] = out
    return {"workload": "Smith form: the paper's test matrices A_ij = i^j mod n (n = 1009, 2003, 5003), the "
                        "constructed n = 64 matrix U diag(s) V (s = 58 ones, 2, 6, 12, 60, 120, 840) and a dense "
                        "random n = 10007 matrix with entries uniform in [-100, 100]",
            "metric": "s/matrix", "runs": runs,
            "note": "paper_s is the paper's Table 1 time on an Apple M4 Max CPU (context only); its n = 10007 "
                    "matrix is its test matrix, not the random one timed here"}


def _percentile(xs, q):
    xs = sorted(xs)
    if not xs:
        return None
    i = min(len(xs) - 1, max(0, int(round(q / 100.0 * (len(xs) - 1)))))
    return xs[i]


def run_smith_serving(dev, local, workers=4, with_fp64=True):
    """Serving Smith-form requests (the Smith form as a request stream): a pool
    of jobs with n log-uniform in [64, 4096] and entries uniform in [-2^k, 2^k],
    k cycling 7 / 20 / 40, through smf_smith_server.  Capacity: every job
    submitted at once, drained.  Then Poisson arrivals at half the capacity rate.
    Latency is submit -> finish per job.  The FP64 form on the jobs with
    n <= 1024 (its lifting would take minutes on the larger ones), beside the
    limb form on the same jobs."""
    import numpy as np

    from paper_2605_19254_gb300 import inputs, smf

    ns = inputs.log_uniform_int(5, "serve_n", 12, 64, 4096)
    ks = (7, 20, 40)
    pool = []
    for i, n in enumerate(ns):
        k = ks[i % 3]
        pool.append((inputs.uniform_int(200 + i, "SS", (int(n), int(n)), -(1 << k), 1 << k), k + 1))

    def run(form, jobs, rate=None):
        srv = smf.SmithServer(local, form, 0, workers)
        rng = np.random.default_rng(7)
        t0 = time.perf_counter()
        ids = []
        for A, b in jobs:
            if rate:
                time.sleep(rng.exponential(1.0 / rate))
            ids.append(srv.submit(A, b, 1))
        srv.drain()
        wall = time.perf_counter() - t0
        lat = []
        for jid in ids:
            st, code, (ts, tb, te) = srv.job(jid)
            if st != smf.SMF_JOB_DONE:
                raise RuntimeError(f"smith job {jid} failed: {code}")
            lat.append(te - ts)
        srv.destroy()
        return {"jobs": len(jobs), "jobs_per_s": len(jobs) / wall, "wall_s": wall,
                "p50_s": _percentile(lat, 50), "p99_s": _percentile(lat, 99)}

    out = {"workload": "Smith-form requests: n log-uniform in [64, 4096] (12 jobs, seeded), entries uniform in "
                       "[-2^k, 2^k], k cycling 7/20/40; smf_smith_server with %d workers" % workers,
           "n": [int(v) for v in ns]}
    cap = run(smf.SMF_FORM_INT8LIMB, pool)
    out["capacity"] = cap
    out["poisson_0.5x"] = run(smf.SMF_FORM_INT8LIMB, pool, rate=0.5 * cap["jobs_per_s"])
    if with_fp64:
        small = [j for j in pool if j[0].shape[0] <= 1024]
        out["small_jobs"] = {"n": [int(j[0].shape[0]) for j in small],
                             "limb": run(smf.SMF_FORM_INT8LIMB, small), "fp64": run(smf.SMF_FORM_FP64, small)}
    return out


def run_smith_batch(dev, local, workers=8):
    """The batched Smith-form workload: 512 matrices, n log-uniform in [32, 1024];
    half uniform in [-2^k, 2^k] (k = 7 / 20), half built as U diag(s) V with a
    known s, every one through smf_smith_server (one Smith form per matrix,
    `workers` at a time).  The planted ones are checked against their s."""
    from paper_2605_19254_gb300 import inputs, smf

    batch = inputs.batched_smith_workload(0, 512)
    srv = smf.SmithServer(local, smf.SMF_FORM_INT8LIMB, 0, workers)
    t0 = time.perf_counter()
    ids = [srv.submit(A, b, 1) for _, b, A, _ in batch]
    srv.drain()
    wall = time.perf_counter() - t0
    failed = wrong = 0
    for jid, (n, _, _, s) in zip(ids, batch):
        st, code, _ = srv.job(jid)
        if st != smf.SMF_JOB_DONE:
            failed += 1
        elif s is not None and srv.result(jid, n) != s:
            wrong += 1
    srv.destroy()
    return {"workload": "512 Smith forms: n log-uniform in [32, 1024], half uniform in [-2^k, 2^k] (k = 7/20), "
                        "half U diag(s) V with known s; smf_smith_server, %d workers, limb form" % workers,
            "matrices_per_s": len(batch) / wall, "wall_s": wall, "planted_checked": len(batch) // 2,
            "failed": failed, "planted_wrong": wrong}


SERVE_R, SERVE_BWORDS = 64, 8
SERVE_WORKLOAD = ("serving: exact-product jobs A (n x n, n log-uniform in [64,2048], entries uniform [-2^k,2^k], "
                  "k cycling 7/20/40) x B (n x 64 signed 512-bit); Poisson arrivals")


def run_serving(dev, local, with_fp64=True):
    """The serving loop under load: capacity (jobs submitted at once), then Poisson
    arrivals at fractions of it, with each job's latency from submit to finish."""
    import numpy as np
    import torch

    from paper_2605_19254_gb300 import inputs, smf

    pool = []
    for i, n in enumerate(inputs.log_uniform_int(4, "serve_n", 64, 64, 2048)):
        n, k = int(n), (7, 20, 40)[i % 3]
        A, B = inputs.rns_matmul_workload(inputs.stream_seed(4, f"sj{i}"), n, n, SERVE_R, k, SERVE_BWORDS)
        Wc = (k + 64 * SERVE_BWORDS - 1 + int(np.ceil(np.log2(n))) + 2 + 63) // 64
        pool.append((n, k, torch.from_numpy(A.view(np.int64)).to(dev), torch.from_numpy(B.view(np.int64)).to(dev), Wc))

    def out(job):
        n, _, _, _, Wc = job
        return torch.empty((n, SERVE_R, Wc), dtype=torch.int64, device=dev)

    def ops(job):
        return 2 * job[0] * job[0] * SERVE_R

    def capacity(form):
        ctx = smf.Context(local, form)
        srv = smf.Server(ctx, 16 << 30, max_batch=64)
        outs = [out(j) for j in pool]
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for j, C in zip(pool, outs):
            srv.submit(j[2], j[3], C, a_bits=j[1])
        srv.drain()
        dt = time.perf_counter() - t0
        srv.destroy()
        ctx.destroy()
        return len(pool) / dt, sum(ops(j) for j in pool) / dt / 1e12

    capacity(smf.SMF_FORM_INT8LIMB)  # warm-up: bases, allocator pool
    cap_jobs, cap_tops = capacity(smf.SMF_FORM_INT8LIMB)
    res = {"workload": SERVE_WORKLOAD, "capacity_jobs_per_s": cap_jobs, "capacity_tops": cap_tops, "loads": []}
    ctx = smf.Context(local, smf.SMF_FORM_INT8LIMB)
    rng = np.random.default_rng(11)
    for frac in (0.5, 0.9):
        rate = frac * cap_jobs
        count = int(min(400, max(60, rate * 2.0)))
        arrivals = np.cumsum(rng.exponential(1.0 / rate, count))
        picks = rng.integers(0, len(pool), count)
        outs = [out(pool[p]) for p in picks]
        srv = smf.Server(ctx, 16 << 30, max_batch=64)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        ids, i, done, batches = [], 0, set(), 0
        while len(done) < count:
            now = time.perf_counter() - t0
            while i < count and arrivals[i] <= now:
                j = pool[picks[i]]
                ids.append(srv.submit(j[2], j[3], outs[i], a_bits=j[1]))
                i += 1
            batches += srv.step() > 0
            for jid in ids:
                if jid not in done and srv.job(jid)[0] in (smf.SMF_JOB_DONE, smf.SMF_JOB_FAILED):
                    done.add(jid)
        times = [srv.job(jid)[2] for jid in ids]
        assert all(srv.job(jid)[0] == smf.SMF_JOB_DONE for jid in ids)
        lat = np.array([t[2] - t[0] for t in times]) * 1e3
        span = max(t[2] for t in times) - min(t[0] for t in times)
        res["loads"].append({"offered_jobs_per_s": rate, "jobs": count, "achieved_jobs_per_s": count / span,
                             "achieved_tops": sum(ops(pool[p]) for p in picks) / span / 1e12,
                             "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                             "batches": int(batches)})
        srv.destroy()
    ctx.destroy()
    if with_fp64:
        f_jobs, f_tops = capacity(smf.SMF_FORM_FP64)
        res["fp64_form_capacity"] = {"jobs_per_s": f_jobs, "tops": f_tops}
    return res


def profile_run(rows: int, form: str, calls: int = 3):
    """Run the product with the first `rows` rows of A a few times and exit (a
    small, self-contained case for ncu captures; prints no benchmark line)."""
    import numpy as np
    import torch

    from paper_2605_19254_gb300 import build, inputs, smf

    build.build()
    A_np, B_np = inputs.rns_matmul_workload(0, rows, K_, N_, A_BITS, B_WORDS)
    A = torch.from_numpy(A_np.view(np.int64)).cuda()
    B = torch.from_numpy(B_np.view(np.int64)).cuda()
    C = torch.zeros((rows, N_, C_WORDS), dtype=torch.int64, device="cuda")
    ctx = smf.Context(0, smf.SMF_FORM_INT8LIMB if form == "limb" else smf.SMF_FORM_FP64)
    work = torch.empty(ctx.rns_matmul_workspace(A, B, C, a_bits=A_BITS), dtype=torch.uint8, device="cuda")
    for _ in range(calls):
        ctx.rns_matmul(A, B, C, a_bits=A_BITS, workspace=work)
    ctx.status_sync()
    ctx.destroy()
    print(f"profile run: {calls} x rns_matmul {rows}x{K_} @ {K_}x{N_} ({form})", flush=True)


def profile_batched(count: int, calls: int = 3, bits: int = 0):
    """Run the grouped product on the first `count` products of the batched
    workload (only those with `bits`-bit A when bits > 0) a few times and exit (a
    small case for ncu; prints no benchmark line)."""
    import numpy as np
    import torch

    from paper_2605_19254_gb300 import build, inputs, smf

    build.build()
    batch = inputs.batched_workload(0, BATCH_COUNT, BATCH_R, BATCH_BWORDS)[:count]
    if bits:
        batch = [b for b in batch if b[1] == bits]
    As = [torch.from_numpy(A.view(np.int64)).cuda() for _, _, A, _ in batch]
    Bs = [torch.from_numpy(B.view(np.int64)).cuda() for _, _, _, B in batch]
    Cs = [torch.zeros((n, BATCH_R, (k + 64 * BATCH_BWORDS - 1 + int(np.ceil(np.log2(n))) + 2 + 63) // 64),
                      dtype=torch.int64, device="cuda") for n, k, _, _ in batch]
    bits = [k for _, k, _, _ in batch]
    ctx = smf.Context(0, smf.SMF_FORM_INT8LIMB)
    work = torch.empty(ctx.rns_matmul_grouped_workspace(As, Bs, Cs, a_bits=bits), dtype=torch.uint8, device="cuda")
    for _ in range(calls):
        ctx.rns_matmul_grouped(As, Bs, Cs, a_bits=bits, workspace=work)
    ctx.status_sync()
    ctx.destroy()
    print(f"profile run: {calls} x rns_matmul_grouped over {len(batch)} products", flush=True)


def profile_convert(calls: int = 3):
    """Convert the 4096 x 256 residue matrix from 23 to 23 primes a few times
    and exit (a small case for ncu; prints no benchmark line)."""
    import numpy as np
    import torch

    from paper_2605_19254_gb300 import build, inputs, smf

    build.build()
    ctx = smf.Context(0, smf.SMF_FORM_INT8LIMB)
    src = ctx.basis_create(A_BITS + 64 * B_WORDS - 1 + 12)
    dst = ctx.basis_create(A_BITS + 64 * B_WORDS - 1 + 12, min(src.primes))
    r = np.stack([inputs.uniform_int(7, f"cv{i}", (M_ * N_,), 0, int(p) - 1) for i, p in enumerate(src.primes)])
    rin = torch.from_numpy(r.astype(np.int32)).cuda()
    rout = torch.empty((len(dst.primes), M_ * N_), dtype=torch.int32, device="cuda")
    for _ in range(calls):
        ctx.base_convert(src, dst, rin, rout)
    ctx.status_sync()
    src.destroy()
    dst.destroy()
    ctx.destroy()
    print(f"profile run: {calls} x base_convert of {M_ * N_} entries", flush=True)


def profile_lif(n: int, dense: bool = False):
    """The largest invariant factor of the paper's test matrix of dimension n
    (dense: a dense random matrix with entries in [-100, 100], as the n = 10007
    Smith-form workload), once, and exit (a case for ncu's launch list; prints
    no benchmark line)."""
    import numpy as np
    import torch

    from paper_2605_19254_gb300 import build, inputs, smf

    build.build()
    ctx = smf.Context(0, smf.SMF_FORM_INT8LIMB)
    if dense:
        A = torch.from_numpy(inputs.uniform_int(0, "dense", (n, n), -100, 100).astype(np.int64)[..., None].copy())
        bits = 7
    else:
        A = torch.from_numpy(inputs.vandermonde_mod(n)[..., None].copy())
        bits = max(1, (n - 1).bit_length())
    s, secs = ctx.largest_invariant_factor(A, m=32, seed=1, a_bits=bits)
    ctx.destroy()
    print(f"profile run: largest invariant factor, n = {n}: {s.bit_length()} bits, {secs[3]:.3f} s "
          f"(A^-1 mod p {secs[0]:.3f}, lifting {secs[1]:.3f}, reconstruction {secs[2]:.3f})", flush=True)


def profile_smith(n: int):
    """The Smith form of the paper's test matrix of dimension n, once after a small
    warm-up, and exit (for ncu's launch list; prints no benchmark line)."""
    import torch

    from paper_2605_19254_gb300 import build, inputs, smf

    build.build()
    ctx = smf.Context(0, smf.SMF_FORM_INT8LIMB)
    ctx.smith_form(torch.from_numpy(inputs.vandermonde_mod(23)[..., None].copy()), seed=1, a_bits=5)
    A = torch.from_numpy(inputs.vandermonde_mod(n)[..., None].copy())
    s, secs, attempts = ctx.smith_form(A, seed=1, a_bits=max(1, (n - 1).bit_length()))
    ctx.destroy()
    print(f"profile run: Smith form, n = {n}: {sum(1 for v in s if v > 1)} nontrivial factors, s_n of "
          f"{s[-1].bit_length()} bits, {secs[3]:.3f} s, {attempts} attempt(s)", flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--form", default="limb", choices=["limb", "fp64"])
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-batched", action="store_true", help="leave out the 512-product grouped workload")
    ap.add_argument("--skip-serving", action="store_true", help="leave out the serving loop under Poisson load")
    ap.add_argument("--skip-smith", action="store_true", help="leave out the Smith-form runs")
    ap.add_argument("--parallel", default="replicas", choices=["replicas", "split"],
                    help="with N > 1 GPUs: one product per rank, or one product split by rows over the ranks")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--profile-rows", type=int, default=0,
                    help="only run the product on the first ROWS rows of A three times (for ncu)")
    ap.add_argument("--profile-convert", action="store_true",
                    help="only run the base conversion of the 4096 x 256 residue matrix three times (for ncu)")
    ap.add_argument("--profile-batched", type=int, default=0,
                    help="only run the grouped product on the first COUNT batched products three times (for ncu)")
    ap.add_argument("--profile-batched-bits", type=int, default=0,
                    help="with --profile-batched: only the products whose A has this many bits (7 or 20)")
    ap.add_argument("--profile-lif-dense", action="store_true",
                    help="with --profile-lif: a dense random matrix with entries in [-100, 100]")
    ap.add_argument("--profile-lif", type=int, default=0,
                    help="only run the largest invariant factor of the N x N test matrix once (for ncu)")
    ap.add_argument("--profile-smith", type=int, default=0,
                    help="only run the Smith form of the N x N test matrix once (for ncu)")
    args = ap.parse_args()
    if args.profile_smith:
        profile_smith(args.profile_smith)
    elif args.profile_lif:
        profile_lif(args.profile_lif, dense=args.profile_lif_dense)
    elif args.profile_rows:
        profile_run(args.profile_rows, args.form)
    elif args.profile_batched:
        profile_batched(args.profile_batched, bits=args.profile_batched_bits)
    elif args.profile_convert:
        profile_convert()
    elif args.impl == "reference":
        run_reference(args)
    else:
        run(args)


if __name__ == "__main__":
    main()
