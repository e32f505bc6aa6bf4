#!/usr/bin/env python3
"""Benchmark: SCF-sequence solve time and effective TFLOP/s of the warm-started
generalized Hermitian eigensolver (libgevp) on synthetic FLAPW-shaped sequences.

One step = one call of the sequence solver over the whole workload (20 problems,
n = 2048, nev = 100, nex = 40, B fixed), inputs resident in HBM. Prints ONE JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gevp|reference]
                  [--workload scf_seq_n2048] [--prec fp64|bf16|fp32]

Under torchrun (N > 1) every rank solves its own replica of the sequence (a single
sequence is sequential in the SCF index, so there is nothing to shard: replicas only),
timing is the max over ranks and value is the whole-job aggregate.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SCF-sequence solve time & effective TFLOP/s at 1e-10 residual vs plain FP64"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gevp", choices=["gevp", "reference"])
    p.add_argument("--workload", default="scf_seq_n2048")
    p.add_argument("--prec", default="fp32", choices=["fp64", "bf16", "fp32"],
                   help="filter precision of the timed form (fp32: FP32-class tensor-core filter)")
    p.add_argument("--no-baseline", action="store_true", help="skip the CPU oracle baseline")
    p.add_argument("--no-compare", action="store_true", help="skip the plain FP64 cold-start comparison")
    p.add_argument("--no-e2e", action="store_true",
                   help="skip the host-buffer end-to-end measurement (large workloads: tens of GB pinned)")
    p.add_argument("--cpu-sample-s", type=float, default=20.0)
    p.add_argument("--gen-device", default="cuda", choices=["cuda", "cpu"],
                   help="where the synthetic inputs are generated (cpu for runs under ncu)")
    p.add_argument("--kpoints", type=int, default=64, help="kpoint_batch workload: number of k-points")
    p.add_argument("--seq-steps", type=int, default=10, help="kpoint_batch workload: problems per k-point")
    p.add_argument("--reduce-slices", type=int, default=8,
                   help="digits of the emulated FP64 products of the reduction (0: FP64 pipe)")
    p.add_argument("--kernel-case", choices=["zgemm", "tc", "reduce", "batched", "variation", "ozaki", "seq_small", "cholqr",
                            "update"],
                   default=None,
                   help="run only a few launches of one kernel (n 2048, m 140) for ncu captures")
    return p.parse_args()


def kernel_case(args):
    """A few launches of one kernel at the bench sizes, for ncu (no timing, no JSON)."""
    import torch
    from paper_1007_4400_gb300 import gevp, synth
    dev = torch.device("cuda", 0)
    if args.kernel_case == "variation":
        # entry-variation statistics of two n = 6144 matrices (1.2 GB, beyond L2), timed with
        # CUDA events. Algorithmic bytes: both matrices read once (32 n^2); the kernels also
        # write and re-read the squared moduli (16 n^2) and spend 5 FP64 operations per entry
        n = 6144
        g = torch.Generator(device=dev).manual_seed(11)
        A0 = torch.randn((n, n), dtype=torch.complex128, device=dev, generator=g)
        A1 = A0 + 1e-3 * torch.randn((n, n), dtype=torch.complex128, device=dev, generator=g)
        ps = [0.01, 0.1, 0.5]
        for _ in range(3):
            gevp.matrix_variation(A1, A0, ps)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 10
        e0.record()
        for _ in range(reps):
            d, c, _ = gevp.matrix_variation(A1, A0, ps)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        alg = 32.0 * n * n
        print(json.dumps({"kernel_case": "variation", "n": n, "ms": ms, "alg_bytes": alg,
                          "GBps": alg / (ms * 1e-3) / 1e9, "bytes_moved": 48.0 * n * n,
                          "fp64_ops": 5.0 * n * n, "delta": d, "counts": c}))
        return 0
    if args.kernel_case == "seq_small":
        # a short sequence (3 problems, n 1024, nev 64, nex 24, FP32-class filter) for
        # captures of the small dense kernels (Cholesky blocks, Jacobi, refinement)
        seq = synth.make_sequence(1, 1024, 3, 64, 24, device="cpu")
        r = gevp.solve_sequence([a.to(dev) for a in seq.A], seq.B.to(dev), 64, nex=24, filter_prec="fp32")
        torch.cuda.synchronize()
        print(f"kernel case seq_small done: status {r.status}, max residual {float(r.resid.max()):.2e}")
        return 0
    if args.kernel_case == "update":
        # the localised update of the standard form (64 of 2048 rows and columns changed,
        # 8 digits) against a full emulated reduction, timed with CUDA events; the factor of
        # B is reused by the update and part of the full reduction's call, so the factor-only
        # time (an update of one row with a fresh factorisation) is measured and subtracted
        import numpy as np
        n, k = 2048, 64
        seq = synth.make_sequence(1, n, 1, 100, 40, device=dev)
        rng = np.random.default_rng(7)
        J = np.sort(rng.choice(n, size=k, replace=False))
        D = torch.randn((n, n), dtype=torch.complex128, device=dev)
        D = 0.5 * (D + D.conj().T)
        mask = torch.zeros((n, n), dtype=torch.bool, device=dev)
        mask[torch.from_numpy(J).to(dev), :] = True
        mask[:, torch.from_numpy(J).to(dev)] = True
        dA = torch.where(mask, D, torch.zeros_like(D)) * 0.01
        _, C0 = gevp.reduce(seq.A[0], seq.B, slices=8)

        def timed(f, reps=5):
            for _ in range(2):
                f()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                f()
            e1.record()
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / reps
        ms_full = timed(lambda: gevp.reduce(seq.A[0], seq.B, slices=8))
        ms_factor = timed(lambda: gevp.reduce_update(C0.clone(), seq.B, dA, J[:1], slices=8))
        gevp.reduce_update(C0.clone(), seq.B, dA, J, slices=8)
        ms_upd = timed(lambda: gevp.reduce_update(C0.clone(), seq.B, dA, J, slices=8, reuse_factor=True))
        ms_upd64 = timed(lambda: gevp.reduce_update(C0.clone(), seq.B, dA, J, slices=0, reuse_factor=True))
        ms_copy = timed(lambda: C0.clone())
        print(json.dumps({"kernel_case": "update", "n": n, "k": k, "ms_full_reduction_with_factor": ms_full,
                          "ms_factor_only": ms_factor, "ms_full_reduction_products": ms_full - ms_factor,
                          "ms_update_emulated": ms_upd - ms_copy, "ms_update_fp64": ms_upd64 - ms_copy}))
        return 0
    if args.kernel_case == "cholqr":
        # the bench shape of the tall-skinny kernels: CholQR2 of a 2048 x 140 block with
        # columns scaled over three decades (Gram kernel, cluster Cholesky-inverse, product)
        # and one Rayleigh-Ritz projection on the result
        n, m = 2048, 140
        g = torch.Generator(device=dev).manual_seed(5)
        Y = torch.randn((n, m), dtype=torch.complex128, device=dev, generator=g)
        Y = Y * torch.logspace(0, 3, m, dtype=torch.float64, device=dev)[None, :]
        G = torch.randn((n, n), dtype=torch.complex128, device=dev, generator=g)
        C = (0.5 * (G + G.conj().T) * (25.0 / n ** 0.5)).contiguous()
        Q = gevp.cholqr2(Y)
        Q = gevp.cholqr2(Q)
        gevp.rayleigh_ritz(C, Q)
        torch.cuda.synchronize()
        print(f"kernel case cholqr done: n={n} m={m}")
        return 0
    if args.kernel_case == "ozaki":
        # the emulated FP64 product D = A B^H (n = 2048, 8 digits) and the reduction to
        # standard form with and without it, timed with CUDA events (inputs are 67 MB per
        # matrix; the digit planes, 200+ MB per operand, exceed L2)
        n = 2048
        g = torch.Generator(device=dev).manual_seed(13)
        A = torch.randn((n, n), dtype=torch.complex128, device=dev, generator=g)
        Bm = torch.randn((n, n), dtype=torch.complex128, device=dev, generator=g)
        H = 0.5 * (A + A.conj().T)
        P = torch.eye(n, dtype=torch.complex128, device=dev) * 2.0 + 0.01 * H
        def timed(f, reps=5):
            for _ in range(2):
                f()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                out = f()
            e1.record()
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / reps, out
        ms_oz, D = timed(lambda: gevp.zgemm_emulated(A, Bm, 8))
        ref = A @ Bm.conj().T
        err = float((D - ref).abs().max() / ref.abs().max())
        ms_red64, (L0, C0) = timed(lambda: gevp.reduce(H, P))
        ms_red_oz, (L1, C1) = timed(lambda: gevp.reduce(H, P, slices=8))
        cdiff = float((C1 - C0).abs().max() / C0.abs().max())
        pairs = 36
        print(json.dumps({"kernel_case": "ozaki", "n": n, "ms_zgemm_emulated": ms_oz,
                          "fp64_equiv_tflops": 8.0 * n ** 3 / (ms_oz * 1e-3) / 1e12,
                          "bf16_exec_tflops": pairs * 8.0 * n ** 3 / (ms_oz * 1e-3) / 1e12,
                          "max_err_vs_cublas_zgemm": err, "ms_reduce_fp64": ms_red64, "ms_reduce_emulated": ms_red_oz,
                          "reduce_rel_diff": cdiff}))
        return 0
    if args.kernel_case == "batched":
        # one step of a small k-point batch (inputs built on the host), FP32-class filter:
        # the grouped tcgen05 filter, grouped FP64 GEMMs and the batched small kernels
        seqs = synth.kpoint_batch(args.kpoints, 1, device="cpu")
        A = [[a.to(dev) for a in s.A] for s in seqs]
        B = [s.B.to(dev) for s in seqs]
        r = gevp.solve_batched(A, B, [s.nev for s in seqs], nex=[s.nex for s in seqs], filter_prec="fp32",
                               want_X=False)
        torch.cuda.synchronize()
        print(f"kernel case batched done: {len(seqs)} k-points, status {r.status}, rounds {r.stats['rounds']}")
        return 0
    kw = synth.WORKLOADS[args.workload]
    n, m = kw["n"], kw["nev"] + kw["nex"]
    # a random Hermitian matrix of the workload's size and scale (no factorisations, so the
    # filter cases launch no other GEMM before the profiled ones)
    g = torch.Generator(device=dev).manual_seed(7)
    G = torch.randn((n, n), dtype=torch.complex128, device=dev, generator=g)
    C = (0.5 * (G + G.conj().T) * (25.0 / n ** 0.5)).contiguous()
    Y = torch.randn((n, m), dtype=torch.complex128, device=dev, generator=g)
    if args.kernel_case == "zgemm":
        gevp.chebyshev_filter(C, Y, 3, 5.0, 80.0, -3.0, prec="fp64")
    elif args.kernel_case == "tc":
        gevp.chebyshev_filter(C, Y, 4, 5.0, 80.0, -3.0, prec="bf16")
    else:
        B = torch.eye(n, dtype=torch.complex128, device=dev) * 2.0 + 0.01 * C
        gevp.reduce(C, B)
    torch.cuda.synchronize()
    print(f"kernel case {args.kernel_case} done: n={n} m={m}")
    return 0


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        return summarize_clock_lines(self.lines)


def summarize_clock_lines(lines) -> dict:
    """Median SM clock, the maximum clock and the throttle reasons seen in nvidia-smi
    samples (csv, noheader, nounits, in ClockSampler.FIELDS order); malformed lines are
    skipped."""
    sm, smax, reasons = [], None, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for ln in lines:
        parts = [x.strip() for x in ln.split(",")]
        if len(parts) < 9:
            continue
        try:
            sm.append(float(parts[1]))
            smax = float(parts[2])
        except ValueError:
            continue
        for nm, v in zip(names, parts[5:9]):
            if v.lower() == "active":
                reasons.add(nm)
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
            "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- helpers
def measured_peaks() -> dict:
    """The measured peaks of this machine's GPUs (MEASURED_PEAKS.json), or {}."""
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float, world: int, device) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def seq_flops(stats) -> float:
    return sum(s["flops_fp64"] + s["flops_lowp"] for s in stats)


def nominal_flops_per_problem(n: int, m: int, nev: int, nprob: int) -> float:
    """Fixed work of one warm-started problem, independent of how many iterations a given
    implementation needs: the reduction (4 n^3), three filter rounds of degree 16 on the
    whole block (8 n^2 m each step), three Rayleigh-Ritz projections (8 n^2 m) with CholQR2
    (~40 n m^2), the back-transform and original-space check (20 n^2 nev), and the
    Cholesky of B amortised over the sequence. The headline value is this count divided by
    the measured time, so values of different implementations compare as time ratios."""
    rounds, deg = 3, 16
    return (4.0 * n ** 3 + rounds * (8.0 * n * n * m * deg + 8.0 * n * n * m + 40.0 * n * m * m)
            + 20.0 * n * n * nev + (4.0 / 3.0) * n ** 3 / max(nprob, 1))


# ----------------------------------------------------------------------------- rooflines
def _profile_traffic(name):
    """Per-launch DRAM traffic from a committed ncu summary (profiles/<name>.json), or None."""
    try:
        return json.load(open(os.path.join(ROOT, "profiles", name + ".json"))).get("traffic_bytes_per_launch")
    except (OSError, ValueError):
        return None


def _timed_class(gevp, cls, fn, reps):
    """Run fn() reps times with the live kernel timing on; that class's record."""
    import torch
    fn()
    torch.cuda.synchronize()
    gevp.kernel_timing(True)
    for _ in range(reps):
        fn()
    torch.cuda.synchronize()
    gevp.kernel_timing(False)
    return gevp.kernel_timing_read()[cls]


def roofline_entries(gevp, dev, live, ms_total, steps, sm_mhz):
    """Achieved fraction of the roofline for each product kernel of the step.

    live: per class, all launches of the timed region (CUDA events on the launching stream;
    the next problem's reduction runs concurrently on a side stream, so these include
    contention). isolated: one launch shape timed alone, the shape of the committed ncu
    capture whose DRAM traffic is quoted: the emulated product on the reduction's shape (the
    largest share of its time), the Gram kernel on the bench's Gram matrix, the FP64 GEMM on
    an FP64 filter step (its largest single shape; in the default step it runs the n m^2
    and m^3 products of the projections, CholQR and the small eigensolver).
    Peaks: FP64 from the unit count (152 SMs x 2 FMA/clk x 2 flop x the max SM clock); BF16
    the measured burst (isolated) and sustained (live) rates."""
    import torch
    mp = measured_peaks()
    fp64_peak = 152 * 2 * 2 * sm_mhz * 1e6 / 1e12
    bf16_burst = mp.get("bf16_tflops") or 1900.0
    bf16_sust = mp.get("bf16_tflops_sustained") or 1700.0
    per = {}

    def live_entry(cls, bound, flop_key, peak, peak_source, work):
        rec = live[cls]
        if rec["launches"] == 0:
            return None
        ach = rec[flop_key] / (max(rec["ms"], 1e-9) * 1e-3) / 1e12
        return {"bound": bound, "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "peak_source": peak_source, "work": work, "launches_per_step": rec["launches"] / max(1, steps),
                "ms_per_launch": rec["ms"] / rec["launches"], "share_of_step": rec["ms"] / max(1e-9, ms_total),
                "traffic": None, "traffic_note": "launch shapes vary within the step: see isolated"}

    per["oz_gemm_kernel"] = live_entry(
        "oz_gemm_kernel", "tensor", "exec_flop", bf16_sust, "BF16 sustained, of measured (MEASURED_PEAKS.json)",
        "executed BF16 flop of the digit-pair products (36 x the FP64-equivalent 8 flop per complex "
        "multiply-add over the K ranges processed)")
    per["zgemm_kernel"] = live_entry(
        "zgemm_kernel", "alu", "alg_flop", fp64_peak, "FP64 unit count x measured max SM clock",
        "8 flop per complex multiply-add over the K ranges processed (64-block granularity)")
    per["zgram_kernel"] = live_entry(
        "zgram_kernel", "alu", "alg_flop", fp64_peak, "FP64 unit count x measured max SM clock",
        "8 flop per complex multiply-add of the tiles formed (16 x 16 granularity; lower tiles of "
        "Hermitian results)")
    per = {k: v for k, v in per.items() if v is not None}

    g = torch.Generator(device=dev).manual_seed(13)
    # emulated product, reduction shape A B^H, 2048^3
    if "oz_gemm_kernel" in per:
        Ai = torch.randn((2048, 2048), dtype=torch.complex128, device=dev, generator=g)
        Bi = torch.randn((2048, 2048), dtype=torch.complex128, device=dev, generator=g)
        rec = _timed_class(gevp, "oz_gemm_kernel", lambda: gevp.zgemm_emulated(Ai, Bi, 8), 5)
        ms = rec["ms"] / max(1, rec["launches"])
        ach = rec["exec_flop"] / (rec["ms"] * 1e-3) / 1e12
        per["oz_gemm_kernel"]["isolated"] = {
            "shape": "A B^H, 2048 x 2048 x 2048 complex (the reduction's product shape)", "ms_per_launch": ms,
            "achieved": ach, "peak": bf16_burst, "frac": ach / bf16_burst, "peak_source": "BF16 burst, of measured",
            "traffic": _profile_traffic("oz_gemm_n2048"), "alg_bytes_per_launch": 3 * 16.0 * 2048 ** 2,
            "fp64_equiv_tflops": rec["alg_flop"] / (rec["ms"] * 1e-3) / 1e12}
        del Ai, Bi
    # Gram kernel, the bench's Gram matrix Y^H Y (n 2048, m 140): 8 n m (m + 1) / 2 flop
    if "zgram_kernel" in per:
        n, m = 2048, 140
        Y0 = torch.randn((n, m), dtype=torch.complex128, device=dev, generator=g)
        Y0 = Y0 * torch.logspace(0, 3, m, dtype=torch.float64, device=dev)[None, :]
        rec = _timed_class(gevp, "zgram_kernel", lambda: gevp.cholqr2(Y0.clone()), 5)
        ms = rec["ms"] / max(1, rec["launches"])
        ach = 8.0 * n * m * (m + 1) / 2 / (ms * 1e-3) / 1e12
        per["zgram_kernel"]["isolated"] = {
            "shape": "Gram matrix Y^H Y, n 2048, m 140 (lower triangle, 8 n m (m+1)/2 flop)", "ms_per_launch": ms,
            "achieved": ach, "peak": fp64_peak, "frac": ach / fp64_peak, "traffic": _profile_traffic("zgram_n2048_m140"),
            "alg_bytes_per_launch": 16.0 * n * m}
        del Y0
    # FP64 GEMM: one FP64 filter step C Y, n 2048 x m 140 (8 n^2 m flop), C read once
    if "zgemm_kernel" in per:
        Gm = torch.randn((2048, 2048), dtype=torch.complex128, device=dev, generator=g)
        Ci = (0.5 * (Gm + Gm.conj().T) * (25.0 / 2048 ** 0.5)).contiguous()
        Yi = torch.randn((2048, 140), dtype=torch.complex128, device=dev, generator=g)
        rec = _timed_class(gevp, "zgemm_kernel",
                           lambda: gevp.chebyshev_filter(Ci, Yi, 4, 5.0, 80.0, -3.0, prec="fp64"), 2)
        ms = rec["ms"] / max(1, rec["launches"])
        ach = rec["alg_flop"] / (rec["ms"] * 1e-3) / 1e12
        per["zgemm_kernel"]["isolated"] = {
            "shape": "FP64 filter step C.Y, n 2048 x m 140", "ms_per_launch": ms, "achieved": ach,
            "peak": fp64_peak, "frac": ach / fp64_peak, "traffic": _profile_traffic("zgemm_filter_n2048_m140"),
            "alg_bytes_per_launch": 16.0 * 2048 ** 2 + 48.0 * 2048 * 140}
        del Gm, Ci, Yi
    top = max(per, key=lambda k: per[k]["share_of_step"])
    out = dict(per[top])
    out["kernel"] = top
    out["per_kernel"] = per
    return out


# ----------------------------------------------------------------------------- CPU oracle baseline
def cpu_baseline(seq, n_solves_budget_s: float, flops_per_problem: float):
    """Time the FP64 CPU oracle (tridiagonal path, all host cores) on a bounded sample of the
    same workload (problem 1 of the sequence, then more while within budget), reported in
    the metric's unit with the same fixed work per problem as the GPU line, so the ratio
    of the two values is the per-problem time ratio. Above n = 2048 a full oracle solve
    takes many minutes, so the sample is the leading 2048 x 2048 sub-pencil of problem 1
    (value = the nominal work of an order-2048 problem / time). Also returns the oracle's
    solution of the first timed problem when it is a full one (for the accuracy block)."""
    import numpy as np
    import oracle
    full = seq.n <= 2048
    ns = seq.n if full else 2048
    B = seq.B.cpu().numpy()[:ns, :ns].copy()
    if not full:
        flops_per_problem = nominal_flops_per_problem(ns, seq.nev + seq.nex, seq.nev, len(seq.A))
    times = []
    first = None
    t_all = time.perf_counter()
    l = 1 if len(seq.A) > 1 else 0
    while True:
        A = seq.A[l].cpu().numpy()[:ns, :ns].copy()
        t0 = time.perf_counter()
        sol = oracle.solve(A, B, seq.nev, method="tridiag")
        times.append(time.perf_counter() - t0)
        if first is None and full:
            first = (l, sol)
        l += 1
        if l >= len(seq.A) or time.perf_counter() - t_all + times[-1] > n_solves_budget_s:
            break
    per = sum(times) / len(times)
    what = "problem(s)" if full else f"leading {ns}x{ns} sub-pencil(s) of problem(s)"
    return {"value": flops_per_problem / per / 1e12, "unit": "TFLOP/s", "cores": oracle.get_threads(),
            "kind": "oracle",
            "sample": f"{len(times)} {what} of the {seq.n}x{seq.n} sequence, oracle full FP64 solve "
                      f"(Cholesky, reduction, Householder tridiagonal + bisection + inverse iteration, "
                      f"back-transform), {per:.2f} s each; numerator = the fixed nominal work of a problem "
                      f"of order {ns}",
            "seconds_per_problem": per, "cpu": oracle.cpu_info()}, first


def accuracy_block(seq, lam_all, X_all, oracle_sol):
    """Error of every eigenvalue and eigenvector of sampled problems against a reference:
    problem 0 against its closed form (A = L Q diag(lam) Q^H L^H: eigenvalues lam, vectors
    L^-H Q e_i), problem l against the FP64 CPU oracle's solution when one was computed.
    Eigenvalue error: max_i |lam_i - lam_i*| / max_j |lam_j*| (full-spectrum scale of
    problem 0). Eigenvectors: per cluster of reference eigenvalues closer than 1e-8 of the
    scale, the largest principal-angle sine between the computed and the reference
    subspaces in the B inner product (the oracle's principal_sines on L_B^H X)."""
    import numpy as np
    import torch
    from oracle import pieces
    nev = seq.nev
    scale = float(np.abs(seq.lam0).max())
    B = seq.B.cpu().numpy()
    LbH = np.linalg.cholesky(B).conj().T
    refs = {}
    L = seq.L_true.cpu()
    X0 = torch.linalg.solve_triangular(L.conj().transpose(0, 1), seq.Q_true.cpu()[:, :nev], upper=True)
    refs[0] = (np.asarray(seq.lam0[:nev]), X0.numpy(), "closed form")
    if oracle_sol is not None:
        l, (lam_r, X_r) = oracle_sol
        refs[l] = (lam_r, X_r, "FP64 CPU oracle (tridiagonal path)")
    out = {"scale": scale, "tol": {"eig_rel": 1e-12, "resid": 1e-10}, "problems": {}}
    worst_e, worst_s = 0.0, 0.0
    for l, (lam_r, X_r, what) in sorted(refs.items()):
        lam_g = lam_all[l]
        X_g = X_all[l]
        e = float(np.abs(lam_g - lam_r).max() / scale)
        Xg_t, Xr_t = LbH @ X_g, LbH @ X_r
        smax, start = 0.0, 0
        for i in range(nev):
            if i == nev - 1 or lam_r[i + 1] - lam_r[i] > 1e-8 * scale:
                sines = pieces.principal_sines(Xg_t[:, start:i + 1], Xr_t[:, start:i + 1], None)
                smax = max(smax, float(np.max(sines)))
                start = i + 1
        out["problems"][str(l)] = {"reference": what, "eig_rel_err_max": e, "cluster_sine_max": smax}
        worst_e, worst_s = max(worst_e, e), max(worst_s, smax)
    out["eig_rel_err_max"] = worst_e
    out["cluster_sine_max"] = worst_s
    return out


# ----------------------------------------------------------------------------- reference arm
def run_reference(args):
    """The reference arm of this method: the FP64 CPU oracle as it stands (all host cores,
    tridiagonal path), each step a bounded sample of the workload so that the whole
    --steps K --warmup W run ends within a few minutes: the full oracle solve of the leading
    n/2 x n/2 sub-pencil of one problem of the sequence (a principal sub-pencil of a
    Hermitian-definite pencil is Hermitian-definite; same entry distributions; about 1/8 of
    the dense n^3 work). The value is the nominal work of a problem of that order divided by
    the measured time. The filter terms of the nominal count scale as n^2 m, the oracle's
    dense work as n^3, so the sample's rate is above the oracle's rate on full-size problems
    (by about 2x at n = 2048): the ratio against the GPU arm is understated, not inflated."""
    rank, world, _ = dist_info()
    if rank != 0:
        return 0
    from paper_1007_4400_gb300 import synth
    seq = synth.workload(args.workload, device="cpu")
    n, m = seq.n, seq.nev + seq.nex
    ns = max(seq.nev + 1, n // 2)
    flops_per_sample = nominal_flops_per_problem(ns, m, seq.nev, len(seq.A))
    import oracle
    B = seq.B.numpy()[:ns, :ns].copy()
    times = []
    for k in range(args.warmup + args.steps):
        A = seq.A[(1 + k) % len(seq.A)].numpy()[:ns, :ns].copy()
        t0 = time.perf_counter()
        oracle.solve(A, B, seq.nev, method="tridiag")
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
    per = statistics.mean(times)
    val = flops_per_sample / per / 1e12
    sample = (f"per step: the oracle's full FP64 solve (Cholesky, reduction, Householder tridiagonal + "
              f"bisection + inverse iteration, back-transform; lowest {seq.nev}) of the leading {ns}x{ns} "
              f"sub-pencil of one problem of the {n}x{n} sequence; value = nominal work of an order-{ns} "
              f"problem / time")
    cb = {"value": val, "unit": "TFLOP/s", "cores": oracle.get_threads(), "kind": "oracle", "sample": sample}
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": "TFLOP/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": args.workload, "n": n, "nev": seq.nev, "nex": seq.nex,
                      "sample": f"leading {ns}x{ns} sub-pencil of one problem per step"},
           "cpu_baseline": cb,
           "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


# ----------------------------------------------------------------------------- batched k-point arm
def bench_batched(args):
    """The batched form: nk k-points (n ~ U{800..3000}, nev = round(0.06 n)), each a warm
    sequence of seq_steps problems, all solved by one gevp_solve_batched call per step."""
    import torch
    from paper_1007_4400_gb300 import gevp, shard, synth
    rank, world, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    # k-points are independent: each rank solves a cost-balanced subset (no collective on
    # the data path; only the timings are reduced)
    sizes_all = synth.batched_sizes(args.kpoints)
    mine = shard.shard_kpoints(sizes_all, world)[rank]
    seqs = [synth.make_sequence(3, sizes_all[k][0], args.seq_steps, sizes_all[k][1], sizes_all[k][2], device=dev,
                                problem_index=k) for k in mine]
    A = [s.A for s in seqs]
    B = [s.B for s in seqs]
    nev = [s.nev for s in seqs]
    nex = [s.nex for s in seqs]
    nominal = sum(args.seq_steps * nominal_flops_per_problem(n, ne + nx, ne, args.seq_steps)
                  for n, ne, nx in sizes_all)

    def step(**kw):
        o = dict(filter_prec=args.prec)
        o.update(kw)
        return gevp.solve_batched(A, B, nev, nex=nex, want_X=False, **o)

    for _ in range(args.warmup):
        r = step()
    torch.cuda.synchronize()
    launches0 = gevp.kernel_launches(local)
    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    results = [step() for _ in range(args.steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    launches = (gevp.kernel_launches(local) - launches0) // max(1, args.steps)
    ms_step = max_over_ranks(e0.elapsed_time(e1) / args.steps, world, dev)
    r = results[-1]
    maxres = max_over_ranks(max(float(t.max()) for t in r.resid), world, dev)
    compare = None
    if not args.no_compare and world == 1:
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        rc = step(filter_prec="fp64", cold_start=1)
        c1.record(stream)
        torch.cuda.synchronize()
        ms_cold = c0.elapsed_time(c1)
        compare = {"batched_fp64_cold_ms": ms_cold, "speedup_vs_batched_fp64_cold": ms_cold / ms_step,
                   "batched_fp64_cold_resid_max": max(float(t.max()) for t in rc.resid),
                   "batched_fp64_cold_rounds": rc.stats["rounds"]}
    nprob = args.kpoints * args.seq_steps
    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return 0
    out = {"metric": METRIC, "value": nominal / (ms_step * 1e-3) / 1e12, "unit": "TFLOP/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": "f64" if args.prec == "fp64" else f"f64+{args.prec}", "data": "synthetic",
           "config": {"workload": "kpoint_batch", "kpoints": args.kpoints, "problems_per_kpoint": args.seq_steps,
                      "n_range": [min(x[0] for x in sizes_all), max(x[0] for x in sizes_all)],
                      "parallelism": f"k-points sharded over {world} GPU(s)" if world > 1 else "single GPU",
                      "nev": "round(0.06 n)", "nex": "ceil(0.4 nev)", "filter_prec": args.prec,
                      "start": "warm within each k-point", "l2": "inputs larger than L2"},
           "problems_per_s": nprob / (ms_step * 1e-3), "converged": all(x.status == 0 for x in results),
           "max_resid": maxres, "stats": r.stats, "clocks": clk, "gpu_launches": launches,
           "gpu_launches_note": "host-enqueued launches; graph replays are counted in stats.graph_replays",
           "compare": compare}
    print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


# ----------------------------------------------------------------------------- main arm
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.kernel_case:
        return kernel_case(args)
    if args.workload == "kpoint_batch":
        return bench_batched(args)
    import torch
    rank, world, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1007_4400_gb300 import gevp, synth

    seq = synth.workload(args.workload, device=args.gen_device)
    if args.gen_device != "cuda":
        seq.A = [a.to(dev) for a in seq.A]
        seq.B = seq.B.to(dev)
    nprob, n, nev, nex = len(seq.A), seq.n, seq.nev, seq.nex
    m = nev + nex
    opts = dict(nex=nex, filter_prec=args.prec, reduce_slices=args.reduce_slices)
    peaks = gevp.probe_peaks(local)

    def step(**kw):
        o = dict(opts)
        o.update(kw)
        return gevp.solve_sequence(seq.A, seq.B, nev, **o)

    for _ in range(args.warmup):
        r = step()
    torch.cuda.synchronize()
    launches0 = gevp.kernel_launches(local)
    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    # live timing of the GEMM kernels over the timed region (an event pair per launch on
    # its own stream: about 0.2 % of the step)
    gevp.kernel_timing(True)
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    results = []
    for _ in range(args.steps):
        results.append(step())
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    gevp.kernel_timing(False)
    live = gevp.kernel_timing_read()
    launches = (gevp.kernel_launches(local) - launches0) // max(1, args.steps)
    ms_total = e0.elapsed_time(e1)
    ms_step = max_over_ranks(ms_total / args.steps, world, dev)
    r = results[-1]
    ok = all(x.status == 0 for x in results) and float(r.resid.max()) <= 1e-10
    flops = seq_flops(r.stats)
    nominal = nprob * nominal_flops_per_problem(n, m, nev, nprob)
    value = world * nominal / (ms_step * 1e-3) / 1e12
    executed_tflops = world * flops / (ms_step * 1e-3) / 1e12

    # ---- per-kernel rooflines, from the live timing of the timed region; the top-level
    # entry is the kernel class with the largest device time
    sm_mhz = clk.get("sm_max_mhz") or 2070.0
    roofline = roofline_entries(gevp, dev, live, ms_total, args.steps, sm_mhz)

    # ---- plain FP64 cold-start GPU solver on the same sequence (the comparison form)
    compare = None
    if not args.no_compare and rank == 0:
        torch.cuda.synchronize()
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        rc = step(cold_start=1, filter_prec="fp64", reduce_slices=0)
        c1.record(stream)
        torch.cuda.synchronize()
        ms_cold = c0.elapsed_time(c1)
        compare = {"plain_fp64_cold_ms": ms_cold, "speedup_vs_plain_fp64_cold": ms_cold / ms_step,
                   "plain_fp64_cold_resid_max": float(rc.resid.max()),
                   "plain_fp64_cold_matvecs": sum(s["matvecs"] for s in rc.stats)}

    # ---- end to end through the C ABI with host buffers (copies inside the timed region)
    e2e = None
    if rank == 0 and not args.no_e2e:
        hostA = [a.cpu().pin_memory() for a in seq.A]
        hostB = seq.B.cpu().pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(max(1, args.steps)):
            rr = gevp.solve_sequence_host(hostA, hostB, nev, device=local, **opts)
        dt = (time.perf_counter() - t0) / max(1, args.steps)
        h2d = (nprob + 1) * n * n * 16
        d2h = rr.Lambda.numel() * 8 + rr.resid.numel() * 8 + rr.X.numel() * 16
        e2e = {"value": nominal / dt / 1e12, "unit": "TFLOP/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "ms_per_step": dt * 1e3, "converged": rr.status == 0,
               "path": "gevp_solve_sequence_host: pinned host A_l, B -> device staging -> solve -> Lambda, resid, X "
                       "to host, all inside the call"}

    cb, osol = None, None
    if rank == 0 and world == 1 and not args.no_baseline:
        cb, osol = cpu_baseline(seq, args.cpu_sample_s, nominal / nprob)

    # ---- accuracy of sampled problems (untimed solve keeping every problem's eigenvectors)
    accuracy = None
    if rank == 0:
        ra = step(keep_all_X=1)
        torch.cuda.synchronize()
        lam_all = ra.Lambda.cpu().numpy()
        X_all = ra.X.cpu().numpy().reshape(nprob, n, nev)
        accuracy = accuracy_block(seq, lam_all, X_all, osol)
        accuracy["resid_max_all_problems"] = float(ra.resid.max())
        del ra, X_all

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f64" if args.prec == "fp64" else f"f64+{args.prec}",
               "data": "synthetic",
               "config": {"workload": args.workload, "n": n, "problems": nprob, "nev": nev, "nex": nex,
                          "B": "fixed", "start": "warm (previous problem's block)", "filter_prec": args.prec,
                          "parallelism": "replicas" if world > 1 else "single GPU",
                          "l2": f"inputs larger than L2 ({nprob} x {n * n * 16 / 2 ** 20:.0f} MiB matrices per step)"},
               "sequence_ms": ms_step, "problems_per_s": world * nprob / (ms_step * 1e-3),
               "value_definition": "nominal TFLOP/s: fixed work per problem (nominal_flops_per_problem) x problems / "
                                   "sequence time",
               "executed_tflops": executed_tflops,
               "converged": ok, "max_resid": float(r.resid.max()),
               "outer_iters": [s["outer_iters"] for s in r.stats],
               "phase_ms": {k: round(sum(s[k] for s in r.stats), 3) for k in
                            ("ms_chol", "ms_reduce", "ms_bounds", "ms_filter", "ms_orth", "ms_rr", "ms_final")},
               "roofline": roofline, "peaks_measured": peaks, "clocks": clk, "gpu_launches": launches,
               "e2e": e2e, "cpu_baseline": cb, "compare": compare, "accuracy": accuracy}
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
