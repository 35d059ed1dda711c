"""Benchmark: emulated FP64 GEMM on the INT8 tensor cores of one GB300.

Workload (one "step"): Scheme I emulated DGEMM C = A @ B, M = N = K = 8192,
row-major float64, A and B drawn by the paper's test-matrix generator
(Eq. 19) with phi = 0.5, p = 8 INT8 slices: exponent scan, split into
interleaved slices, fused INT8 GEMM with the exact shift-reduce epilogue.
Inputs (512 MiB each) are larger than L2 (129 MB), so no L2 flush is needed.

Printed: one JSON line with the effective FP64 TFLOP/s (2 M N K / t), the
INT8 tensor rate and its fraction of the measured INT8 peak, the roofline
of the fused GEMM kernel, an end-to-end number through host buffers, cuBLAS
DGEMM on the same GPU at its own accuracy, the error of both against a
double-double reference on sampled entries, the CPU oracle baseline, and the
SM clocks seen during the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
For N > 1 run under torch.distributed.run: every rank computes its own
independent product (weak scaling, no collective on the data path).
"""
from __future__ import annotations

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

import synth  # noqa: E402

METRIC = "emulated FP64 TFLOP/s (Scheme I DGEMM on INT8 tensor cores)"
UNIT = "TFLOP/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=8192)
    ap.add_argument("--p", type=int, default=8)
    ap.add_argument("--phi", type=float, default=0.5)
    ap.add_argument("--scheme", default="I", choices=["I", "I_F8", "II"],
                    help="I: INT8 slices; I_F8: E4M3 slices on the FP8 tensor path; II: CRT (p = moduli)")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--cpu-rows", type=int, default=96, help="rows of C in the CPU oracle sample")
    ap.add_argument("--no-extras", action="store_true", help="skip cuBLAS / accuracy / CPU legs")
    ap.add_argument("--suite", default=None, help="write the secondary measurements (all paths) to this JSONL file")
    ap.add_argument("--suite-md", default=None, nargs="+",
                    help="print the summary tables of --suite JSONL files (rows of later files replace the "
                         "matching rows of earlier ones)")
    ap.add_argument("--grouped-run", action="store_true",
                    help="run the 512-product grouped batch (p = --p) --warmup + --steps times with the handle's "
                         "default configuration (no tuning) and print its time; for profiling launch lists")
    ap.add_argument("--selector-md", default=None,
                    help="print the selector end-to-end summary of a --suite-part selector JSONL file")
    ap.add_argument("--suite-part", default="all", choices=["all", "ii", "scheme2", "selector", "grouped"],
                    help="ii: only the Scheme II DGEMM points (run in a child with EMU_II_ENGINE=mma by the full "
                         "suite); scheme2: every row of the bf16 tcgen05 Scheme II paths (DGEMM, SGEMM, norm "
                         "scaling, ZGEMM 3M, CGEMM 3M); selector: the selector's end-to-end points; grouped: the "
                         "grouped-batch points")
    return ap.parse_args()


SCHEME_NAME = {"I": "Scheme I", "I_F8": "Scheme I on E4M3 slices", "II": "Scheme II"}


def ops_per_mnk(scheme, p):
    """Tensor ops per M*N*K of one product: the triangle p(p+1) or 2 N_m."""
    return 2 * p if scheme == "II" else p * (p + 1)


def config(args, world):
    return {"workload": "%s emulated DGEMM M=N=K=%d phi=%g %s=%d (Eq. 19 generator, seed %d)"
                        % (SCHEME_NAME[args.scheme], args.n, args.phi, "N" if args.scheme == "II" else "p", args.p,
                           args.seed),
            "m": args.n, "n": args.n, "k": args.n, "p": args.p, "phi": args.phi, "layout": "row-major",
            "scheme": args.scheme, "l2": "inputs larger than L2 (2 x %d MiB), no flush" % (8 * args.n * args.n >> 20),
            "parallelism": "replicas" if world == 1 else "dp%d independent products" % world}


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
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
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ helpers
def file_sha(paths):
    h = hashlib.sha256()
    for path in paths:
        with open(path, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def load_traffic(name, key):
    """DRAM bytes per launch of a fused GEMM kernel from the committed ncu
    summary profiles/<name>_traffic.json, only if the kernel sources are
    unchanged since the capture."""
    path = os.path.join(ROOT, "profiles", name + "_traffic.json")
    if not os.path.exists(path):
        return None
    try:
        d = json.load(open(path))
        srcs = [os.path.join(ROOT, "paper_2606_25453_gb300", "csrc", f) for f in d["sources"]]
        if d.get("source_sha256") != file_sha(srcs):
            return None
        return d.get("per_launch", {}).get(key)
    except Exception:
        return None


def max_over_ranks(x: float, dist, device) -> float:
    """Largest value of x over all ranks (x itself without a process group)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_tflops(world: int, flops_per_rank_step: float, steps: int, ms_max: float) -> float:
    """Whole-job throughput: all ranks' work divided by the slowest rank's time."""
    return world * flops_per_rank_step * steps / (ms_max * 1e-3) / 1e12


def fp8_engine_leg(emu, h, Ad, Bd, Cd, n, stream, ri, ci, A, B, hi, lo, den, cublas_tflops):
    """Scheme I on E4M3 slices (p = 11 and 12) on the same inputs: TFLOP/s,
    GEMM-kernel 8-bit TOP/s and sampled error, with the same CUDA-event timing."""
    import torch
    out = {}
    for p in (11, 12):
        def call():
            emu.check(emu.emu_dgemm(h.h, emu.EMU_ROW_MAJOR, n, n, n, 1.0, Ad.data_ptr(), n, Bd.data_ptr(), n, 0.0,
                                    Cd.data_ptr(), n, emu.EMU_SCHEME_I_F8, p, stream.cuda_stream), "emu_dgemm")
        for _ in range(3):
            call()
        torch.cuda.synchronize()
        h.trace(True)
        h.trace_read()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(5):
            call()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 5
        tr = h.trace_read()
        h.trace(False)
        got = Cd[ri][:, ci].cpu().numpy()
        err = float(np.max(np.abs((got - hi) - lo) / den))
        gms = tr["ms_gemm"] / max(tr["gemm_launches"], 1)
        f8_tops = p * (p + 1) * n ** 3 / (gms * 1e-3) / 1e12
        bf16 = measured_peaks().get("bf16_tflops") or 1900.0
        bf16s = measured_peaks().get("bf16_tflops_sustained")
        out["p%d" % p] = {"tflops": 2.0 * n ** 3 / (ms * 1e-3) / 1e12, "ms_per_step": ms,
                          "gemm_8bit_tops": f8_tops, "gemm_ms": gms,
                          "frac_of_fp8_peak": f8_tops / (2.0 * bf16),
                          "fp8_peak_tflops": 2.0 * bf16,
                          "frac_of_fp8_peak_sustained": (f8_tops / (2.0 * bf16s)) if bf16s else None,
                          "algorithmic_bytes": p * 2 * n * n + 8 * n * n,
                          "dram_traffic_bytes": load_traffic("gemm_f8tc", "p%d_n%d" % (p, n)),
                          "err_max_rel_absAB": err, "speedup_vs_cublas_dgemm": 2.0 * n ** 3 / (ms * 1e-3) / 1e12 / cublas_tflops,
                          "bits_per_slice": 5, "kernel": "gemm_f8tc_kernel<%d, OUT_F64> (tcgen05)" % p}
    return out


def scheme_II_leg(emu, h, Ad, Bd, Cd, n, stream, ri, ci, hi, lo, den, cublas_tflops):
    """Scheme II (16 and 20 moduli) on the same inputs with the default engine
    (bf16 tcgen05): TFLOP/s, residue-GEMM bf16 TFLOP/s against the measured
    bf16 peak (alone and with the CRT kernel's time), and sampled error, with
    the same CUDA-event timing."""
    import torch
    out = {}
    bf16 = measured_peaks().get("bf16_tflops") or 1900.0
    bf16s = measured_peaks().get("bf16_tflops_sustained")
    for nm in (16, 20):
        def call():
            emu.check(emu.emu_dgemm(h.h, emu.EMU_ROW_MAJOR, n, n, n, 1.0, Ad.data_ptr(), n, Bd.data_ptr(), n, 0.0,
                                    Cd.data_ptr(), n, emu.EMU_SCHEME_II, nm, stream.cuda_stream), "emu_dgemm")
        for _ in range(3):
            call()
        torch.cuda.synchronize()
        h.trace(True)
        h.trace_read()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(5):
            call()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 5
        tr = h.trace_read()
        h.trace(False)
        got = Cd[ri][:, ci].cpu().numpy()
        err = float(np.max(np.abs((got - hi) - lo) / den))
        gms = tr["ms_gemm"] / max(tr["gemm_launches"], 1)
        cms = tr["ms_other"] / max(tr["gemm_launches"], 1)
        tc = 2.0 * nm * n ** 3 / (gms * 1e-3) / 1e12
        out["nm%d" % nm] = {"tflops": 2.0 * n ** 3 / (ms * 1e-3) / 1e12, "ms_per_step": ms, "gemm_ms": gms,
                            "crt_ms": cms, "gemm_bf16_tflops": tc, "frac_of_bf16_peak": tc / bf16,
                            "frac_of_bf16_peak_with_crt": 2.0 * nm * n ** 3 / ((gms + cms) * 1e-3) / 1e12 / bf16,
                            "frac_of_bf16_peak_sustained": (tc / bf16s) if bf16s else None,
                            "bf16_peak_tflops": bf16,
                            "err_max_rel_absAB": err,
                            "speedup_vs_cublas_dgemm": 2.0 * n ** 3 / (ms * 1e-3) / 1e12 / cublas_tflops,
                            "kernel": "gemm_II_tc_kernel (tcgen05 bf16, 128 x 256 tiles)"}
    return out


def probe_ref(emu, h, Ad, Bd, ri, ci, stream=None):
    """Double-double reference of the sampled entries C[ri][:, ci] of A @ B and
    sum_h |a_ih||b_hj| for each, from the library's probe kernel (emu_probe_dd:
    error-free FP64 transformations on the GPU, checked against the CPU
    oracle's double-double product in the tests).  A, B: row-major float64
    CUDA tensors.  Returns (hi, lo, den) as numpy arrays of shape (len(ri), len(ci))."""
    import torch
    m, k = Ad.shape
    n = Bd.shape[1]
    pairs = np.array([[i, j] for i in ri for j in ci], dtype=np.int32).reshape(-1)
    cnt = len(ri) * len(ci)
    idx = torch.from_numpy(pairs).to(Ad.device)
    ref = torch.empty(2 * cnt, dtype=torch.float64, device=Ad.device)
    ab = torch.empty(cnt, dtype=torch.float64, device=Ad.device)
    st = None if stream is None else stream.cuda_stream
    emu.check(emu.emu_probe_dd(h.h, emu.EMU_ROW_MAJOR, m, n, k, Ad.data_ptr(), max(Ad.stride(0), 1), Bd.data_ptr(),
                               max(Bd.stride(0), 1), cnt, idx.data_ptr(), ref.data_ptr(), ab.data_ptr(), st),
              "emu_probe_dd")
    torch.cuda.synchronize()
    r = ref.cpu().numpy().reshape(cnt, 2)
    shp = (len(ri), len(ci))
    return r[:, 0].reshape(shp), r[:, 1].reshape(shp), ab.cpu().numpy().reshape(shp)


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(path))
    except Exception:
        return {}


def oracle_cpu_sample(args, A, B, rows):
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    oracle.emu_I(A[rows], B, args.p)
    dt = time.perf_counter() - t0
    return dt, oracle.num_threads()


# ------------------------------------------------------------------ reference arm
def run_reference(args, rank, world):
    """The CPU oracle as it stands, on a bounded sample of the workload per step."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    A, B = synth.gemm_pair(args.n, args.n, args.n, args.phi, args.seed)
    rows = list(range(max(1, args.cpu_rows // 4)))
    for _ in range(args.warmup):
        oracle.emu_I(A[rows[:1]], B, args.p)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.emu_I(A[rows], B, args.p)
        times.append(time.perf_counter() - t0)
    t = sum(times) / len(times)
    v = 2.0 * len(rows) * args.n * args.n / t / 1e12
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config(args, world),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": "%d rows of C (all %d columns, K = %d) per step" % (len(rows), args.n, args.n)},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm
def run_ours(args, rank, world, local_rank):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2606_25453_gb300 as emu

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    n, p = args.n, args.p
    A, B = synth.gemm_pair(n, n, n, args.phi, args.seed + 17 * rank)
    Ad = torch.from_numpy(A).to(dev)
    Bd = torch.from_numpy(B).to(dev)
    Cd = torch.empty((n, n), dtype=torch.float64, device=dev)
    h = emu.Handle(local_rank)
    stream = torch.cuda.current_stream(dev)
    scheme_code = {"I": emu.EMU_SCHEME_I, "I_F8": emu.EMU_SCHEME_I_F8, "II": emu.EMU_SCHEME_II}[args.scheme]

    def step():
        emu.check(emu.emu_dgemm(h.h, emu.EMU_ROW_MAJOR, n, n, n, 1.0, Ad.data_ptr(), n, Bd.data_ptr(), n, 0.0,
                                Cd.data_ptr(), n, scheme_code, p, stream.cuda_stream), "emu_dgemm")

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    if h.status() != 0:
        raise RuntimeError("device status %d after warm-up" % h.status())

    # ---------------- timed region: inputs resident in HBM
    h.trace(True)
    h.trace_read()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    tr = h.trace_read()
    h.trace(False)
    ms = max_over_ranks(ms, dist, dev)
    ms_step = ms / args.steps
    flops = 2.0 * n * n * n
    value = aggregate_tflops(world, flops, args.steps, ms)
    int8_ops = float(ops_per_mnk(args.scheme, p)) * n * n * n
    status = h.status()

    # ---------------- end to end through host buffers (pinned), copies timed
    A_pin = torch.from_numpy(A).pin_memory()
    B_pin = torch.from_numpy(B).pin_memory()
    C_pin = torch.empty((n, n), dtype=torch.float64).pin_memory()
    e2 = torch.cuda.Event(enable_timing=True)
    e3 = torch.cuda.Event(enable_timing=True)

    def e2e_step():
        # the public host-buffer entry point: it copies A and B in, computes
        # (Scheme I in row chunks whose copies overlap the GEMM) and returns
        # once C is back in C_pin
        emu.check(emu.emu_dgemm_host(h.h, emu.EMU_ROW_MAJOR, n, n, n, 1.0, A_pin.data_ptr(), n, B_pin.data_ptr(), n,
                                     0.0, C_pin.data_ptr(), n, scheme_code, p, stream.cuda_stream), "emu_dgemm_host")

    # untimed warm-up: the first transfers from freshly pinned buffers pay a
    # one-time mapping cost (tens of ms per step when spread over the steps)
    e2e_step()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e2.record(stream)
    for _ in range(args.steps):
        e2e_step()
    e3.record(stream)
    torch.cuda.synchronize()
    ms_e2e = max_over_ranks(e2.elapsed_time(e3), dist, dev)
    e2e_value = aggregate_tflops(world, flops, args.steps, ms_e2e)
    # the host-buffer result is the device result, bit for bit (sampled)
    if not torch.equal(C_pin[::997, ::991], Cd[::997, ::991].cpu()):
        raise RuntimeError("emu_dgemm_host result differs from emu_dgemm")

    extras = {}
    int8_peak = None
    if rank == 0 and not args.no_extras:
        # measured dense INT8 peak on this GPU: cuBLASLt INT8 GEMM 8192^3 (best of 5)
        a8 = torch.randint(-128, 127, (8192, 8192), dtype=torch.int8, device=dev)
        b8 = torch.randint(-128, 127, (8192, 8192), dtype=torch.int8, device=dev).t().contiguous().t()
        torch._int_mm(a8, b8)
        best = 1e30
        for _ in range(5):
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            torch._int_mm(a8, b8)
            s1.record(stream)
            torch.cuda.synchronize()
            best = min(best, s0.elapsed_time(s1))
        int8_peak = 2.0 * 8192 ** 3 / (best * 1e-3) / 1e12
        del a8, b8
        # cuBLAS DGEMM (native FP64) on the same inputs
        ref = Ad @ Bd
        torch.cuda.synchronize()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for _ in range(2):
            ref = Ad @ Bd
        s1.record(stream)
        torch.cuda.synchronize()
        cublas_tflops = 2 * flops / (s0.elapsed_time(s1) * 1e-3) / 1e12
        # accuracy on sampled entries against the double-double reference
        # (the library's GPU probe kernel)
        rng = np.random.Generator(np.random.PCG64(1234))
        ri = np.sort(rng.choice(n, 8, replace=False))
        ci = np.sort(rng.choice(n, 64, replace=False))
        hi, lo, den = probe_ref(emu, h, Ad, Bd, ri, ci, stream)
        ours_s = Cd[ri][:, ci].cpu().numpy()
        cub_s = ref[ri][:, ci].cpu().numpy()
        err_ours = float(np.max(np.abs((ours_s - hi) - lo) / den))
        err_cub = float(np.max(np.abs((cub_s - hi) - lo) / den))
        extras = {"cublas_dgemm_tflops": cublas_tflops, "speedup_vs_cublas_dgemm": value / world / cublas_tflops,
                  "err_max_rel_absAB": err_ours, "err_cublas_dgemm": err_cub,
                  "err_bound_4k_u": 4 * n * 2.0 ** -53, "err_sample": "8 x 64 entries vs double-double"}
        if args.scheme == "I":
            # the same product on the FP8 tensor path (Scheme I with E4M3 slices,
            # tcgen05 kernel) at FP64-level accuracy, timed the same way
            extras["fp8_tcgen05_engine"] = fp8_engine_leg(emu, h, Ad, Bd, Cd, n, stream, ri, ci, A, B, hi, lo, den,
                                                          cublas_tflops)
            extras["scheme_II_tcgen05_engine"] = scheme_II_leg(emu, h, Ad, Bd, Cd, n, stream, ri, ci, hi, lo, den,
                                                               cublas_tflops)
        del ref
        # CPU oracle baseline on a bounded sample of rows
        rows = list(range(args.cpu_rows))
        dt, cores = oracle_cpu_sample(args, A, B, rows)
        extras["cpu_baseline"] = {"value": 2.0 * len(rows) * n * n / dt / 1e12, "unit": UNIT, "cores": cores,
                                  "kind": "oracle",
                                  "sample": "%d rows of C (all %d columns, K = %d), %.1f s" % (len(rows), n, n, dt)}

    if rank == 0:
        gemm_ms = tr["ms_gemm"] / max(tr["gemm_launches"], 1)
        achieved = int8_ops / (gemm_ms * 1e-3) / 1e12
        peak, peak_src = int8_peak, "measured live: cuBLASLt INT8 GEMM 8192^3 on this GPU"
        ii_tc = args.scheme == "II" and os.environ.get("EMU_II_ENGINE") != "mma"
        if ii_tc:
            bf16 = measured_peaks().get("bf16_tflops")
            peak = bf16 if bf16 else 1900.0
            peak_src = ("measured dense bf16 peak (MEASURED_PEAKS.json)" if bf16 else
                        "fallback dense bf16 peak 1.9 PFLOP/s")
        if args.scheme == "I_F8":
            bf16 = measured_peaks().get("bf16_tflops")
            peak = 2.0 * bf16 if bf16 else 2.0 * 1900.0
            peak_src = ("FP8 dense peak = measured bf16 %s x nominal FP8/bf16 ratio 2 (4.5 / 2.25 PFLOP/s)"
                        % ("(MEASURED_PEAKS.json)" if bf16 else "(fallback 1.9 PFLOP/s)"))
        traffic = (load_traffic("gemm_I", "p%d_n%d" % (p, n)) if args.scheme == "I" else
                   load_traffic("gemm_f8tc", "p%d_n%d" % (p, n)) if args.scheme == "I_F8" else
                   load_traffic("gemm_II_tc", "nm%d_n%d" % (p, n)) if ii_tc else None)
        kname = ("gemm_II_tc_kernel (tcgen05 bf16 residue GEMM; the CRT kernel is timed apart)" if ii_tc else "gemm_II_kernel (mma.sync INT8)" if args.scheme == "II" else
                 "gemm_f8tc_kernel<%d, OUT_F64> (tcgen05)" % p if args.scheme == "I_F8" else
                 "gemm_I_kernel<%d, OUT_F64> (mma.sync INT8)" % p)
        ops_desc = ("bf16 tensor ops 2 N_m M N K (residue products)" if ii_tc else
                    "INT8 ops 2 N_m M N K" if args.scheme == "II" else
                    "exact E4M3 products p(p+1) M N K (multiply+add = 2)" if args.scheme == "I_F8" else
                    "INT8 ops p(p+1) M N K (multiply+add = 2)")
        metric = METRIC if args.scheme == "I" else (
            "emulated FP64 TFLOP/s (Scheme II DGEMM on %s tensor cores)" % ("bf16" if ii_tc else "INT8")
            if args.scheme == "II" else "emulated FP64 TFLOP/s (Scheme I DGEMM on E4M3 tensor cores)")
        line = {"metric": metric, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": max(args.warmup, 3), "ms_per_step": ms_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": ("e4m3->fp32 (f64 in/out)" if args.scheme == "I_F8" else
                          "bf16->fp32 (f64 in/out)" if ii_tc else "int8->int32 (f64 in/out)"),
                "data": "synthetic",
                "config": config(args, world),
                "int8_tops": (int8_ops * args.steps * world / (ms * 1e-3) / 1e12) if not ii_tc else None,
                "int8_frac_of_peak": ((int8_ops * args.steps / (ms * 1e-3) / 1e12 / int8_peak)
                                      if int8_peak and args.scheme != "I_F8" and not ii_tc else None),
                "roofline": {"bound": "tensor",
                             "kernel": kname,
                             "achieved": achieved,
                             "peak": peak, "unit": UNIT, "frac": (achieved / peak) if peak else None,
                             "traffic": traffic,
                             "ops": ops_desc,
                             "peak_source": peak_src},
                "phase_ms_per_step": {k2: tr[k2] / args.steps for k2 in ("ms_scan", "ms_split", "ms_gemm")},
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 2 * 8 * n * n,
                        "d2h_bytes_per_step": 8 * n * n},
                "gpu_launches": tr["kernel_launches"],
                "clocks": clk.summary(),
                "device_status": status,
                "measured_peaks_file": {k2: measured_peaks().get(k2) for k2 in ("hbm_gbs", "bf16_tflops")}}
        if "cpu_baseline" in extras:
            line["cpu_baseline"] = extras.pop("cpu_baseline")
        line.update(extras)
        print(json.dumps(line), flush=True)
    h.close()
    if dist:
        dist.destroy_process_group()


# ------------------------------------------------------------------ suite
def suite_key(d):
    """What a suite row measures (path and parameters), without its results."""
    return tuple((f, d.get(f)) for f in ("path", "scheme", "n", "phi", "p", "nm", "p_or_nm", "count"))


def suite_markdown(paths):
    """The summary tables of --suite JSONL files (the text of
    profiles/bench_suite_gb300.md); a row of a later file replaces the row
    of an earlier file that measures the same path and parameters."""
    import math
    if isinstance(paths, str):
        paths = [paths]
    merged = {}
    for path in paths:
        for line in open(path):
            d = json.loads(line)
            merged[suite_key(d)] = d
    rows = list(merged.values())

    def bits(e):
        return "-" if e is None else ("inf" if e == 0 else f"{-math.log2(e):.1f}")

    o = []
    o.append("# Measurement suite on one GB300 (all paths)\n")
    o.append("Command: `python bench.py --suite suite.jsonl`, then `python bench.py --suite-md suite.jsonl"
             + "".join(" " + os.path.basename(x) for x in paths[1:]))
    bf16 = measured_peaks().get("bf16_tflops") or 1900.0
    o.append("> profiles/bench_suite_gb300.md` (device-resident inputs, CUDA events,")
    o.append("1 warm-up + 3 timed calls per point, 1 at n = 16384 and for ZGEMM; accuracy = -log2 of")
    o.append("max |C - C_ref| / (|A||B|) on 8 x 64 sampled entries against the library's double-double probe")
    o.append("kernel, emu_probe_dd).")
    o.append("Slice-product rates count executed products x 2: Scheme I p(p+1)MNK (8-bit), Scheme II 2 N_m MNK and 3M")
    o.append("6 N_m MNK (residue products; bf16 on the default tcgen05 engine, INT8 on the mma.sync engine).")
    o.append("Measured INT8 peak of this GPU: 150-156 TOP/s (cuBLASLt INT8 GEMM; register-only mma.sync s8 loop")
    o.append("150.9).  bf16 peak: %.1f TFLOP/s (MEASURED_PEAKS.json); FP8 tensor peak: %.0f TFLOP/s (that x 2, the"
             % (bf16, 2 * bf16))
    o.append("nominal FP8/bf16 ratio).\n")
    for extra in paths[1:]:
        o.append(f"Rows of `{os.path.basename(extra)}` replace the rows of earlier files that measure the same path and")
        o.append("parameters.\n")
    o.append("## Native cuBLAS on the same GPU\n")
    o.append("| routine | n | TFLOP/s | bits |\n|---|---|---|---|")
    for d in rows:
        if d["path"].startswith("cublas"):
            t = d.get("tflops", d.get("tflops_8mnk"))
            unit = " (8MNK)" if "tflops_8mnk" in d else ""
            o.append(f"| {d['path']} | {d['n']} | {t:.3f}{unit} | {bits(d.get('err'))} |")
    o.append("\n## Scheme I emulated DGEMM / SGEMM, INT8 slices (mma.sync)\n")
    o.append("| path | n | phi | p | TFLOP/s | INT8 TOP/s | bits |\n|---|---|---|---|---|---|---|")
    for d in rows:
        if d["path"] in ("emu_dgemm_I", "emu_sgemm_I"):
            o.append(f"| {d['path']} | {d['n']} | {d['phi']:g} | {d['p']} | {d['tflops']:.3f} | {d['int8_tops']:.1f} | {bits(d['err'])} |")
    o.append("\n## Scheme I emulated DGEMM, E4M3 slices (tcgen05, TMEM accumulators)\n")
    o.append("| n | phi | p | TFLOP/s | FP8 TOP/s | x cuBLAS DGEMM | bits |\n|---|---|---|---|---|---|---|")
    cub = {d["n"]: d["tflops"] for d in rows if d["path"] == "cublas_dgemm"}
    for d in rows:
        if d["path"] == "emu_dgemm_I_F8":
            c = cub.get(d["n"], cub.get(8192))
            o.append(f"| {d['n']} | {d['phi']:g} | {d['p']} | {d['tflops']:.2f} | {d['f8_tops']:.0f} | {d['tflops']/c:.1f} | {bits(d['err'])} |")
    o.append("\n## Scheme II emulated DGEMM, bf16 tcgen05 engine (default; residue GEMM, then the CRT kernel)\n")
    o.append("| n | phi | N_m | TFLOP/s | tensor TOP/s | bits |\n|---|---|---|---|---|---|")
    for d in rows:
        if d["path"] == "emu_dgemm_II":
            o.append(f"| {d['n']} | {d['phi']:g} | {d['nm']} | {d['tflops']:.3f} | {d['tensor_tops']:.1f} | {bits(d['err'])} |")
    o.append("\n## SGEMM through Scheme II (bf16 tcgen05), n = 8192, phi = 0.5\n")
    csg = {d["n"]: d for d in rows if d["path"] == "cublas_sgemm"}
    o.append("| N_m | TFLOP/s | bits | x cuBLAS SGEMM (" + (f"{csg[8192]['tflops']:.1f} TFLOP/s, {bits(csg[8192].get('err'))} bits" if 8192 in csg else "-") + ") |\n|---|---|---|---|")
    for d in rows:
        if d["path"] == "emu_sgemm_II":
            o.append(f"| {d['nm']} | {d['tflops']:.2f} | {bits(d['err'])} | {d['tflops'] / csg[8192]['tflops']:.2f}x |" if 8192 in csg else f"| {d['nm']} | {d['tflops']:.2f} | {bits(d['err'])} | - |")
    o.append("\n## Scheme II on the INT8 mma.sync engine (EMU_II_ENGINE=mma), same inputs\n")
    o.append("| n | phi | N_m | TFLOP/s | INT8 TOP/s | bits | bf16 tcgen05 speedup |\n|---|---|---|---|---|---|---|")
    tc = {(d["n"], d["phi"], d["nm"]): d["ms"] for d in rows if d["path"] == "emu_dgemm_II"}
    for d in rows:
        if d["path"] == "emu_dgemm_II_int8":
            key = (d["n"], d["phi"], d["nm"])
            sp = d["ms"] / tc[key] if key in tc else float("nan")
            o.append(f"| {d['n']} | {d['phi']:g} | {d['nm']} | {d['tflops']:.3f} | {d['tensor_tops']:.1f} | {bits(d['err'])} | {sp:.2f}x |")
    o.append("\n## Scheme II with norm-based scaling (EMU_SCHEME_II_NORM)\n")
    o.append("| n | phi | N_m | TFLOP/s | tensor TOP/s | bits | bits, worst-case scaling |\n|---|---|---|---|---|---|---|")
    worst = {(d["n"], d["phi"], d["nm"]): d["err"] for d in rows if d["path"] == "emu_dgemm_II"}
    for d in rows:
        if d["path"] == "emu_dgemm_II_norm":
            w = worst.get((d["n"], d["phi"], d["nm"]))
            o.append(f"| {d['n']} | {d['phi']:g} | {d['nm']} | {d['tflops']:.3f} | {d['tensor_tops']:.1f} | {bits(d['err'])} | {bits(w) if w is not None else '-'} |")
    o.append("\n## Complex: ZGEMM (3M Scheme II, 4M Scheme I) and CGEMM, n = 8192, phi = 1\n")
    o.append("| path | scheme | p / N_m | TFLOP/s (8MNK) | bits |\n|---|---|---|---|---|")
    for d in rows:
        if d["path"] == "emu_zgemm_3m":
            o.append(f"| emu_zgemm | II (3M) | {d['nm']} | {d['tflops_8mnk']:.2f} | {bits(d['err'])} |")
        if d["path"] == "emu_zgemm_4m":
            o.append(f"| emu_zgemm | {d['scheme']} (4M) | {d['p']} | {d['tflops_8mnk']:.2f} | {bits(d['err'])} |")
        if d["path"] == "emu_cgemm":
            o.append(f"| emu_cgemm | {d['scheme']} ({'3M' if d['scheme']=='II' else '4M'}) | {d['p_or_nm']} | {d['tflops_8mnk']:.2f} | {bits(d['err'])} |")
    o.append("\n## Naive (INT32 partials to HBM + separate shift-reduce) vs fused, n = 4096, k <= K_c\n")
    o.append("`emu_partials_I` / `emu_partials_F8` + `emu_shift_reduce_I` against `emu_dgemm` (results")
    o.append("bit-identical).\n")
    o.append("| slices | p | naive ms | fused ms | fused speedup | INT32 partials bytes |\n|---|---|---|---|---|---|")
    for d in rows:
        if d["path"] == "ablation_naive_vs_fused":
            o.append(f"| {'E4M3 (tcgen05)' if d['slices'] == 'e4m3' else 'INT8 (mma.sync)'} | {d['p']} | {d['ms_naive']:.2f} | "
                     f"{d['ms_fused']:.2f} | {d['speedup_fused']:.2f} | {d['int32_partials_bytes']} |")
    # Fig. 7 analogue: precision, throughput and workspace of every real DGEMM
    # path at n = 8192, phi = 0.5 (workspace from the library's size query,
    # default engines)
    try:
        import ctypes

        import paper_2606_25453_gb300 as emu

        def ws_gb(scheme, p):
            sz = ctypes.c_size_t()
            emu.check(emu.emu_workspace_size(scheme, 8192, 8192, 8192, p, 0, ctypes.byref(sz)), "workspace")
            return sz.value / 2 ** 30
        pts = []
        for d in rows:
            if d.get("n") != 8192 or d.get("phi") != 0.5:
                continue
            if d["path"] == "emu_dgemm_I":
                pts.append(("Scheme I, INT8 (mma.sync)", "p = %d" % d["p"], d, ws_gb(emu.EMU_SCHEME_I, d["p"])))
            elif d["path"] == "emu_dgemm_I_F8":
                pts.append(("Scheme I, E4M3 (tcgen05)", "p = %d" % d["p"], d, ws_gb(emu.EMU_SCHEME_I_F8, d["p"])))
            elif d["path"] == "emu_dgemm_II":
                pts.append(("Scheme II (bf16 tcgen05)", "N = %d" % d["nm"], d, ws_gb(emu.EMU_SCHEME_II, d["nm"])))
        if pts:
            o.append("\n## Precision, throughput and workspace (n = 8192, phi = 0.5; the paper's Fig. 7 trade-off)\n")
            o.append("| path | slices / moduli | bits | TFLOP/s | workspace GiB |\n|---|---|---|---|---|")
            for name, par, d, gb in sorted(pts, key=lambda x: (-math.inf if x[2]["err"] == 0 else
                                                                  -math.log2(x[2]["err"]))):
                o.append(f"| {name} | {par} | {bits(d['err'])} | {d['tflops']:.2f} | {gb:.2f} |")
    except ImportError:
        pass
    o.append("\n## Grouped: 512 uneven products, one CUDA graph vs per-product loop\n")
    for d in rows:
        if d["path"] == "emu_dgemm_grouped":
            o.append(f"p = {d['p']}: graph (tuned) {d['ms_graph_tuned']:.2f} ms, untuned (64 x 32, B-slice-major) "
                     f"{d['ms_graph_default_tile']:.2f} ms, loop {d['ms_loop']:.2f} ms: "
                     f"{d['speedup_graph_vs_loop']:.2f}x; {d['tflops_graph']:.2f} emulated TFLOP/s, "
                     f"{d['int8_tops_graph']:.1f} INT8 TOP/s.")
            if d.get("tuned"):
                hist = {}
                for v in d["tuned"].values():
                    hist[v] = hist.get(v, 0) + 1
                o.append(f"  Tuned: {d.get('stages')} stage(s); shape buckets per configuration (tile, slice-pair "
                         "order): " + ", ".join(f"{v} {c}" for v, c in sorted(hist.items(), key=lambda x: -x[1])) +
                         ".")
    return "\n".join(o)


GROUPED_CFGS = ("64x32 B-major", "32x32 B-major", "32x64 B-major",
                "64x32 A-major", "32x32 A-major", "32x64 A-major")


def grouped_points(emu, h, dev, emit, timed):
    """512 uneven products (M, N log-uniform in [32, 1024], K in [64, 2048]):
    the grouped CUDA graph untuned and after the autotuner, against the
    per-product loop, at p = 6 and p = 10."""
    import tempfile

    import torch
    shapes = synth.grouped_shapes(512, 0)
    As, Bs, Cs = [], [], []
    for i, (m, nn, k) in enumerate(shapes):
        A, B = synth.gemm_pair(m, nn, k, 1.0, 5000 + i)
        As.append(torch.from_numpy(A).to(dev))
        Bs.append(torch.from_numpy(B).to(dev))
        Cs.append(torch.empty((m, nn), dtype=torch.float64, device=dev))
    d = emu.grouped_descs(As, Bs, Cs)
    flops = sum(2 * m * nn * k for m, nn, k in shapes)
    for p in (6, 10):
        ms_default = timed(lambda: emu.dgemm_grouped(d, p, handle=h), reps=5)
        with tempfile.TemporaryDirectory() as td:
            path = os.path.join(td, "tune.json")
            ncfg = emu.tune_grouped(d, p, path=path, handle=h)
            with open(path) as fh:
                tuned = json.load(fh)
        ms_tuned = timed(lambda: emu.dgemm_grouped(d, p, handle=h), reps=5)
        ms_loop = timed(lambda: emu.dgemm_grouped(d, p, handle=h, loop=True), reps=2)
        emit({"path": "emu_dgemm_grouped", "count": 512, "p": p, "ms_graph_default_tile": ms_default,
              "ms_graph_tuned": ms_tuned, "configs_timed": ncfg, "ms_loop": ms_loop,
              "tuned": {k: GROUPED_CFGS[v] for k, v in sorted(tuned.items())
                        if k.startswith("p%d_s" % p) and not k.endswith("_stages")},
              "stages": tuned.get("p%d_stages" % p),
              "tflops_graph": flops / ms_tuned / 1e9, "tflops_loop": flops / ms_loop / 1e9,
              "int8_tops_graph": (p * (p + 1) // 2) * flops / ms_tuned / 1e9,
              "speedup_graph_vs_loop": ms_loop / ms_tuned})


def grouped_run(args):
    """The 512-product grouped batch (the grouped_points shapes) at p = args.p,
    untuned: args.warmup + args.steps graph launches, CUDA-event time of the
    timed ones."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2606_25453_gb300 as emu
    dev = torch.device("cuda", 0)
    shapes = synth.grouped_shapes(512, 0)
    As, Bs, Cs = [], [], []
    for i, (m, nn, k) in enumerate(shapes):
        A, B = synth.gemm_pair(m, nn, k, 1.0, 5000 + i)
        As.append(torch.from_numpy(A).to(dev))
        Bs.append(torch.from_numpy(B).to(dev))
        Cs.append(torch.empty((m, nn), dtype=torch.float64, device=dev))
    h = emu.Handle(0)
    d = emu.grouped_descs(As, Bs, Cs)
    for _ in range(args.warmup):
        emu.dgemm_grouped(d, args.p, handle=h)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        emu.dgemm_grouped(d, args.p, handle=h)
    e1.record()
    torch.cuda.synchronize()
    if h.status() != 0:
        raise RuntimeError("device status %d" % h.status())
    ms = e0.elapsed_time(e1) / max(args.steps, 1)
    flops = sum(2 * m * nn * k for m, nn, k in shapes)
    print(json.dumps({"path": "emu_dgemm_grouped", "count": 512, "p": args.p, "ms": ms,
                      "tflops": flops / ms / 1e9, "int8_tops": args.p * (args.p + 1) // 2 * flops / ms / 1e9}))
    h.close()


SEL_TOLS = (1e-8, 1e-12, 1e-15)


def selector_products(count=12, seed=4242):
    """Held-out products for the selector's end-to-end timing: square, n
    log-uniform in [1024, 4096] (rounded to a multiple of 64), phi ~ U(0, 8)
    (the selector's training range), seeds disjoint from its training data."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(count):
        n = int(round(float(np.exp(rng.uniform(np.log(1024), np.log(4096)))) / 64)) * 64
        out.append((n, float(rng.uniform(0.0, 8.0)), 7_000_000 + 2 * i))
    return out


def selector_points(emu, h, dev, emit, products=None, schemes=(("I", 12), ("II", 20)),
                    tols=SEL_TOLS):
    """emu_dgemm_auto / emu_dgemm_auto_II (committed selector weights; feature
    scan, MLP, probe and every escalation inside the timed region) against
    emu_dgemm at the fixed p (N) that passes every training product -- p = 12
    for Scheme I, N = 20 for Scheme II with norm scaling -- on the same
    products, CUDA-event time on the stream, one timed call each after a
    warm-up at the largest size (both outputs preallocated outside the
    timing).  Pass = max |C - AB| / (|A||B|) <= tol on 256
    sampled entries against the GPU double-double probe."""
    import torch
    from paper_2606_25453_gb300 import selector as sel
    sel.install_default(h)
    products = products or selector_products()
    rng = np.random.Generator(np.random.PCG64(77))
    stream = torch.cuda.current_stream(dev)
    nmax = max(n for n, _, _ in products)
    Aw = synth.test_matrix_torch(nmax, nmax, 1.0, 1, dev)
    for sc, fixed in schemes:  # workspace at the largest size, and first-call costs, outside the timing
        emu.dgemm(Aw, Aw, scheme="I" if sc == "I" else "II_NORM", p=fixed, handle=h)
        emu.dgemm_auto(Aw, Aw, 1e-8, handle=h, scheme=sc)
    del Aw
    torch.cuda.synchronize()
    rows = []
    for n, phi, seed in products:
        Ad = synth.test_matrix_torch(n, n, phi, seed, dev)
        Bd = synth.test_matrix_torch(n, n, phi, seed + 1, dev)
        Cf = torch.empty((n, n), dtype=torch.float64, device=dev)
        Ca = torch.empty((n, n), dtype=torch.float64, device=dev)
        ri = np.sort(rng.choice(n, 16, replace=False))
        ci = np.sort(rng.choice(n, 16, replace=False))
        hi, lo, den = probe_ref(emu, h, Ad, Bd, ri, ci)

        def err(C):
            return float(np.max(np.abs((C[ri][:, ci].cpu().numpy() - hi) - lo) / den))

        for sc, fixed in schemes:
            fixed_scheme = "I" if sc == "I" else "II_NORM"
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            emu.dgemm(Ad, Bd, Cf, scheme=fixed_scheme, p=fixed, handle=h)
            e1.record(stream)
            torch.cuda.synchronize()
            ms_fixed = e0.elapsed_time(e1)
            err_fixed = err(Cf)
            for tol in tols:
                e0.record(stream)
                C, used, code = emu.dgemm_auto(Ad, Bd, tol, handle=h, scheme=sc, C=Ca)
                e1.record(stream)
                torch.cuda.synchronize()
                ms_auto = e0.elapsed_time(e1)
                d = {"path": "selector_e2e", "scheme": sc, "n": n, "phi": phi, "tol": tol, "fixed": fixed,
                     "used": used, "code": code, "ms_auto": ms_auto, "ms_fixed": ms_fixed,
                     "err_auto": err(C), "err_fixed": err_fixed}
                d["pass_auto"] = d["err_auto"] <= tol
                d["pass_fixed"] = err_fixed <= tol
                rows.append(d)
                emit(d)
        del Ad, Bd, Cf, Ca
    for sc, fixed in schemes:
        for tol in tols:
            r = [d for d in rows if d["scheme"] == sc and d["tol"] == tol]
            ta, tf = sum(d["ms_auto"] for d in r), sum(d["ms_fixed"] for d in r)
            emit({"path": "selector_e2e_summary", "scheme": sc, "tol": tol, "products": len(r), "fixed": fixed,
                  "ms_auto_total": ta, "ms_fixed_total": tf, "speedup_vs_fixed": tf / ta,
                  "pass_auto": float(np.mean([d["pass_auto"] for d in r])),
                  "pass_fixed": float(np.mean([d["pass_fixed"] for d in r])),
                  "mean_used": float(np.mean([d["used"] for d in r]))})
    return rows


def selector_markdown(path):
    """The text of profiles/selector_e2e_gb300.md from a --suite-part selector file."""
    rows = [json.loads(x) for x in open(path)]
    pts = [d for d in rows if d.get("path") == "selector_e2e"]
    summ = [d for d in rows if d.get("path") == "selector_e2e_summary"]
    o = ["# Learned selector, end to end, on one GB300\n",
         "Command: `python bench.py --suite selector.jsonl --suite-part selector`, then",
         "`python bench.py --selector-md selector.jsonl > profiles/selector_e2e_gb300.md`.\n",
         "Held-out products (square, n log-uniform in [1024, 4096], phi ~ U(0, 8), seeds outside the",
         "training data; A and B drawn on the GPU by the Eq. 19 generator).  Timed with CUDA events on the",
         "stream, one call each into preallocated outputs: `emu_dgemm_auto` / `emu_dgemm_auto_II` with the",
         "committed weights -- feature",
         "scan, MLP, the 64-entry double-double probe and every escalation and recomputation inside the",
         "timed region -- against `emu_dgemm` at the fixed p (N) that passes every training product (Scheme I",
         "INT8 p = 12; Scheme II with norm scaling N = 20).  Pass: max |C - AB| / (|A||B|) <= tol on 256",
         "other sampled entries against the GPU double-double probe.\n",
         "| scheme | tol | products | fixed | mean chosen | auto pass | fixed pass | auto total ms | fixed total ms"
         " | speed-up |",
         "|---|---|---|---|---|---|---|---|---|---|"]
    for d in summ:
        o.append("| %s | %.0e | %d | %d | %.2f | %.0f %% | %.0f %% | %.1f | %.1f | %.2fx |" % (
            d["scheme"], d["tol"], d["products"], d["fixed"], d["mean_used"], 100 * d["pass_auto"],
            100 * d["pass_fixed"], d["ms_auto_total"], d["ms_fixed_total"], d["speedup_vs_fixed"]))
    o.append("\nPer product (time in ms; chosen = the p or N of the returned result):\n")
    o.append("| scheme | n | phi | tol | chosen | ms auto | ms fixed | err auto | err fixed |")
    o.append("|---|---|---|---|---|---|---|---|---|")
    for d in pts:
        o.append("| %s | %d | %.2f | %.0e | %d | %.2f | %.2f | %.2e | %.2e |" % (
            d["scheme"], d["n"], d["phi"], d["tol"], d["used"], d["ms_auto"], d["ms_fixed"], d["err_auto"],
            d["err_fixed"]))
    return "\n".join(o) + "\n"


def run_suite(path, args):
    """Secondary measurements: every path of the library on one GPU, one JSON
    object per point (device-resident inputs, CUDA-event timing, 1 warm-up +
    3 timed calls, error on 8 x 64 sampled entries vs double-double)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2606_25453_gb300 as emu
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    h = emu.Handle(0)
    out = open(path, "w")

    def emit(d):
        out.write(json.dumps(d) + "\n")
        out.flush()
        print(json.dumps(d), flush=True)

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    rng = np.random.Generator(np.random.PCG64(99))

    def sampled_err(A, B, C, complex_=False):
        """max |C - AB| / (|A||B|) over 8 x 64 sampled entries, AB from the GPU
        double-double probe (complex: each part as a real dot product of the
        sampled rows and columns over 2K terms; |.| the complex modulus)."""
        ri = np.sort(rng.choice(A.shape[0], 8, replace=False))
        ci = np.sort(rng.choice(B.shape[1], 64, replace=False))
        As = torch.from_numpy(np.ascontiguousarray(A[ri])).to(dev)
        Bs = torch.from_numpy(np.ascontiguousarray(B[:, ci])).to(dev)
        rs, cs = np.arange(len(ri)), np.arange(len(ci))
        if not complex_:
            hi, lo, den = probe_ref(emu, h, As.double(), Bs.double(), rs, cs)
            return float(np.max(np.abs((C[ri][:, ci] - hi) - lo) / den))
        Ae = torch.cat([As.real.double(), As.imag.double()], dim=1).contiguous()
        Bre = torch.cat([Bs.real.double(), -Bs.imag.double()], dim=0).contiguous()
        Bim = torch.cat([Bs.imag.double(), Bs.real.double()], dim=0).contiguous()
        hr, lr, _ = probe_ref(emu, h, Ae, Bre, rs, cs)
        hm, lm, _ = probe_ref(emu, h, Ae, Bim, rs, cs)
        den = (As.abs().double() @ Bs.abs().double()).cpu().numpy()
        Cs = C[ri][:, ci]
        d = np.hypot((Cs.real - hr) - lr, (Cs.imag - hm) - lm)
        return float(np.max(d / den))

    if args.suite_part in ("selector", "grouped"):
        (selector_points if args.suite_part == "selector" else
         lambda *a: grouped_points(*a, timed))(emu, h, dev, emit)
        out.close()
        h.close()
        return

    cache = {}

    def pair(n, phi, dtype=np.float64):
        key = (n, phi, dtype)
        if key not in cache:
            cache.clear()
            A, B = synth.gemm_pair(n, n, n, phi, 7)
            if dtype is np.float32:
                A, B = A.astype(np.float32), B.astype(np.float32)
            cache[key] = (A, B, torch.from_numpy(A).to(dev), torch.from_numpy(B).to(dev))
        return cache[key]

    def scheme_II_points():
        """Scheme II DGEMM with the engine of this process (the default bf16
        tcgen05 one, or INT8 mma.sync under EMU_II_ENGINE=mma): n = 8192 at
        two phi and N_m = 8..20, and (default engine only) n = 4096 and 16384
        at phi = 0.5 and N_m = 12, 16, 20."""
        engine = "int8 mma.sync" if os.environ.get("EMU_II_ENGINE") == "mma" else "bf16 tcgen05"
        pts = [(8192, 0.5, (12, 16, 20) if args.suite_part == "ii" else (8, 10, 12, 14, 16, 18, 20))]
        if args.suite_part != "ii":
            pts += [(8192, 4.0, (8, 10, 12, 14, 16, 18, 20)), (4096, 0.5, (12, 16, 20)), (16384, 0.5, (12, 16, 20))]
        for n2, phi, nms in pts:
            A, B, Ad, Bd = pair(n2, phi)
            Cd = torch.empty((n2, n2), dtype=torch.float64, device=dev)
            for nm in nms:
                ms = timed(lambda: emu.dgemm(Ad, Bd, Cd, scheme="II", p=nm, handle=h), reps=1 if n2 > 8192 else 3)
                emit({"path": "emu_dgemm_II", "n": n2, "phi": phi, "nm": nm, "tflops": 2 * n2 ** 3 / ms / 1e9,
                      "engine": engine, "tensor_tops": 2 * nm * n2 ** 3 / ms / 1e9, "ms": ms,
                      "err": sampled_err(A, B, Cd.cpu().numpy())})
            del Cd

    if args.suite_part == "ii":
        scheme_II_points()
        out.close()
        h.close()
        return
    every = args.suite_part == "all"  # scheme2: only the rows of the bf16 tcgen05 Scheme II paths

    # cuBLAS references on this GPU
    for n in (4096, 8192) if every else ():
        A, B, Ad, Bd = pair(n, 0.5)
        ms = timed(lambda: Ad @ Bd, reps=2)
        C = (Ad @ Bd).cpu().numpy()
        emit({"path": "cublas_dgemm", "n": n, "tflops": 2 * n ** 3 / ms / 1e9, "ms": ms, "err": sampled_err(A, B, C)})
        Af, Bf = Ad.float(), Bd.float()
        ms = timed(lambda: Af @ Bf)
        emit({"path": "cublas_sgemm", "n": n, "tflops": 2 * n ** 3 / ms / 1e9, "ms": ms,
              "err": sampled_err(A.astype(np.float32).astype(np.float64), B.astype(np.float32).astype(np.float64),
                                 (Af @ Bf).cpu().numpy().astype(np.float64))})
    # Scheme I DGEMM: p sweep, phi sweep
    for n in (4096, 8192) if every else ():
        for phi in (0.5, 2.0, 4.0):
            A, B, Ad, Bd = pair(n, phi)
            Cd = torch.empty((n, n), dtype=torch.float64, device=dev)
            for p in range(4, 13) if phi == 4.0 else range(4, 9):
                ms = timed(lambda: emu.dgemm(Ad, Bd, Cd, scheme="I", p=p, handle=h))
                emit({"path": "emu_dgemm_I", "n": n, "phi": phi, "p": p, "tflops": 2 * n ** 3 / ms / 1e9,
                      "int8_tops": p * (p + 1) * n ** 3 / ms / 1e9, "ms": ms,
                      "err": sampled_err(A, B, Cd.cpu().numpy())})
    n = 16384
    if every:
        A, B = synth.gemm_pair(n, n, n, 0.5, 7)
        Ad, Bd = torch.from_numpy(A).to(dev), torch.from_numpy(B).to(dev)
        Cd = torch.empty((n, n), dtype=torch.float64, device=dev)
    for p in (7, 8) if every else ():
        ms = timed(lambda: emu.dgemm(Ad, Bd, Cd, scheme="I", p=p, handle=h), reps=1)
        emit({"path": "emu_dgemm_I", "n": n, "phi": 0.5, "p": p, "tflops": 2 * n ** 3 / ms / 1e9,
              "int8_tops": p * (p + 1) * n ** 3 / ms / 1e9, "ms": ms, "err": sampled_err(A, B, Cd.cpu().numpy())})
    # Scheme I on E4M3 slices (tcgen05 kernel)
    for p in (8, 10, 11, 12) if every else ():
        ms = timed(lambda: emu.dgemm(Ad, Bd, Cd, scheme="I_F8", p=p, handle=h), reps=1)
        emit({"path": "emu_dgemm_I_F8", "n": n, "phi": 0.5, "p": p, "tflops": 2 * n ** 3 / ms / 1e9,
              "f8_tops": p * (p + 1) * n ** 3 / ms / 1e9, "ms": ms, "err": sampled_err(A, B, Cd.cpu().numpy())})
    if every:
        del Ad, Bd, Cd
    for n in (4096, 8192) if every else ():
        for phi in (0.5, 4.0):
            A, B, Ad, Bd = pair(n, phi)
            Cd = torch.empty((n, n), dtype=torch.float64, device=dev)
            for p in (8, 10, 11, 12):
                ms = timed(lambda: emu.dgemm(Ad, Bd, Cd, scheme="I_F8", p=p, handle=h))
                emit({"path": "emu_dgemm_I_F8", "n": n, "phi": phi, "p": p, "tflops": 2 * n ** 3 / ms / 1e9,
                      "f8_tops": p * (p + 1) * n ** 3 / ms / 1e9, "ms": ms,
                      "err": sampled_err(A, B, Cd.cpu().numpy())})
    # naive (INT32 partials to HBM + separate shift-reduce) vs fused, k <= K_c
    n = 4096
    if every:
        A, B, Ad, Bd = pair(n, 0.5)
    for f8, p in ((False, 8), (True, 11)) if every else ():
        _, EA = emu.split_I(Ad, p, operand=0, handle=h, f8=f8)
        _, FB = emu.split_I(Bd, p, operand=1, handle=h, f8=f8)
        Cn = torch.empty((n, n), dtype=torch.float64, device=dev)
        Cf = torch.empty((n, n), dtype=torch.float64, device=dev)

        def naive():
            Cs = emu.partials_I(Ad, Bd, p, handle=h, f8=f8)
            emu.shift_reduce_I(Cs, EA, FB, p, f8=f8, C=Cn, handle=h)

        ms_naive = timed(naive)
        ms_fused = timed(lambda: emu.dgemm(Ad, Bd, Cf, scheme="I_F8" if f8 else "I", p=p, handle=h))
        emit({"path": "ablation_naive_vs_fused", "n": n, "p": p, "slices": "e4m3" if f8 else "int8",
              "ms_naive": ms_naive, "ms_fused": ms_fused, "speedup_fused": ms_naive / ms_fused,
              "int32_partials_bytes": 4 * p * n * n, "bit_identical": bool(torch.equal(Cn, Cf))})
    # Scheme I SGEMM
    for p in (3, 4) if every else ():
        A, B, Ad, Bd = pair(8192, 0.5, np.float32)
        Cd = torch.empty((8192, 8192), dtype=torch.float32, device=dev)
        ms = timed(lambda: emu.sgemm(Ad, Bd, Cd, scheme="I", p=p, handle=h))
        emit({"path": "emu_sgemm_I", "n": 8192, "phi": 0.5, "p": p, "tflops": 2 * 8192 ** 3 / ms / 1e9,
              "int8_tops": p * (p + 1) * 8192 ** 3 / ms / 1e9, "ms": ms,
              "err": sampled_err(A.astype(np.float64), B.astype(np.float64), Cd.cpu().numpy().astype(np.float64))})
    # Scheme II SGEMM on the bf16 engine: FP32-level accuracy from 6-8 moduli
    A, B, Ad, Bd = pair(8192, 0.5, np.float32)
    Cd = torch.empty((8192, 8192), dtype=torch.float32, device=dev)
    for nm in (6, 7, 8):
        ms = timed(lambda: emu.sgemm(Ad, Bd, Cd, scheme="II", p=nm, handle=h))
        emit({"path": "emu_sgemm_II", "n": 8192, "phi": 0.5, "nm": nm, "tflops": 2 * 8192 ** 3 / ms / 1e9,
              "tensor_tops": 2 * nm * 8192 ** 3 / ms / 1e9, "ms": ms,
              "err": sampled_err(A.astype(np.float64), B.astype(np.float64), Cd.cpu().numpy().astype(np.float64))})
    scheme_II_points()
    engine = "int8 mma.sync" if os.environ.get("EMU_II_ENGINE") == "mma" else "bf16 tcgen05"
    import tempfile
    if every:
        with tempfile.NamedTemporaryFile(suffix=".jsonl", delete=False) as tf:
            child_path = tf.name
        subprocess.run([sys.executable, os.path.abspath(__file__), "--suite", child_path, "--suite-part", "ii"],
                       env=dict(os.environ, EMU_II_ENGINE="mma"), check=True, stdout=subprocess.DEVNULL)
        for line in open(child_path):
            d = json.loads(line)
            d["path"] = "emu_dgemm_II_int8"
            emit(d)
        os.unlink(child_path)
    # Scheme II with norm-based scaling: bits and speed at the same N_m
    for phi in (0.5, 4.0):
        A, B, Ad, Bd = pair(8192, phi)
        Cd = torch.empty((8192, 8192), dtype=torch.float64, device=dev)
        for nm in (8, 10, 12, 14, 16):
            ms = timed(lambda: emu.dgemm(Ad, Bd, Cd, scheme="II_NORM", p=nm, handle=h))
            emit({"path": "emu_dgemm_II_norm", "n": 8192, "phi": phi, "nm": nm, "tflops": 2 * 8192 ** 3 / ms / 1e9,
                  "engine": engine, "tensor_tops": 2 * nm * 8192 ** 3 / ms / 1e9, "ms": ms,
                  "err": sampled_err(A, B, Cd.cpu().numpy())})
    cache.clear()
    # ZGEMM 3M vs cuBLAS ZGEMM
    n = 8192
    A, B = synth.gemm_pair_complex(n, n, n, 1.0, 7)
    Ad, Bd = torch.from_numpy(A).to(dev), torch.from_numpy(B).to(dev)
    if every:
        ms = timed(lambda: Ad @ Bd, reps=1)
        emit({"path": "cublas_zgemm", "n": n, "tflops_8mnk": 8 * n ** 3 / ms / 1e9, "ms": ms,
              "err": sampled_err(A, B, (Ad @ Bd).cpu().numpy(), True)})
    Cd = torch.empty((n, n), dtype=torch.complex128, device=dev)
    for nm in (12, 16, 20):
        ms = timed(lambda: emu.zgemm(Ad, Bd, Cd, nm=nm, handle=h), reps=1)
        emit({"path": "emu_zgemm_3m", "n": n, "phi": 1.0, "nm": nm, "tflops_8mnk": 8 * n ** 3 / ms / 1e9,
              "tflops_2mnk": 2 * n ** 3 / ms / 1e9, "tensor_tops": 6 * nm * n ** 3 / ms / 1e9, "engine": engine, "ms": ms,
              "err": sampled_err(A, B, Cd.cpu().numpy(), True)})
    # ZGEMM 4M (Scheme I)
    for sc, p in (("I", 8), ("I_F8", 11), ("I_F8", 12)) if every else ():
        ms = timed(lambda: emu.zgemm(Ad, Bd, Cd, scheme=sc, p=p, handle=h), reps=1)
        emit({"path": "emu_zgemm_4m", "scheme": sc, "n": n, "phi": 1.0, "p": p, "tflops_8mnk": 8 * n ** 3 / ms / 1e9,
              "tflops_2mnk": 2 * n ** 3 / ms / 1e9, "ms": ms, "err": sampled_err(A, B, Cd.cpu().numpy(), True)})
    # CGEMM (complex64): cuBLAS, Scheme I 4M, Scheme II 3M
    Af, Bf = Ad.to(torch.complex64), Bd.to(torch.complex64)
    A32, B32 = A.astype(np.complex64).astype(np.complex128), B.astype(np.complex64).astype(np.complex128)
    if every:
        ms = timed(lambda: Af @ Bf, reps=2)
        emit({"path": "cublas_cgemm", "n": n, "tflops_8mnk": 8 * n ** 3 / ms / 1e9, "ms": ms,
              "err": sampled_err(A32, B32, (Af @ Bf).cpu().numpy().astype(np.complex128), True)})
    Cf = torch.empty((n, n), dtype=torch.complex64, device=dev)
    for sc, p in (("I", 4), ("I_F8", 6), ("II", 8), ("II", 10)) if every else (("II", 8), ("II", 10)):
        ms = timed(lambda: emu.cgemm(Af, Bf, Cf, scheme=sc, p=p, handle=h), reps=2)
        emit({"path": "emu_cgemm", "scheme": sc, "n": n, "p_or_nm": p, "tflops_8mnk": 8 * n ** 3 / ms / 1e9,
              "ms": ms, "err": sampled_err(A32, B32, Cf.cpu().numpy().astype(np.complex128), True)})
    del Ad, Bd, Cd, Af, Bf, Cf
    if not every:
        out.close()
        h.close()
        return
    grouped_points(emu, h, dev, emit, timed)
    out.close()
    h.close()


def main():
    args = parse()
    if args.selector_md:
        print(selector_markdown(args.selector_md), end="")
        return
    if args.suite_md:
        print(suite_markdown(args.suite_md))
        return
    if args.suite:
        run_suite(args.suite, args)
        return
    if args.grouped_run:
        grouped_run(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
