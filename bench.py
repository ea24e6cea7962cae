"""Benchmark of the blaz compressed-matrix hot path on GB300.

One step = one pass of the path over the bandwidth-sweep workload: two
16384 x 16384 binary64 smooth fields A and B (16 Gaussian bumps + 1e-4
noise), resident in HBM:
    compress A, compress B, decompress A, A+B (compressed), 3.5*A
    (compressed), flattened dot <A,B>, and one line-column dot (Algorithm 3).
value = algorithmic bytes of the step (557 B per block for compress and
decompress, 135 for add, 90 for scale and for the dot inputs) / step time,
in GB/s, summed over all ranks.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl blaz|reference]

--impl reference times the CPU oracle (single-threaded C, the method as the
paper defines it) on a bounded sample of the same workload.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "compressed add/scale/dot GB/s (% HBM peak), matmul TFLOP/s, serve p50/p99"
BYTES_PER_BLOCK = {"compress": 557, "decompress": 557, "add": 135, "scale": 90, "dot": 90}
STEP_OPS = ["compress", "compress", "decompress", "add", "scale", "dot"]

def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="blaz", choices=["blaz", "reference"])
    p.add_argument("--side", type=int, default=16384)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--workload", default="sweep", choices=["sweep", "batch", "serve", "matmul", "rates"],
                   help="sweep: the bandwidth-sweep step (default line); batch / serve / matmul: the batched, "
                        "served and precision (matrix product) configurations, each printed as its own line")
    p.add_argument("--mm-side", type=int, default=4096, help="matmul workload: n = k = m")
    p.add_argument("--mm-mode", default="both", choices=["fp64", "split_bf16", "both"])
    p.add_argument("--serve-seconds", type=float, default=2.0)
    p.add_argument("--no-extras", action="store_true", help="skip the matmul and serve fields of the sweep line")
    return p.parse_args()


def step_bytes(side: int) -> int:
    nb = (side // 8) ** 2
    return nb * sum(BYTES_PER_BLOCK[o] for o in STEP_OPS)


KERNEL_SOURCES = {"k_compress": ["paper_2202_13007_gb300/csrc/k_codec.cu",
                                  "paper_2202_13007_gb300/csrc/compress_fast.cuh",
                                  "paper_2202_13007_gb300/csrc/compress_fix.cuh",
                                  "paper_2202_13007_gb300/csrc/exact_div.cuh",
                                  "paper_2202_13007_gb300/csrc/block_codec.cuh",
                                  "paper_2202_13007_gb300/csrc/gmap.cuh",
                                  "paper_2202_13007_gb300/csrc/blaz_internal.cuh"]}


def kernel_sha(name: str) -> str:
    import hashlib

    h = hashlib.sha256()
    for f in KERNEL_SOURCES[name]:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled(name: str, key: str):
    """A per-block figure of the committed ncu summary (profiles/traffic.json);
    None when the kernel source changed since the capture."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            d = json.load(fh)[name]
    except Exception:
        return None
    if d.get("source_sha") != kernel_sha(name):
        return None
    return d.get(key)


def profiled_traffic(name: str, blocks: int):
    """DRAM bytes per launch from the committed ncu summary, scaled to `blocks`
    blocks; None when the kernel source changed since the capture."""
    per_block = profiled(name, "dram_bytes_per_block")
    return None if per_block is None else per_block * blocks


def probe_fp64(dev, st):
    """Measured binary64 issue rate (G additions/s) of the library's probe
    (4 independent DADD chains per thread, one CTA per SM) at 1, 2, 4, 8 and
    16 warps per SM, best of 3 launches each timed with CUDA events on `st`;
    returns (the maximum, {warps per SM: rate})."""
    import torch

    from paper_2202_13007_gb300 import blaz as B

    out = torch.empty(torch.cuda.get_device_properties(dev).multi_processor_count * 16 * 32, dtype=torch.float64,
                      device=dev)
    rates = {}
    for w in (1, 2, 4, 8, 16):
        B.probe_fp64_rate(64, out, w, st)
        best = None
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            ops = B.probe_fp64_rate(4096 if w >= 4 else 1024, out, w, st)
            e1.record(st)
            torch.cuda.synchronize()
            rate = ops / (e0.elapsed_time(e1) * 1e-3) / 1e9
            best = rate if best is None else max(best, rate)
        rates[w] = best
    return max(rates.values()), rates


def max_over_ranks(ms: float, dist, device) -> float:
    """The slowest rank's elapsed time: the job's time when every rank runs
    its own replica of the step (weak scaling)."""
    if dist is None:
        return ms
    import torch

    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, side: int, steps: int, ms: float) -> float:
    """Whole-job GB/s of algorithmic bytes: every rank's steps over the job's time."""
    return world * step_bytes(side) * steps / (ms * 1e-3) / 1e9


def replica_seeds(side: int, rank: int):
    """Seeds of fields A and B on a rank: each replica draws its own pair."""
    return side + 2 * rank, side + 1 + 2 * rank


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.gpu)], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except Exception:
            pass
        finally:
            try:
                os.unlink(self.path)
            except Exception:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        busy = [x for x in sm if x >= 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(busy), "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def per_op_table(op_events, nb, hbm):
    """Per operation of the timed steps: mean CUDA-event time of one call, and
    the algorithmic bytes of one call (bytes per block x blocks; the
    line-column dot reads 2 x 2048 blocks of 45 B) over that time, as GB/s
    and as a fraction of the HBM peak."""
    out = {}
    for name, pairs in op_events.items():
        ms = statistics.mean(a.elapsed_time(b) for a, b in pairs)
        byts = BYTES_PER_BLOCK[name] * nb if name in BYTES_PER_BLOCK else 2 * 45 * int(round(nb ** 0.5))
        out[name] = {"ms": ms, "bytes": byts, "gb_per_s": byts / (ms * 1e-3) / 1e9,
                     "frac_of_hbm_peak": byts / (ms * 1e-3) / 1e9 / hbm, "calls": len(pairs)}
    return out


def compress_roofline(nb, comp_ms, hbm, hbm_src, fp64_probe, fp64_by_warps):
    """Roofline of the dominant kernel pair (k_compress_fast + k_compress_fix,
    one compress call): the algorithmic 557 B per block (512 in, 45 out)
    over the call's mean CUDA-event time, against the measured HBM copy
    peak.  Beside it, the binary64 instructions the kernels issue (ncu count
    per block, committed under profiles/) over the same time, against the
    binary64 issue ceiling measured live by the library's probe."""
    achieved = 557 * nb / (comp_ms * 1e-3) / 1e9
    inst = profiled("k_compress", "fp64_inst_per_block")
    issued = inst * nb / (comp_ms * 1e-3) / 1e9 if inst else None
    return {"kernel": "k_compress_fast + k_compress_fix", "bound": "hbm", "achieved": achieved, "peak": hbm,
            "unit": "GB/s", "frac": achieved / hbm, "traffic": profiled_traffic("k_compress", nb),
            "traffic_unit": "bytes per launch (ncu DRAM read + write per block x blocks)",
            "source_sha": kernel_sha("k_compress"), "peak_source": hbm_src, "ms_per_launch": comp_ms,
            "algorithmic_bytes_per_launch": 557 * nb,
            "limiter": "binary64 issue: the specification's exact binary64 steps, not memory",
            "fp64_issue": {"achieved_gops": issued, "peak_gops": fp64_probe,
                           "frac": issued / fp64_probe if issued and fp64_probe else None,
                           "inst_per_block": inst,
                           "basis": "ncu binary64 warp instructions x 32 / 32 blocks per block, x blocks / launch "
                                    "time; peak: blaz_probe_fp64_rate measured in this run",
                           "probe_by_warps_per_sm": fp64_by_warps}}


def run_oracle_step(O, A, Bm):
    """One step of the path evaluated by the CPU oracle (the line-column dot,
    whose bytes the step does not count, is left out); returns seconds."""
    t = time.perf_counter()
    ca = O.compress(A)
    cb = O.compress(Bm)
    O.decompress(ca)
    O.add(ca, cb)
    O.scale(ca, 3.5)
    O.dot(ca, cb)
    return time.perf_counter() - t


def oracle_sample(side: int, rows: int):
    import workloads as W

    A = W.bump_field(side, side, rows=rows)
    Bm = W.bump_field(side, side + 1, rows=rows)
    return A, Bm


def cpu_baseline(side: int, rows: int = 8192):
    """The oracle (single-threaded C) on the first `rows` rows of both fields."""
    import oracle as O

    O.build()
    A, Bm = oracle_sample(side, rows)
    secs = run_oracle_step(O, A, Bm)
    nb = (rows // 8) * (side // 8)
    byts = nb * sum(BYTES_PER_BLOCK[o] for o in STEP_OPS)
    return {"value": byts / secs / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": f"one oracle step on the first {rows} rows of both {side}x{side} fields "
                      f"({nb} blocks, {secs:.1f} s)"}


def cpu_parallel(side: int, rows: int = 8192):
    """The same oracle step block-parallel over the host cores: the sample is
    cut into block-row slabs, one oracle call chain per slab, on a thread pool
    (the C oracle runs without the GIL)."""
    import concurrent.futures as cf

    import oracle as O

    O.build()
    O.dct_tables()                      # initialise the oracle's tables before threading
    A, Bm = oracle_sample(side, rows)
    cores = os.cpu_count() or 1
    step = max(8, (rows // cores) // 8 * 8)
    spans = [(r, min(rows, r + step)) for r in range(0, rows, step)]
    t = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=cores) as ex:
        list(ex.map(lambda sp: run_oracle_step(O, A[sp[0]:sp[1]], Bm[sp[0]:sp[1]]), spans))
    secs = time.perf_counter() - t
    nb = (rows // 8) * (side // 8)
    byts = nb * sum(BYTES_PER_BLOCK[o] for o in STEP_OPS)
    return {"value": byts / secs / 1e9, "unit": "GB/s", "cores": cores, "kind": "oracle, block-parallel",
            "sample": f"the oracle step on the first {rows} rows of both {side}x{side} fields in "
                      f"{len(spans)} block-row slabs on {cores} threads ({secs:.2f} s)"}


def plain_way(B, torch, ca, cb, dev):
    """The same operations done the plain way on the same GPU: decompress,
    operate in binary64 (torch), recompress; against the compressed-domain
    operations.  Accuracy: each result against the exact operation on the
    decompressed operands (max |error| / max |exact|)."""
    n = ca.rows
    Ah = torch.empty((n, n), dtype=torch.float64, device=dev)
    Bh = torch.empty_like(Ah)
    Xh = torch.empty_like(Ah)
    cx = B.CMat.empty(n, n, dev)
    res = torch.empty((), dtype=torch.float64, device=dev)

    def timed(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    def plain_add():
        B.decompress(ca, out=Ah)
        B.decompress(cb, out=Bh)
        torch.add(Ah, Bh, out=Xh)
        B.compress(Xh, out=cx)

    def plain_scale():
        B.decompress(ca, out=Ah)
        torch.mul(Ah, 3.5, out=Xh)
        B.compress(Xh, out=cx)

    def plain_dot():
        B.decompress(ca, out=Ah)
        B.decompress(cb, out=Bh)
        torch.dot(Ah.view(-1), Bh.view(-1), out=res)

    out = {"add": {"compressed_ms": timed(lambda: B.add(ca, cb, out=cx)), "plain_ms": timed(plain_add)},
           "scale": {"compressed_ms": timed(lambda: B.scale(ca, 3.5, out=cx)), "plain_ms": timed(plain_scale)},
           "dot": {"compressed_ms": timed(lambda: B.dot(ca, cb, out=res)), "plain_ms": timed(plain_dot)}}
    # accuracy against the exact operation on the decompressed operands
    B.decompress(ca, out=Ah)
    B.decompress(cb, out=Bh)
    exact = Ah + Bh
    scale_ = float(exact.abs().max())
    B.add(ca, cb, out=cx)
    B.decompress(cx, out=Xh)
    out["add"]["compressed_err"] = float((Xh - exact).abs().max()) / scale_
    B.compress(exact, out=cx)
    B.decompress(cx, out=Xh)
    out["add"]["plain_err"] = float((Xh - exact).abs().max()) / scale_
    exact = Ah * 3.5
    scale_ = float(exact.abs().max())
    B.scale(ca, 3.5, out=cx)
    B.decompress(cx, out=Xh)
    out["scale"]["compressed_err"] = float((Xh - exact).abs().max()) / scale_
    B.compress(exact, out=cx)
    B.decompress(cx, out=Xh)
    out["scale"]["plain_err"] = float((Xh - exact).abs().max()) / scale_
    ref = float(torch.dot(Ah.view(-1), Bh.view(-1)))
    absref = float(torch.dot(Ah.abs().view(-1), Bh.abs().view(-1)))
    out["dot"]["compressed_err"] = abs(float(B.dot(ca, cb, out=res)) - ref) / absref
    out["dot"]["plain_err"] = 0.0
    for v in out.values():
        v["speedup"] = v["plain_ms"] / v["compressed_ms"]
    out["config"] = (f"{n}x{n} bump fields: plain = decompress (blaz), binary64 op (torch), recompress (blaz); "
                     "err = max|result - exact op on the decompressed operands| / max|exact| "
                     "(dot: |error| / sum|A_hat B_hat|)")
    del Ah, Bh, Xh
    return out


def reference_arm(args, rank: int, world: int):
    """--impl reference: the oracle as it stands, timed on the host cores."""
    if rank != 0:
        return
    import oracle as O

    O.build()
    rows = 2048
    A, Bm = oracle_sample(args.side, rows)
    for _ in range(args.warmup):
        run_oracle_step(O, A, Bm)
    secs = [run_oracle_step(O, A, Bm) for _ in range(args.steps)]
    nb = (rows // 8) * (args.side // 8)
    byts = nb * sum(BYTES_PER_BLOCK[o] for o in STEP_OPS)
    total = sum(secs)
    value = byts * args.steps / total / 1e9
    sample = (f"each step: one oracle step on the first {rows} rows of both {args.side}x{args.side} fields "
              f"({nb} blocks)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config(args.side),
            "cpu_baseline": {"value": value, "unit": "GB/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config(side):
    return {"workload": f"bandwidth sweep {side}x{side} binary64 bump fields: compress A, compress B, "
                        "decompress A, A+B, 3.5*A, dot <A,B>, dot line 17 . column 200",
            "side": side, "blocks_per_matrix": (side // 8) ** 2,
            "l2": "inputs larger than L2 (2 GiB per field), no flush", "parallelism": "replicas"}


def matmul_errors(torch, Ah, Bh, C):
    """Errors of a product C against the binary64 product of the decompressed
    operands (cuBLAS DGEMM, whose own error, about sqrt(k) 2^-53 of
    (|A_hat||B|)_ij, is far below the 1e-12 being checked): the componentwise
    max_ij |C - C_ref|_ij / (|A_hat||B|)_ij, and the elementwise max relative
    error over the entries with |C_ref| > 1e-8 max |C_ref|."""
    ref = Ah @ Bh
    err = (C - ref).abs()
    comp = float((err / (Ah.abs() @ Bh.abs()).clamp_min(1e-300)).max())
    big = ref.abs() > 1e-8 * float(ref.abs().max())
    rel = float((err[big] / ref.abs()[big]).max())
    return {"max_componentwise_error": comp, "max_relative_error": rel,
            "error_basis": "against cuBLAS DGEMM of the decompressed operands"}


def matmul_extras(B, W, torch, dev):
    """Precision configuration: compressed 4096^2 bump field times a smoothed
    N(0,1) 4096^2 matrix, FP64 DMMA path and split-bf16 tcgen05 path."""
    n = 4096
    ta = W.bump_field_torch(n, n, dev)
    g = torch.Generator(device=dev)
    g.manual_seed(7)
    z = torch.randn((n, n), generator=g, dtype=torch.float64, device=dev)
    Bd = sum(torch.roll(z, (di, dj), (0, 1)) for di in range(-2, 3) for dj in range(-2, 3)) / 25.0
    ga = B.compress(ta)
    gb = B.compress(Bd)
    C = torch.empty((n, n), dtype=torch.float64, device=dev)
    out = {}
    cases = (("fp64", 2, lambda m: B.matmul(ga, Bd, mode=m, out=C)),
             ("split_bf16", 10, lambda m: B.matmul(ga, Bd, mode=m, out=C)),
             ("cc_fp64", 2, lambda m: B.matmul_cc(ga, gb, mode="fp64", out=C)),
             ("cc_split_bf16", 10, lambda m: B.matmul_cc(ga, gb, mode="split_bf16", out=C)))
    for name, reps, fn in cases:
        fn(name)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn(name)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        out[name] = {"ms": ms, "tflops": 2 * n ** 3 / (ms * 1e-3) / 1e12}
        Ah = B.decompress(ga)
        out[name].update(matmul_errors(torch, Ah, B.decompress(gb) if name.startswith("cc_") else Bd, C))
        del Ah
    out["shape"] = ("4096x4096x4096: compressed A times dense B (fp64, split_bf16) and times compressed B "
                    "(cc_*, both operands decompressed once)")
    return out


def shape_and_file_extras(B, W, torch, dev):
    """Any-shape matrices and files: compress and dot of a 4095 x 4093 bump
    field (edge-replicated to 4096 x 4096) against the 4096 x 4096 field, and
    save / load of its compressed form (11.8 MB) through a local file."""
    import os
    import tempfile

    def timed(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    n = 4096
    ta = W.bump_field_torch(n, n, dev)
    tb = W.bump_field_torch(n, n + 1, dev)
    pa, pb = ta[:n - 1, :n - 3], tb[:n - 1, :n - 3]
    ga, gb = B.compress(ta), B.compress(tb)
    qa, qb = B.compress_padded(pa), B.compress_padded(pb)
    res = torch.empty((), dtype=torch.float64, device=dev)
    out = {
        "compress_ms": timed(lambda: B.compress(ta, out=ga)),
        "compress_padded_ms": timed(lambda: B.compress_padded(pa, out=qa)),
        "dot_ms": timed(lambda: B.dot(ga, gb, out=res)),
        "dot_padded_ms": timed(lambda: B.dot_padded(qa, qb, out=res)),
    }
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "a.blaz")
        import time

        t0 = time.perf_counter()
        B.save(ga, path)
        t1 = time.perf_counter()
        B.load(path, out=gb)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        out.update({"save_ms": (t1 - t0) * 1e3, "load_ms": (t2 - t1) * 1e3, "file_bytes": os.path.getsize(path)})
    out["config"] = ("4095x4093 padded vs 4096x4096 bump fields (CUDA events); save/load of a 4096x4096 "
                     "compressed matrix through a local file (host wall clock)")
    return out


def rate_extras(B, W, torch, dev):
    """Tunable rate (the first r DCT rows and columns kept): compress,
    decompress, add and dot of 4096 x 4096 bump fields at r = 1, 2, 4, 8, with the
    compression ratio 512 / (17 + keep(r)) and the relative 2-norm error of the
    round trip.  r = 2 is also timed on the 28-code kernels for comparison."""

    def timed(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    n = 4096
    ta = W.bump_field_torch(n, n, dev)
    tb = W.bump_field_torch(n, n + 1, dev)
    back = torch.empty_like(ta)
    res = torch.empty((), dtype=torch.float64, device=dev)
    out = {}
    for r in (1, 2, 4, 8):
        ga, gb = B.compress_rate(ta, r), B.compress_rate(tb, r)
        gs = B.CMat.empty(n, n, dev, rate=r)
        B.decompress_rate(ga, out=back)
        err = float(torch.linalg.vector_norm(back - ta) / torch.linalg.vector_norm(ta))
        out[f"r{r}"] = {"keep": B.keep_count(r), "ratio": 512.0 / (17 + B.keep_count(r)), "rel_err": err,
                        "compress_ms": timed(lambda: B.compress_rate(ta, r, out=ga)),
                        "decompress_ms": timed(lambda: B.decompress_rate(ga, out=back)),
                        "add_ms": timed(lambda: B.add_rate(ga, gb, out=gs)),
                        "dot_ms": timed(lambda: B.dot_rate(ga, gb, out=res))}
        del ga, gb, gs
    g2, h2 = B.compress(ta), B.compress(tb)
    s2 = B.CMat.empty(n, n, dev)
    out["r2_28code_kernels"] = {"compress_ms": timed(lambda: B.compress(ta, out=g2)),
                                "decompress_ms": timed(lambda: B.decompress(g2, out=back)),
                                "add_ms": timed(lambda: B.add(g2, h2, out=s2)),
                                "dot_ms": timed(lambda: B.dot(g2, h2, out=res))}
    out["config"] = "4096x4096 bump fields (CUDA events, 5 reps after one warm-up); rate kernels: binary64, one thread per block"
    return out


def run_serve(args, B, W, torch, dev, seconds, max_batch, streams, mode="fp64", seed=13, rate=5000.0):
    """Poisson stream (5k req/s, sides log-uniform over multiples of 8 in
    [64, 4096], op mix 40/30/15/10/5 %) against a server with a 40 GB budget.
    Compress inputs and product operands are page-locked host views; add /
    scale / dot / matmul operate on a pool of resident matrices compressed
    beforehand (48 shapes drawn from the same law)."""
    import numpy as np

    side = 4096
    src_t = torch.empty((side, side), dtype=torch.float64, pin_memory=True)
    src_t.copy_(W.bump_field_torch(side, 4096, dev))
    bsrc_t = torch.empty((side, side), dtype=torch.float64, pin_memory=True)
    g = torch.Generator(device=dev)
    g.manual_seed(17)
    bsrc_t.copy_(torch.randn((side, side), generator=g, dtype=torch.float64, device=dev))
    src, bsrc = src_t.numpy(), bsrc_t.numpy()
    arena_t = torch.empty(2 << 27, dtype=torch.float64, pin_memory=True)     # 2 GiB of outputs
    arena = arena_t.numpy()
    reqs = W.poisson_requests(rate=rate, duration_s=seconds, seed=seed, lo=64, hi=side)
    prng = np.random.default_rng(seed + 1)
    pool_shapes = [(W._side(prng, 64, side), W._side(prng, 64, side)) for _ in range(48)]
    srv = B.Server(budget_bytes=40 << 30, streams=streams, max_batch=max_batch, matmul_mode=mode)
    pool = []
    for r, c in pool_shapes:
        ha = srv.submit("compress", A=src[:r, :c], pinned=True)
        hb = srv.submit("compress", A=src[side - r:, side - c:], pinned=True)
        pool.append((r, c, srv.wait(ha)["handle"], srv.wait(hb)["handle"]))
    warm = srv.stats()
    dots = torch.zeros(len(reqs), dtype=torch.float64, pin_memory=True).numpy()
    tickets, busy, waited = [], {}, set()
    off = 0
    t0 = time.perf_counter()
    for i, d in enumerate(reqs):
        now = time.perf_counter() - t0
        if d["t"] > now:
            time.sleep(d["t"] - now)
        r, c, ha, hb = pool[i % len(pool)]
        if d["op"] == "compress":
            tk = srv.submit("compress", A=src[:d["rows"], :d["cols"]], pinned=True)
        elif d["op"] == "add":
            tk = srv.submit("add", a=ha, b=hb)
        elif d["op"] == "scale":
            tk = srv.submit("scale", a=ha, c=d["c"])
        elif d["op"] == "dot":
            tk = srv.submit("dot", a=ha, b=hb, out=dots[i:i + 1], pinned=True)
        else:
            m = d["m"]
            need = r * m
            if off + need > arena.size:
                off = 0
            for lo_hi, tk_old in list(busy.items()):       # the region must be free again
                if lo_hi[0] < off + need and off < lo_hi[1]:
                    srv.wait(tk_old)
                    waited.add(tk_old)
                    del busy[lo_hi]
            out = arena[off:off + need].reshape(r, m)
            tk = srv.submit("matmul", a=ha, B=bsrc[:c, :m], out=out, pinned=True)
            busy[(off, off + need)] = tk
            off += need
        tickets.append(tk)
    for tk in tickets:
        if tk not in waited:
            srv.wait(tk)
    elapsed = time.perf_counter() - t0
    st = srv.stats()
    srv.destroy()
    n = len(reqs)
    return {"requests": n, "offered_rps": n / seconds, "throughput_rps": n / elapsed, "p50_ms": st["p50_us"] / 1e3,
            "p99_ms": st["p99_us"] / 1e3, "launches": st["launches"] - warm["launches"],
            "mean_batch": st["mean_batch"], "peak_device_gb": st["peak_bytes"] / 1e9, "matmul_mode": mode,
            "max_batch": max_batch, "streams": streams}


def serve_line(args):
    import torch

    import workloads as W
    from paper_2202_13007_gb300 import blaz as B

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    B.lib()
    with ClockSampler(0) as clk:
        batched = run_serve(args, B, W, torch, dev, args.serve_seconds, max_batch=0, streams=4, mode="split_bf16")
        single = run_serve(args, B, W, torch, dev, args.serve_seconds, max_batch=1, streams=1, mode="split_bf16")
    line = {"metric": METRIC + " [serve]", "value": batched["throughput_rps"], "unit": "req/s", "n_gpus": 1,
            "steps": 1, "warmup": 0, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": "served Poisson stream 5k req/s, sides log-uniform multiples of 8 in [64,4096], "
                                   "mix 40/30/15/10/5 % compress/add/scale/dot/matmul, 40 GB admission budget",
                       "seconds": args.serve_seconds},
            "serve": batched, "one_request_per_launch": single, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def matmul_line(args):
    """Precision configuration alone: compressed n x n bump field A (seed n)
    times a dense N(0,1) n x n matrix smoothed by a 5x5 box filter (seed 7),
    timed over --steps calls after --warmup, per mode; TFLOP/s = 2 n^3 / time."""
    import torch

    import workloads as W
    from paper_2202_13007_gb300 import blaz as B

    n = args.mm_side
    dev = torch.device("cuda", 0)
    ta = W.bump_field_torch(n, n, dev)
    g = torch.Generator(device=dev)
    g.manual_seed(7)
    z = torch.randn((n, n), generator=g, dtype=torch.float64, device=dev)
    Bd = sum(torch.roll(z, (di, dj), (0, 1)) for di in range(-2, 3) for dj in range(-2, 3)) / 25.0
    ga = B.compress(ta)
    C = torch.empty((n, n), dtype=torch.float64, device=dev)
    modes = ["fp64", "split_bf16"] if args.mm_mode == "both" else [args.mm_mode]
    res = {}
    for mode in modes:
        for _ in range(args.warmup):
            B.matmul(ga, Bd, mode=mode, out=C)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            B.matmul(ga, Bd, mode=mode, out=C)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        res[mode] = {"ms": ms, "tflops": 2 * n ** 3 / (ms * 1e-3) / 1e12}
        res[mode].update(matmul_errors(torch, B.decompress(ga), Bd, C))
    first = res[modes[0]]
    print(json.dumps({"metric": METRIC + " [matmul]", "value": first["tflops"], "unit": "TFLOP/s", "n_gpus": 1,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": first["ms"],
                      "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                      "data": "synthetic",
                      "config": {"workload": f"matmul {n}^3: compressed bump field times smoothed N(0,1)",
                                 "modes": res, "status": B.device_status()}}), flush=True)


def rates_line(args):
    """Tunable rate alone: the rates field of the sweep line (4096 x 4096
    bump fields, r = 1, 2, 4, 8 and the 28-code kernels) as its own line."""
    import torch

    import workloads as W
    from paper_2202_13007_gb300 import blaz as B

    dev = torch.device("cuda", 0)
    res = rate_extras(B, W, torch, dev)
    r2 = res["r2"]
    print(json.dumps({"metric": METRIC + " [tunable rate]", "value": r2["compress_ms"], "unit": "ms",
                      "n_gpus": 1, "steps": 5, "warmup": 1, "ms_per_step": r2["compress_ms"],
                      "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                      "data": "synthetic",
                      "config": {"workload": "tunable rate, 4096x4096 bump fields; value: rate-2 compress ms",
                                 "rates": res, "status": B.device_status()}}), flush=True)


def batch_line(args):
    """2000 mixed ops (sides log-uniform over multiples of 8 in [64, 2048]) as
    one autotuned, graph-captured persistent launch, against the same ops
    launched one by one through the single-op entry points."""
    import torch

    import workloads as W
    from paper_2202_13007_gb300 import blaz as B

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    B.lib()
    with ClockSampler(0) as clk:
        r = run_batch(B, W, torch, dev, max(3, args.steps))
    line = {"metric": METRIC + " [batch]", "value": r["ops"] / (r["ms"] * 1e-3), "unit": "ops/s", "n_gpus": 1,
            "steps": r["reps"], "warmup": 1, "ms_per_step": r["ms"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "2000 mixed ops, sides log-uniform multiples of 8 in [64,2048], mix 40/30/15/10/5 % "
                                   "compress/add/scale/dot/matmul (FP64 DMMA products), one persistent graph launch",
                       "autotuned": r["autotuned"], "plan_seconds": r["plan_seconds"]},
            "gb_per_s": r["gb_per_s"], "one_op_per_launch_ms": r["one_op_per_launch_ms"],
            "speedup_vs_one_op_per_launch": r["speedup_vs_one_op_per_launch"], "items": r["items"],
            "gpu_launches": r["reps"], "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def run_batch(B, W, torch, dev, reps):
    """Builds the 2000-op batch, plans it (autotuned, graph-captured) and
    times `reps` runs of the plan and two passes of the same ops launched one
    by one (CUDA events)."""
    specs = W.batch_ops(count=2000, seed=11)
    ops, singles = [], []
    byts = 0
    for d in specs:
        r, c, seed = d["rows"], d["cols"], d["seed"]
        X = W.bump_field_torch(c, seed, dev, rows=r)
        nb = (r // 8) * (c // 8)
        if d["op"] == "compress":
            out = B.CMat.empty(r, c)
            ops.append({"op": "compress", "A": X, "out": out})
            singles.append(lambda X=X, out=out: B.compress(X, out=out))
            byts += 557 * nb
        elif d["op"] == "add":
            a, b = B.compress(X), B.compress(W.bump_field_torch(c, seed + 1, dev, rows=r))
            out = B.CMat.empty(r, c)
            ops.append({"op": "add", "a": a, "b": b, "out": out})
            singles.append(lambda a=a, b=b, out=out: B.add(a, b, out=out))
            byts += 135 * nb
        elif d["op"] == "scale":
            a = B.compress(X)
            out = B.CMat.empty(r, c)
            ops.append({"op": "scale", "a": a, "c": d["c"], "out": out})
            singles.append(lambda a=a, cc=d["c"], out=out: B.scale(a, cc, out=out))
            byts += 90 * nb
        elif d["op"] == "dot":
            a, b = B.compress(X), B.compress(W.bump_field_torch(c, seed + 1, dev, rows=r))
            res = torch.empty(1, dtype=torch.float64, device=dev)
            ops.append({"op": "dot", "a": a, "b": b, "result": res})
            singles.append(lambda a=a, b=b, res=res: B.dot(a, b, out=res[0]))
            byts += 90 * nb
        else:
            a = B.compress(X)
            Bd = torch.randn((c, d["m"]), dtype=torch.float64, device=dev)
            C = torch.empty((r, d["m"]), dtype=torch.float64, device=dev)
            ops.append({"op": "matmul", "a": a, "B": Bd, "C": C})
            singles.append(lambda a=a, Bd=Bd, C=C: B.matmul(a, Bd, mode="fp64", out=C))
            byts += 45 * nb + 8 * c * d["m"] + 8 * r * d["m"]
    torch.cuda.synchronize()
    t_plan = time.perf_counter()
    plan = B.Batch(ops, autotune=True)
    t_plan = time.perf_counter() - t_plan
    info = plan.info()

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    ms_batch = timed(plan.run, reps)
    ms_single = timed(lambda: [f() for f in singles], 2)
    plan.free()
    del ops, singles
    torch.cuda.empty_cache()
    return {"ops": len(specs), "ms": ms_batch, "reps": reps, "plan_seconds": t_plan,
            "autotuned": {"blocks_per_item": info["blocks_per_item"], "ctas_per_sm": info["ctas_per_sm"]},
            "gb_per_s": byts / (ms_batch * 1e-3) / 1e9, "one_op_per_launch_ms": ms_single,
            "speedup_vs_one_op_per_launch": ms_single / ms_batch, "items": info["items"]}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        reference_arm(args, rank, world)
        return
    if args.workload == "serve":
        serve_line(args)
        return
    if args.workload == "batch":
        batch_line(args)
        return
    if args.workload == "rates":
        return rates_line(args)
    if args.workload == "matmul":
        matmul_line(args)
        return

    import torch

    import workloads as W
    from paper_2202_13007_gb300 import blaz as B

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    B.lib()
    n = args.side
    dev = torch.device("cuda", local)
    st = torch.cuda.current_stream()
    seed_a, seed_b = replica_seeds(n, rank)
    ta = W.bump_field_torch(n, seed_a, dev)
    tb = W.bump_field_torch(n, seed_b, dev)
    ca, cb, cs, cc = (B.CMat.empty(n, n, dev) for _ in range(4))
    dec = torch.empty((n, n), dtype=torch.float64, device=dev)
    res = torch.empty(2, dtype=torch.float64, device=dev)
    # per operation: (name, call), in step order
    step_ops = [("compress", lambda: B.compress(ta, out=ca)),
                ("compress", lambda: B.compress(tb, out=cb)),
                ("decompress", lambda: B.decompress(ca, out=dec)),
                ("add", lambda: B.add(ca, cb, out=cs)),
                ("scale", lambda: B.scale(ca, 3.5, out=cc)),
                ("dot", lambda: B.dot(ca, cb, out=res[0])),
                ("dot_rowcol", lambda: B.dot_rowcol(ca, cb, 17, 200, out=res[1]))]
    op_events = {name: [] for name, _ in step_ops}

    def step(record=False):
        for name, fn in step_ops:
            if record:
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
            fn()
            if record:
                e1.record(st)
                op_events[name].append((e0, e1))

    launches_per_step = 11  # compress x2 (uniform pass, binary64 pass, fix-up), decompress, add, scale, dot, dot_rowcol

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        t0.record(st)
        for _ in range(args.steps):
            step(record=True)
        t1.record(st)
        torch.cuda.synchronize()
    ms = max_over_ranks(t0.elapsed_time(t1), dist, dev)
    if dist:
        dist.barrier()
    ms_step = ms / args.steps
    value = job_throughput(world, n, args.steps, ms)

    nb = (n // 8) ** 2
    hbm, hbm_src = peaks()
    per_op = per_op_table(op_events, nb, hbm)
    comp_ms = per_op["compress"]["ms"]
    fp64_probe, fp64_by_warps = probe_fp64(dev, st)

    # End to end through the public API with host buffers, every step: A and B
    # compressed from page-locked host memory (blaz_compress_host pipelines the
    # host-to-device transfer with the compression), the same device
    # operations (decompress and scale of A run while B is still in flight),
    # then the packed payload of A+B and both dot results back to the host.
    e2e = None
    if not args.no_e2e:
        ha = torch.empty((n, n), dtype=torch.float64, pin_memory=True)
        hb = torch.empty((n, n), dtype=torch.float64, pin_memory=True)
        ha.copy_(ta)
        hb.copy_(tb)
        hs = torch.empty(cs.nbytes, dtype=torch.uint8, pin_memory=True)
        hr = torch.empty(2, dtype=torch.float64, pin_memory=True)

        def e2e_step():
            B.compress_host(ha, out=ca)
            B.decompress(ca, out=dec)
            B.scale(ca, 3.5, out=cc)
            B.compress_host(hb, out=cb)
            B.add(ca, cb, out=cs)
            B.dot(ca, cb, out=res[0])
            B.dot_rowcol(ca, cb, 17, 200, out=res[1])
            B.download(cs, hs)
            hr.copy_(res, non_blocking=True)

        # the link floor: the same host-to-device bytes as plain page-locked
        # copies, taken before and after the timed steps, so that a slow
        # timed region can be told apart from a link that was slow throughout
        def copy_floor():
            f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            f0.record(st)
            ta.copy_(ha, non_blocking=True)
            tb.copy_(hb, non_blocking=True)
            f1.record(st)
            torch.cuda.synchronize()
            return f0.elapsed_time(f1)

        for _ in range(args.warmup):
            e2e_step()
        torch.cuda.synchronize()
        floor_before = [copy_floor() for _ in range(3)]
        if dist:
            dist.barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(args.steps):
            e2e_step()
        e1.record(st)
        torch.cuda.synchronize()
        ems = max_over_ranks(e0.elapsed_time(e1), dist, dev)
        floor_after = [copy_floor() for _ in range(3)]
        h2d = 2 * n * n * 8
        d2h = cs.nbytes + 16
        e2e = {"value": job_throughput(world, n, args.steps, ems), "unit": "GB/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": ems / args.steps,
               "h2d_copy_ms_per_step": min(floor_before + floor_after),
               "h2d_copy_ms_before_after": [round(min(floor_before), 3), round(min(floor_after), 3)]}

    extras = None
    if rank == 0 and not args.no_extras:
        del dec
        torch.cuda.empty_cache()
        extras = {"matmul": matmul_extras(B, W, torch, dev), "shapes_files": shape_and_file_extras(B, W, torch, dev),
                  "plain_way": plain_way(B, torch, ca, cb, dev), "rates": rate_extras(B, W, torch, dev)}
        keys = ("p50_ms", "p99_ms", "throughput_rps", "offered_rps", "mean_batch", "launches")
        srv = run_serve(args, B, W, torch, dev, 1.0, max_batch=0, streams=4, mode="split_bf16")
        one = run_serve(args, B, W, torch, dev, 1.0, max_batch=1, streams=1, mode="split_bf16")
        extras["serve"] = {k: srv[k] for k in keys}
        extras["serve"]["one_request_per_launch"] = {k: one[k] for k in keys}
        extras["serve"]["config"] = ("1 s of the served Poisson stream (5k req/s), continuous batching on 4 streams, "
                                     "then the same stream one request per launch on one stream; "
                                     "full line: --workload serve")
        extras["batch"] = run_batch(B, W, torch, dev, 3)
        extras["batch"]["config"] = ("2000 mixed ops, one autotuned graph-captured persistent launch (3 runs) against "
                                     "the same ops launched one by one; full line: --workload batch")

    cpu = None
    cpu_par = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(n)
        cpu_par = cpu_parallel(n)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config(n),
            "frac_of_hbm_peak": value / world / hbm,
            "roofline": compress_roofline(nb, comp_ms, hbm, hbm_src, fp64_probe, fp64_by_warps),
            "per_op": per_op,
            "clocks": clk.summary(),
            "e2e": e2e,
            "gpu_launches": launches_per_step * args.steps,
            "cpu_baseline": cpu,
            "matmul_tflops": extras["matmul"] if extras else None,
            "serve": extras["serve"] if extras else None,
            "batch": extras["batch"] if extras else None,
            "shapes_files": extras["shapes_files"] if extras else None,
            "plain_way": extras["plain_way"] if extras else None,
            "rates": extras["rates"] if extras else None,
            "cpu_parallel": cpu_par,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
