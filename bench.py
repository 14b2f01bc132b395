"""Benchmark: batched SAM construction on the 256x256 Q1 diffusion sequence.

Workload (one "step" = the whole hot path once): the sequence of 10
variable-coefficient diffusion matrices (9-point Q1 stencil, n = 65536,
kappa_k = kappa_0 exp(0.05 k GRF_k)), level-2 patterns of every A_k, and the
10 maps M_k = argmin ||A_k M - A_0||_F built in one batched pass: CSR->CSC,
patterns, shadow rows and size bins, gather + FP32 Householder QR + FP64
refinement, scatter into CSR, FP64 residual ||A_k M_k - A_0||_F per map.
Metric: map columns per second (10 x 65536 columns per step).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun each rank builds its own
copy of the sequence (weak scaling, no data-path collective); time is the
maximum over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)

METRIC = "SAM columns/s (batched FP32+refine vs FP64, same GB300, <=1e-10 rel err); % roofline"
UNIT = "columns/s"


def alu_peaks(sms: int, mhz: float):
    """Nominal ALU peaks (FLOP/s) of a Blackwell GPU with `sms` SMs at `mhz`:
    FP32 128 lanes x 2 flops per SM per clock; FP64 2 FMA per SM per clock
    (GB300: 1.25 TFLOP/s nominal at 152 SMs and 2070 MHz)."""
    return sms * 128 * 2 * mhz * 1e6, sms * 2 * 2 * mhz * 1e6


# ALU peaks of the GPU the benchmark runs on (set by set_peaks from its SM
# count and maximum SM clock)
PEAK_FP32 = PEAK_FP64 = None
PEAK_SOURCE = ""


def max_sm_mhz(index: int) -> float:
    """Maximum SM clock of GPU `index` from nvidia-smi, else the driver's
    measured record, else GB300's 2070 MHz."""
    try:
        out = subprocess.run(["nvidia-smi", "-i", str(index), "--query-gpu=clocks.max.sm",
                              "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=20)
        return float(out.stdout.strip().splitlines()[0])
    except Exception:
        pass
    try:
        return float(json.load(open(os.path.join(HERE, "MEASURED_PEAKS.json")))["sm_max_mhz"])
    except Exception:
        return 2070.0


def set_peaks(sms: int, mhz: float):
    global PEAK_FP32, PEAK_FP64, PEAK_SOURCE
    PEAK_FP32, PEAK_FP64 = alu_peaks(sms, mhz)
    PEAK_SOURCE = ("nominal: %d SMs x %.0f MHz (device properties, nvidia-smi); FP32 128 lanes x 2, "
                   "FP64 2 FMA per SM per clock" % (sms, mhz))


def size_classes():
    """The least-squares kernels' size classes, as the library reports them."""
    from paper_2406_17656_gb300 import sam

    return sam.size_classes()


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nx", type=int, default=256)
    ap.add_argument("--maps", type=int, default=10)
    ap.add_argument("--level", type=int, default=2)
    ap.add_argument("--refine", type=int, default=1)
    ap.add_argument("--quick", action="store_true", help="skip the secondary measurements")
    ap.add_argument("--no-tune", action="store_true", help="default tile shapes instead of sam_tune's choice")
    ap.add_argument("--no-configs", action="store_true", help="skip the per-configuration throughput figures")
    ap.add_argument("--profile-gmres", type=int, default=0, metavar="STEPS",
                    help="profiling aid: run one GMRES solve of STEPS Arnoldi steps on the benchmark's last map "
                         "and exit (no JSON line)")
    ap.add_argument("--profile-fem", type=int, default=0, metavar="STEPS",
                    help="profiling aid: run STEPS whole steps (level-2 patterns + batched maps + residuals) of "
                         "the P1 FEM 512x512 sequence and exit (no JSON line)")
    ap.add_argument("--fem-maps", type=int, default=16, help="maps of the --profile-fem sequence")
    ap.add_argument("--profile-sparsify", type=int, default=0, metavar="CALLS",
                    help="profiling aid: run CALLS batched column-tau (0.8) sparsifications of the benchmark's maps "
                         "and exit (no JSON line)")
    ap.add_argument("--profile-build", type=int, default=0, metavar="STEPS",
                    help="profiling aid: run STEPS batched builds of the sequence (--nx, --maps, --level, "
                         "--refine; patterns built once) and print the time per build")
    ap.add_argument("--fp64", action="store_true", help="with --profile-build and --refine 0: the plain FP64 build")
    ap.add_argument("--tape", action="store_true",
                    help="with --profile-adjoint: the build records a factor tape and the adjoints replay it")
    ap.add_argument("--profile-adjoint", type=int, default=0, metavar="STEPS",
                    help="profiling aid: run STEPS adjoints of the benchmark's batched build (dL/dM random, "
                         "residual term on) and exit (no JSON line)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# --------------------------------------------------------------- ranks


def max_over_ranks(x: float, world: int, device="cpu") -> float:
    """The largest x over all ranks (identity on one rank)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank_step: float, world: int, ms_per_step: float) -> float:
    """Whole-job throughput: every rank processes its own copy of the step's
    units (weak scaling), timed by the slowest rank."""
    return units_per_rank_step * world / (ms_per_step * 1e-3)


# --------------------------------------------------------------- accounting


def column_sizes(mats, level):
    """|I_j|, |J_j|, nnz(B_j) of every column from the matrix structures
    (pattern = level-L reachability, shadow = rows reached by A(:, J_j))."""
    import scipy.sparse as sp

    out = []
    for a in mats:
        s = a.to_scipy().copy()
        s.data[:] = 1.0
        s = s.tocsc()
        st = (s + sp.eye(a.n, format="csc")).astype(bool).astype(np.float64)
        pat = sp.eye(a.n, format="csc")
        for _ in range(level):
            pat = (st @ pat).astype(bool).astype(np.float64)
        J = np.diff(pat.indptr)
        I = np.diff((s @ pat).astype(bool).tocsc().indptr)
        colcnt = np.diff(s.indptr).astype(np.float64)
        nB = np.asarray(pat.T @ colcnt).ravel()
        out.append((I.astype(np.int64), J.astype(np.int64), nB.astype(np.int64)))
    return out


def bin_of(I, J, nB, classes=None, schedule=None):
    """Size class that solves every column (the library's rule: the first
    class the column fits, then the handle's bin schedule), -1 where none
    fits."""
    c = classes or size_classes()
    b = np.full(I.shape, -1)
    for q in range(len(c["max_rows"]) - 1, -1, -1):
        ok = ((I <= c["max_rows"][q]) & (J <= c["max_cols"][q]) & (nB <= c["max_entries"][q]) &
              (I * (J + 1) <= c["max_tile"][q]) & (I >= J))
        b[ok] = q
    if schedule is not None:
        to = np.asarray(list(schedule) + [-1])
        b = to[b]
    return b


def algorithmic_flops(I, J, nB, precision, steps):
    """Algorithmic work of one column (m = |I_j|, n = |J_j|, s refinement
    steps): Householder QR with Q^T c and the back-solve,
    2 n^2 (m - n/3) + 4 m n - 2 n^2 + n^2 flops, plus per step an FP32
    correction solve 4 m n - n^2; FP64 per step the residual
    r = c - B m, 2 nnz(B) + m.  The plain FP64 build does the QR part in
    FP64.  Returns (FP32 flops, FP64 flops) per column."""
    m, n = I.astype(np.float64), J.astype(np.float64)
    qr = 2 * n * n * (m - n / 3) + (4 * m * n - 2 * n * n) + n * n
    if precision == "fp64":
        return 0.0 * qr, qr
    f32 = qr + steps * (4 * m * n - n * n)
    f64 = steps * (2 * nB + m)
    return f32, f64


def adjoint_algorithmic_flops(I, J, nB, steps, tape=False):
    """Algorithmic work of the adjoint of one column (m = |I_j|, n = |J_j|,
    b = nnz(B_j), s refinement steps), as the adjoint kernel computes it:
    FP32 the recomputed QR of [B c] (the forward's formula; none when R comes
    from a factor tape) and s + 1 solves with R^T R (2 n^2 each) plus, after
    the last correction, its product B d (2 b); FP64 the residual
    r = c - B m (2 b + m), the products w = B lambda before each correction
    (2 b each, s of them, at least one), B^T w per correction (2 b each),
    the dL/dB entries (3 b: a product and an FMA per entry) and dL/dc (m).
    Returns (FP32, FP64) flops per column."""
    m, n, b = I.astype(np.float64), J.astype(np.float64), nB.astype(np.float64)
    qr = 0.0 if tape else 2 * n * n * (m - n / 3) + (4 * m * n - 2 * n * n) + n * n
    f32 = qr + (steps + 1) * 2 * n * n + (2 * b if steps > 0 else 0.0)
    f64 = (2 * b + m) + max(steps, 1) * 2 * b + steps * 2 * b + 3 * b + m
    return f32, f64


def adjoint_roofline(mats, level, steps, ms, tape=False):
    """Roofline of a whole adjoint call over the maps of `mats`: the slower of
    its algorithmic FP32 flops at the FP32 peak and FP64 flops at the FP64
    peak (adjoint_algorithmic_flops summed over every column), over the
    measured call time."""
    f32 = f64 = 0.0
    seen = {}
    for m in mats:
        key = (m.indptr.tobytes(), m.indices.tobytes())
        if key not in seen:
            I, J, nB = column_sizes([m], level)[0]
            a, b = adjoint_algorithmic_flops(I, J, nB, steps, tape)
            seen[key] = (float(np.sum(a)), float(np.sum(b)))
        f32, f64 = f32 + seen[key][0], f64 + seen[key][1]
    t32, t64 = f32 / PEAK_FP32, f64 / PEAK_FP64
    bound = "fp64" if t64 >= t32 else "fp32"
    t_roof = max(t32, t64)
    ach = (f64 if bound == "fp64" else f32) / (ms * 1e-3)
    return {"bound": "alu (%s pipe)" % bound, "achieved": ach / 1e12,
            "peak": (PEAK_FP64 if bound == "fp64" else PEAK_FP32) / 1e12, "unit": "TFLOP/s",
            "frac": t_roof / (ms * 1e-3), "fp32_flops": f32, "fp64_flops": f64, "ms": ms}


def error_stats(torch, ci, offs, v, vref, n):
    """v against vref (the same map structures, concatenated with offsets
    offs; ci the column index of every entry): the largest whole-map relative
    Frobenius error and the largest per-column relative error over all
    columns of all maps.  Reduced on the device."""
    max_fro = max_col = 0.0
    for k in range(len(offs) - 1):
        a, b = v[offs[k]:offs[k + 1]], vref[offs[k]:offs[k + 1]]
        c = ci[offs[k]:offs[k + 1]].long()
        d = (a - b) ** 2
        max_fro = max(max_fro, float(torch.sqrt(d.sum() / (b * b).sum())))
        d2 = torch.zeros(n, dtype=torch.float64, device=v.device).index_add_(0, c, d)
        w2 = torch.zeros(n, dtype=torch.float64, device=v.device).index_add_(0, c, b * b)
        col = torch.where(w2 > 0, torch.sqrt(d2 / w2.clamp_min(1e-300)), torch.sqrt(d2) * float("inf"))
        col = torch.nan_to_num(col, nan=0.0)
        max_col = max(max_col, float(col.max()))
    return max_fro, max_col


def oracle_column_sample(ak, a0, level, n, ip, ix, v, ncols, seed):
    """Per-column relative errors of the GPU map (CSR ip, ix, v; host) against
    the FP64 oracle on `ncols` sampled columns (plus the first and last):
    (max per-column error, relative Frobenius error over the sample)."""
    import scipy.sparse as sp

    import oracle

    cp, ri = oracle.pattern(ak, level)
    rng = np.random.default_rng(seed)
    cols = np.unique(np.concatenate([rng.choice(n, ncols, replace=False), [0, n - 1]])).astype(np.int32)
    ref = oracle.build_cols(ak, a0, cp, ri, cols)
    m = sp.csr_matrix((v, ix, ip), shape=(n, n)).tocsc()
    m.sort_indices()
    errs, num, den = [], 0.0, 0.0
    for j in cols:
        a, b = m.data[cp[j]:cp[j + 1]], ref["mval"][cp[j]:cp[j + 1]]
        d2, w2 = float(np.sum((a - b) ** 2)), float(np.sum(b * b))
        errs.append(np.sqrt(d2 / w2) if w2 > 0 else (0.0 if d2 == 0 else float("inf")))
        num, den = num + d2, den + w2
    return float(max(errs)), float(np.sqrt(num / den)), len(cols)


def measured_hbm_gbs() -> float:
    """Measured copy bandwidth of the GB300s, else the fallback figure."""
    try:
        return float(json.load(open(os.path.join(HERE, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except Exception:
        return 6800.0


def _code_only(src: bytes) -> bytes:
    """C++ source without its comments and blank lines (string literals kept)."""
    import re

    pat = re.compile(rb'"(?:\\.|[^"\\\n])*"|//[^\n]*|/\*.*?\*/', re.S)
    out = pat.sub(lambda m: m.group(0) if m.group(0).startswith(b'"') else b"", src)
    return b"\n".join(line.rstrip() for line in out.split(b"\n") if line.strip())


def kernel_hash() -> str:
    """sha256 over the code the least-squares kernel is compiled from: its
    kernel header, its translation unit, the shared column routines and the
    device part of common.cuh (constants, LsqArgs, device helpers; the
    host-side declarations after them do not enter the kernel), comments and
    blank lines left out.  A recorded ncu traffic figure is only reported
    while this code is unchanged."""
    import hashlib

    csrc = os.path.join(HERE, "paper_2406_17656_gb300", "csrc")
    h = hashlib.sha256()
    for f in ("lsq_kernel.cuh", "lsq.cu", "lsq_core.cuh"):
        h.update(_code_only(open(os.path.join(csrc, f), "rb").read()))
    common = open(os.path.join(csrc, "common.cuh"), "rb").read()
    cut = common.find(b"// ------------------------------------------------------- host-side helpers")
    h.update(_code_only(common if cut < 0 else common[:cut]))
    return h.hexdigest()


# ------------------------------------------------------------------ clocks


class ClockSampler:
    def __init__(self, index):
        self.index, self.proc, self.path = index, None, None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.path = "/tmp/sam_clocks_%d.csv" % os.getpid()
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc or not self.path or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], [], set()
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"),
                               f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        load = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# -------------------------------------------------------------- reference


def run_reference(args, rank):
    """The FP64 CPU oracle as the reference arm (rank 0 only)."""
    import oracle
    from paper_2406_17656_gb300 import workloads as W

    if rank != 0:
        return
    seq = W.config2(nx=args.nx, nmat=args.maps, level=args.level)
    a0 = seq.mats[0]
    cores = oracle.max_threads()
    times = []

    def step(k):
        ak = seq.mats[k % len(seq.mats)]
        t = time.perf_counter()
        cp, ri = oracle.pattern(ak, args.level)
        oracle.build(ak, a0, cp, ri, nthreads=cores)
        return time.perf_counter() - t

    for w in range(args.warmup):
        step(w)
    for s in range(args.steps):
        times.append(step(s))
    per = float(np.mean(times))
    value = a0.n / per
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": seq.name + "_seq%d_level%d" % (args.maps, args.level), "n": a0.n,
                       "maps": args.maps, "level": args.level},
            "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "each step: one map (all %d columns) of the sequence, pattern + build" % a0.n},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(seq, level, budget_s=12.0):
    """Times the FP64 oracle (as it stands) on whole maps until the budget."""
    import oracle

    cores = oracle.max_threads()
    a0 = seq.mats[0]
    # one map on one core first: the all-core calls below set the oracle's
    # (process-wide) OpenMP thread count back
    ak = seq.mats[-1]
    t = time.perf_counter()
    cp, ri = oracle.pattern(ak, level)
    oracle.build(ak, a0, cp, ri, nthreads=1)
    t1 = time.perf_counter() - t
    # whole maps in sequence order, passing over the sequence again until the
    # budget is spent
    cols, t_tot, maps = 0, 0.0, 0
    while t_tot < budget_s:
        for ak in seq.mats:
            t = time.perf_counter()
            cp, ri = oracle.pattern(ak, level)
            oracle.build(ak, a0, cp, ri, nthreads=cores)
            t_tot += time.perf_counter() - t
            cols += ak.n
            maps += 1
            if t_tot >= budget_s:
                break
    return {"value": cols / t_tot, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d maps (%.1f passes over the %d-map sequence), all columns, pattern + build, "
                      "%d OpenMP threads, %.1f s" % (maps, maps / len(seq.mats), len(seq.mats), cores, t_tot),
            "one_core_value": seq.mats[-1].n / t1, "one_core_sample": "1 map, all columns, pattern + build, 1 thread, %.1f s" % t1}, \
        seq.mats[:maps]


# ------------------------------------------------------------------ krylov


def krylov_bytes(n, nnz_ops, nnz_a, restart, its):
    """Algorithmic bytes of `its` Arnoldi steps of GMRES(restart): per step,
    each CSR product reads its values and column indices (12 B per entry),
    its row pointers and the input vector and writes the output vector; the
    Gram-Schmidt step j reads the j+1 basis vectors twice (projection and
    update) and reads/writes w; per cycle, the update reads the k basis
    vectors and x, the products of the preconditioner run once more, and
    b - A x and its norm read A, x and b."""
    def prod(nnz):
        return 12.0 * nnz + 4.0 * (n + 1) + 16.0 * n

    step_ops = sum(prod(z) for z in nnz_ops) + prod(nnz_a)
    total, done = 0.0, 0
    while done < its:
        k = min(restart, its - done)
        total += k * step_ops + sum(8.0 * n * (2 * (j + 1) + 3) for j in range(k))
        total += 8.0 * n * (k + 2) + sum(prod(z) for z in nnz_ops) + prod(nnz_a) + 16.0 * n
        done += k
    return total


def krylov_flops(n, nnz_ops, nnz_a, restart, its):
    """Algorithmic FP64 flops of `its` Arnoldi steps of GMRES(restart) with
    one Gram-Schmidt sweep (the textbook algorithm): per step 2 nnz for
    each CSR product, 4 n (j+1) for the projections and the update, 3 n
    for the norm and the scaling; per cycle the update 2 n k, the
    preconditioner products, b - A x and its norm."""
    step_ops = 2.0 * (sum(nnz_ops) + nnz_a)
    total, done = 0.0, 0
    while done < its:
        k = min(restart, its - done)
        total += k * (step_ops + 3.0 * n) + sum(4.0 * n * (j + 1) for j in range(k))
        total += 2.0 * n * k + 2.0 * sum(nnz_ops) + 2.0 * nnz_a + 3.0 * n
        done += k
    return total


def krylov_measurement(h, sam, torch, dev, stream, aks, a0, offs, mrp, mci, mval, n, K, world, rank):
    k = K - 1
    ident = sam.Csr(torch.arange(n + 1, dtype=torch.int32, device=dev), torch.arange(n, dtype=torch.int32, device=dev),
                    torch.ones(n, dtype=torch.float64, device=dev), n=n)
    p2 = h.sam_pattern_build(a0, 2)
    P = sam.Csr(*h.sam_build(a0, ident, p2, "fp64"), n=n)
    p2.destroy()
    M = sam.Csr(mrp[k * (n + 1):(k + 1) * (n + 1)].contiguous(), mci[offs[k]:offs[k + 1]],
                mval[offs[k]:offs[k + 1]], n=n)
    A = aks[k]
    b = torch.from_numpy(np.random.default_rng(9).standard_normal(n)).to(dev)
    kw = dict(restart=30, maxiter=5000, rtol=1e-8)
    res = {}
    for name, MM in (("p0", None), ("map", M)):
        h.sam_gmres(A, b, M=MM, P_0=P, **kw)  # warm-up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        x, its, rel = h.sam_gmres(A, b, M=MM, P_0=P, **kw)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        r = b - h.sam_apply(A, x)
        res[name] = (its, rel, float(torch.linalg.norm(r) / torch.linalg.norm(b)), ms)
    its, rel, true_rel, ms = res["map"]
    ms = max_over_ranks(ms, world, dev)
    moved = krylov_bytes(n, (P.nnz, M.nnz), A.nnz, kw["restart"], its)
    gbs = moved / (ms * 1e-3) / 1e9
    flops = krylov_flops(n, (P.nnz, M.nnz), A.nnz, kw["restart"], its)
    out = {"gmres": {"workload": "A_%d x = b, n = %d, GMRES(%d), rtol %g, right preconditioner M_%d (P_0 v), "
                                 "P_0 = level-2 SPAI of A_0" % (k, n, kw["restart"], kw["rtol"], k),
                     "steps_with_map": its, "steps_p0_only": res["p0"][0], "relres_estimate": rel,
                     "true_relres": true_rel, "ms": ms, "us_per_step": ms * 1e3 / max(its, 1),
                     "steps_per_s": job_value(its, world, ms), "ms_p0_only": res["p0"][3],
                     "roofline": {"bound": "alu", "unit": "TFLOP/s", "achieved": flops / (ms * 1e-3) / 1e12,
                                  "peak": PEAK_FP64 / 1e12, "frac": flops / (ms * 1e-3) / PEAK_FP64,
                                  "fp64_flops": flops,
                                  "note": "FP64-instruction bound on GB300 (FP64 at 1/64 of FP32); the "
                                          "working set is L2-resident"},
                     "algorithmic_bytes": moved, "achieved_gbs": gbs, "hbm_frac": gbs / measured_hbm_gbs(),
                     "working_set_mb": (12.0 * (A.nnz + M.nnz + P.nnz) + 8.0 * n * (kw["restart"] + 6)) / 1e6}}
    # the whole sequence: A_k x = b for k = 1..K-1, each with its map M_k, solved
    # together in one batched call and one by one
    Ms = [sam.Csr(mrp[q * (n + 1):(q + 1) * (n + 1)].contiguous(), mci[offs[q]:offs[q + 1]], mval[offs[q]:offs[q + 1]],
                  n=n) for q in range(1, K)]
    As = aks[1:K]
    bb = b.repeat(K - 1)
    h.sam_gmres_batched(As, bb, Ms=Ms, P_0=P, **kw)  # warm-up
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    _, its_b, _ = h.sam_gmres_batched(As, bb, Ms=Ms, P_0=P, **kw)
    e1.record(stream)
    e1.synchronize()
    ms_batched = e0.elapsed_time(e1)
    ms_single, its_single = 0.0, []
    for A_q, M_q in zip(As, Ms):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, its_q, _ = h.sam_gmres(A_q, b, M=M_q, P_0=P, **kw)
        e1.record(stream)
        e1.synchronize()
        ms_single += e0.elapsed_time(e1)
        its_single.append(its_q)
    out["gmres"]["sequence"] = {"systems": K - 1, "steps": [int(v) for v in its_b],
                                "steps_equal_single_solves": [int(v) for v in its_b] == its_single,
                                "batched_ms": ms_batched, "one_by_one_ms": ms_single,
                                "speedup": ms_single / ms_batched}
    if rank == 0 and world == 1:
        # the oracle's textbook GMRES on the same system, 60 steps (two cycles)
        import oracle

        from paper_2406_17656_gb300 import workloads as W

        host = lambda c: W.CSR(n, c.indptr.cpu().numpy(), c.indices.cpu().numpy(), c.data.cpu().numpy())
        t = time.perf_counter()
        oracle.gmres(host(A), b.cpu().numpy(), M=host(M), P0=host(P), restart=30, maxiter=60, rtol=1e-30)
        out["gmres"]["oracle_us_per_step"] = (time.perf_counter() - t) * 1e6 / 60
    return out


def profile_gmres(h, sam, torch, dev, aks, a0, n, level, steps):
    """One GMRES solve of `steps` Arnoldi steps on the last map of the
    sequence (the system of the benchmark's Krylov figure), for ncu."""
    ident = sam.Csr(torch.arange(n + 1, dtype=torch.int32, device=dev), torch.arange(n, dtype=torch.int32, device=dev),
                    torch.ones(n, dtype=torch.float64, device=dev), n=n)
    p2 = h.sam_pattern_build(a0, 2)
    P = sam.Csr(*h.sam_build(a0, ident, p2, "fp64"), n=n)
    sk = h.sam_pattern_build(aks[-1], level)
    M = sam.Csr(*h.sam_build(aks[-1], a0, sk, "fp32r", 1), n=n)
    b = torch.from_numpy(np.random.default_rng(9).standard_normal(n)).to(dev)
    torch.cuda.synchronize()
    t = time.perf_counter()
    _, its, rel = h.sam_gmres(aks[-1], b, M=M, P_0=P, restart=30, maxiter=steps, rtol=1e-30)
    torch.cuda.synchronize()
    print("gmres: %d steps, estimate %.3e, %.1f us per step" % (its, rel, (time.perf_counter() - t) * 1e6 / its))


def profile_fem(h, sam, torch, dev, steps, nmat=16):
    """`steps` whole steps of the P1 FEM sequence whose pattern changes from
    map to map (the workload of the configuration figures), for ncu."""
    from paper_2406_17656_gb300 import workloads as W

    seq = W.config4(nmat=nmat)
    aks = [sam.Csr.from_host(m, dev) for m in seq.mats]
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(steps):
        ps = h.sam_pattern_build_batched(aks, 2)
        h.sam_build_batched(aks, aks[0], ps, "fp32r", 1, want_fro=True)
        for p in ps:
            p.destroy()
    torch.cuda.synchronize()
    print("fem: %d steps, %.2f ms per step" % (steps, (time.perf_counter() - t) * 1e3 / steps))


# ------------------------------------------------------------ all configs


def config_figures(h, sam, torch, dev, stream, nsteps=7):
    """Throughput of the whole path (level-L patterns + batched maps, with
    the per-map residuals) on the other synthetic workloads: CUDA events
    around each step, median of `nsteps` after one warm-up.  Returns a dict
    keyed by workload."""
    from paper_2406_17656_gb300 import workloads as W

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        ms = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return statistics.median(ms)

    size_cache = {}

    def step_roofline(mats, level, precision, steps, ms):
        """Whole-step roofline: the slowest of the algorithmic FP32 flops at the
        FP32 peak, the FP64 flops at the FP64 peak and the gathered bytes at
        the measured HBM bandwidth, over the measured step time (column sizes
        from the structures, computed once per distinct structure)."""
        f32 = f64 = gathered = 0.0
        for m in mats:
            key = (m.indptr.tobytes(), m.indices.tobytes())
            if key not in size_cache:
                I, J, nB = column_sizes([m], level)[0]
                a, b = algorithmic_flops(I, J, nB, precision, steps)
                size_cache[key] = (float(np.sum(a)), float(np.sum(b)), 12.0 * float(np.sum(nB)))
            a, b, g = size_cache[key]
            f32, f64, gathered = f32 + a, f64 + b, gathered + g
        t_roof = max(f32 / PEAK_FP32, f64 / PEAK_FP64, gathered / (measured_hbm_gbs() * 1e9))
        return {"roofline_frac": t_roof / (ms * 1e-3), "fp32_flops": f32, "fp64_flops": f64,
                "gathered_bytes": gathered}

    import oracle

    cores = oracle.max_threads()

    def oracle_rate(ak, a0, level):
        """The FP64 oracle on one map of the workload, all host cores, repeated
        until a quarter of a second has been timed."""
        reps, dt = 0, 0.0
        while dt < 0.25:
            t = time.perf_counter()
            cp, ri = oracle.pattern(ak, level)
            oracle.build(ak, a0, cp, ri, nthreads=cores)
            dt += time.perf_counter() - t
            reps += 1
        return {"oracle_columns_per_s": reps * ak.n / dt, "oracle_cores": cores,
                "oracle_sample": "1 map x %d, all columns, pattern + build, %.2f s" % (reps, dt)}

    def line(name, cols, maps, ms, extra=None, roof=None, orc=None):
        d = {"columns_per_s": cols / (ms * 1e-3), "maps_per_s": maps / (ms * 1e-3), "ms_per_step": ms,
             "columns_per_step": cols, "maps": maps}
        if roof is not None:
            d.update(step_roofline(*roof, ms))
        if orc is not None:
            d.update(oracle_rate(*orc))
        d.update(extra or {})
        out[name] = d

    out = {}
    saved_variants = h.sam_get_tile_variants()
    saved_schedule = h.sam_get_bin_schedule()

    def tune(aks, a0, level, steps):
        """sam_tune on this workload's own patterns (the tile shape per size
        class is the handle's; restored when all configurations are done)."""
        ps = h.sam_pattern_build_batched(aks, level)
        v = h.sam_tune(aks, a0, ps, "fp32r", steps)
        for p in ps:
            p.destroy()
        return {"tile_variants": list(v), "bin_schedule": h.sam_get_bin_schedule()}

    # config 1: 5-point Poisson 32^2, A_1 = A_0 + diag, level 1, plain FP64 single build
    seq = W.config1()
    aks = [sam.Csr.from_host(m, dev) for m in seq.mats]

    def c1():
        ps = h.sam_pattern_build_batched(aks, 1)
        h.sam_build_batched(aks, aks[0], ps, "fp64", 0, want_fro=True)
        for p in ps:
            p.destroy()

    ms1 = timed(c1, nsteps)
    # the same numeric build replayed from a captured graph (patterns fixed):
    # launch-bound at this size, where a graph pays most
    ps = h.sam_pattern_build_batched(aks, 1)
    plan = h.sam_plan_create(aks, aks[0], ps, "fp64", 0)
    for p in ps:
        p.destroy()
    msp1 = timed(plan.execute, nsteps)
    plan.destroy()
    line("poisson5_32x32_seq2_level1_fp64", 2 * aks[0].n, 2, ms1,
         {"graph_replay_columns_per_s": 2 * aks[0].n / (msp1 * 1e-3), "graph_replay_ms": msp1},
         roof=(seq.mats, 1, "fp64", 0), orc=(seq.mats[1], seq.mats[0], 1))
    def build_step(aks, tgt, level, precision, steps):
        """One step of the path: level-L patterns of every A_k and the batched
        maps with the per-map residuals."""
        def fn():
            ps = h.sam_pattern_build_batched(aks, level)
            h.sam_build_batched(aks, tgt, ps, precision, steps, want_fro=True)
            for p in ps:
                p.destroy()
        return fn

    def accuracy(aks, tgt, level, steps, n, ms32, host_pair, nsample=300, seed=0):
        """The plain FP64 GPU build of the same maps (step time, speed-up of FP32
        + refinement over it) and the FP32 + refinement maps' errors against it
        (largest whole-map relative Frobenius error and largest per-column
        relative error, all maps) and against the FP64 oracle (sampled columns
        of the last map); the guard's outcome counts."""
        ps = h.sam_pattern_build_batched(aks, level)
        offs, rp, ci, v32, _ = h.sam_build_batched(aks, tgt, ps, "fp32r", steps)
        one, two, fp64 = h.sam_refine_stats()
        _, _, _, v64, _ = h.sam_build_batched(aks, tgt, ps, "fp64", 0, offsets=offs)
        for p in ps:
            p.destroy()
        fro, col = error_stats(torch, ci, offs, v32, v64, n)
        k = len(aks) - 1
        ak_h, a0_h = host_pair
        ocol, ofro, ncols = oracle_column_sample(ak_h, a0_h, level, n, rp[k * (n + 1):(k + 1) * (n + 1)].cpu().numpy(),
                                                 ci[offs[k]:offs[k + 1]].cpu().numpy(),
                                                 v32[offs[k]:offs[k + 1]].cpu().numpy(), nsample, seed)
        del v32, v64, rp, ci
        ms64 = timed(build_step(aks, tgt, level, "fp64", 0), 3)
        return {"fp64_ms_per_step": ms64, "fp64_columns_per_s": len(aks) * n / (ms64 * 1e-3),
                "speedup_fp32r_vs_fp64": ms64 / ms32, "max_rel_fro_vs_fp64_gpu": fro,
                "max_col_rel_err_vs_fp64_gpu": col, "sample_max_col_rel_err_vs_oracle": ocol,
                "sample_rel_fro_vs_oracle": ofro, "oracle_sample_columns": ncols,
                "refine_outcomes": {"one_step": one, "two_steps": two, "fp64_solved": fp64}}

    def plan_replay(aks, tgt, level, steps, nt):
        """The numeric rebuild replayed from its captured CUDA graph
        (patterns fixed; every replay re-reads the values)."""
        ps = h.sam_pattern_build_batched(aks, level)
        plan = h.sam_plan_create(aks, tgt, ps, "fp32r", steps)
        for p in ps:
            p.destroy()
        ms = timed(plan.execute, nsteps)
        launches = plan.launches()
        plan.destroy()
        return {"graph_replay_columns_per_s": nt / (ms * 1e-3), "graph_replay_ms": ms,
                "graph_replay_launches": launches}

    # config 3: 7-point upwind 64^3, 20 maps, level 2, FP32 QR + 1 FP64 step
    seq = W.config3()
    aks = [sam.Csr.from_host(m, dev) for m in seq.mats]
    n3 = aks[0].n
    tv = tune(aks, aks[0], 2, 1)
    ms3 = timed(build_step(aks, aks[0], 2, "fp32r", 1), nsteps)
    ms3a = timed(build_step(aks, aks[0], 2, "fp32r", "auto"), nsteps)
    ex = {**tv, "auto_columns_per_s": len(aks) * n3 / (ms3a * 1e-3), "auto_ms_per_step": ms3a}
    ex.update(plan_replay(aks, aks[0], 2, 1, len(aks) * n3))
    ex.update(accuracy(aks, aks[0], 2, 1, n3, ms3, (seq.mats[-1], seq.mats[0]), seed=3))
    line("upwind7_64cube_seq20_level2", len(aks) * n3, len(aks), ms3, ex, roof=(seq.mats, 2, "fp32r", 1),
         orc=(seq.mats[-1], seq.mats[0], 2))
    del aks
    torch.cuda.empty_cache()
    # config 4: P1 FEM 512^2 cells, 16 maps whose pattern changes, level 2; direct and captured plan
    seq = W.config4()
    aks = [sam.Csr.from_host(m, dev) for m in seq.mats]
    n4 = aks[0].n
    tv = tune(aks, aks[0], 2, 1)
    ms4 = timed(build_step(aks, aks[0], 2, "fp32r", 1), nsteps)
    cols4 = len(aks) * n4
    ex = {**tv, **plan_replay(aks, aks[0], 2, 1, cols4)}
    ex.update(accuracy(aks, aks[0], 2, 1, n4, ms4, (seq.mats[-1], seq.mats[0]), seed=4))
    line("p1_fem_512x512_seq16_level2", cols4, len(aks), ms4, ex, roof=(seq.mats, 2, "fp32r", 1),
         orc=(seq.mats[-1], seq.mats[0], 2))
    del aks
    torch.cuda.empty_cache()
    # config 5: 32 independent (A_0, A_1) 512^2 pairs, level 1, forward (one target per map) and adjoint
    pairs = [W.config5_pair(b) for b in range(32)]
    a0s = [sam.Csr.from_host(p[0], dev) for p in pairs]
    a1s = [sam.Csr.from_host(p[1], dev) for p in pairs]
    n5 = a0s[0].n
    tv = tune(a1s, a0s[0], 1, 2)
    ms5 = timed(build_step(a1s, a0s, 1, "fp32r", 2), nsteps)
    ps = h.sam_pattern_build_batched(a1s, 1)
    offs, _, _, mv, _ = h.sam_build_batched(a1s, a0s, ps, "fp32r", 2)
    gbar = torch.randn(mv.numel(), dtype=torch.float64, device=dev, generator=torch.Generator(device=dev).manual_seed(5))
    msb_re = timed(lambda: h.sam_build_backward_batched(a1s, a0s, ps, mv, gbar, "fp32r", 2, 1.0, offsets=offs), nsteps)
    tape = torch.empty((h.sam_factor_tape_bytes(ps, "fp32r") + 15) // 16 * 2, dtype=torch.float64, device=dev)
    h.sam_set_factor_tape(sam.SAM_TAPE_RECORD, tape)
    h.sam_build_batched(a1s, a0s, ps, "fp32r", 2, M_val=mv)
    h.sam_set_factor_tape(sam.SAM_TAPE_REPLAY, tape)
    msb = timed(lambda: h.sam_build_backward_batched(a1s, a0s, ps, mv, gbar, "fp32r", 2, 1.0, offsets=offs), nsteps)
    h.sam_set_factor_tape(sam.SAM_TAPE_OFF)
    for p in ps:
        p.destroy()
    del mv, gbar, tape
    ex = {"adjoint_columns_per_s": 32 * n5 / (msb_re * 1e-3), "adjoint_ms": msb_re, "adjoint_tape_ms": msb,
          "refine_steps": 2, **tv}
    ex["adjoint_roofline"] = adjoint_roofline([p[1] for p in pairs], 1, 2, msb_re)
    ex.update(plan_replay(a1s, a0s, 1, 2, 32 * n5))
    ex.update(accuracy(a1s, a0s, 1, 2, n5, ms5, (pairs[-1][1], pairs[-1][0]), seed=5))
    line("q1_pairs_512x512_x32_level1", 32 * n5, 32, ms5, ex,
         roof=([p[1] for p in pairs], 1, "fp32r", 2), orc=(pairs[0][1], pairs[0][0], 1))
    # level-3 maps (the paper's "level 2", Sec. 5.1) of the benchmark's Q1 sequence, 2 maps: interior
    # columns of 81 x 49 go to the large size class (one thread block per column, FP32 tile in shared
    # memory + one guarded FP64 step; the FP64 arm solves them with an FP64 tile)
    seq = W.config2(nmat=2)
    aks = [sam.Csr.from_host(m, dev) for m in seq.mats]
    nq = aks[0].n
    h.sam_set_tile_variants([0] * 6)
    h.sam_set_bin_schedule(list(range(6)))
    msq = timed(build_step(aks, aks[0], 3, "fp32r", 1), 3)
    ex = accuracy(aks, aks[0], 3, 1, nq, msq, (seq.mats[-1], seq.mats[0]), nsample=60, seed=6)
    ex["note"] = "interior columns (81 x 49) are solved by the large size class (a thread block per column)"
    line("q1_diffusion_256x256_seq2_level3", len(aks) * nq, len(aks), msq, ex, roof=(seq.mats, 3, "fp32r", 1))
    del aks
    torch.cuda.empty_cache()
    h.sam_set_tile_variants(saved_variants)
    h.sam_set_bin_schedule(saved_schedule)
    return out


# ------------------------------------------------------------ CD2D study


def cd2d_study(h, sam, torch, dev, stream):
    """The paper's comparison (Sec. 5.1, Figs. 3-4, Tables 1-2) on the CD2D
    stand-in, through the GPU path: for each pattern choice -- S(A_0), and
    the square / cube of S(A~_k) for the column threshold and lfil
    sparsifications -- all 66 maps N_k onto A_0 in one batched build, with
    the pattern sizes and the relative residual ||A_k N_k - A_0||_F / ||A_0||_F
    per map (min / mean / max over the sequence)."""
    from paper_2406_17656_gb300 import workloads as W

    seq = W.cd2d()
    aks = [sam.Csr.from_host(m, dev) for m in seq.mats]
    a0 = aks[0]
    K = len(aks)
    nrm0 = float(np.linalg.norm(seq.mats[0].data))
    choices = [("S(A_0)", None, None, 1), ("tau 0.6, square", "tau", 0.6, 2), ("tau 0.7, square", "tau", 0.7, 2),
               ("tau 0.8, square", "tau", 0.8, 2), ("lfil 3, square", "lfil", 3, 2), ("lfil 5, square", "lfil", 5, 2),
               ("tau 0.8, cube", "tau", 0.8, 3), ("lfil 5, cube", "lfil", 5, 3)]
    out = {"workload": "cd2d_64x64_seq66 (Newton-with-line-search Jacobians, n = 4096)", "maps": K}
    torch.cuda.synchronize()
    for name, mode, param, power in choices:
        t0 = time.perf_counter()
        if mode is None:
            pats = [h.sam_pattern_build(a0, power)] * K
        else:
            pats = h.sam_pattern_build_batched(h.sam_sparsify_batched(aks, mode, param), power)
        _, _, _, _, fro = h.sam_build_batched(aks, a0, pats, "fp32r", 1, want_fro=True)
        torch.cuda.synchronize()
        rel = np.asarray(fro) / nrm0
        out[name] = {"nnz_per_map": sorted({int(p.nnz) for p in pats}), "rel_residual_min": float(rel[1:].min()),
                     "rel_residual_mean": float(rel[1:].mean()), "rel_residual_max": float(rel[1:].max()),
                     "ms": (time.perf_counter() - t0) * 1e3}
        for p in set(pats):
            p.destroy()
    return out


# ------------------------------------------------------------------- ours


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank)
        return
    import torch

    from paper_2406_17656_gb300 import build as _build
    from paper_2406_17656_gb300 import sam
    from paper_2406_17656_gb300 import workloads as W

    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    if rank == 0:
        _build.build()
    if world > 1:
        dist.barrier()
    sam.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    set_peaks(torch.cuda.get_device_properties(dev).multi_processor_count, max_sm_mhz(local))
    if args.profile_fem > 0:
        h = sam.Handle(stream=torch.cuda.current_stream())
        profile_fem(h, sam, torch, dev, args.profile_fem, args.fem_maps)
        h.close()
        return

    seq = W.config2(nx=args.nx, nmat=args.maps, level=args.level)
    a0h = seq.mats[0]
    n, K = a0h.n, len(seq.mats)
    stream = torch.cuda.current_stream()
    h = sam.Handle(stream=stream)
    aks = [sam.Csr.from_host(m, dev) for m in seq.mats]
    a0 = sam.Csr.from_host(a0h, dev)
    if args.profile_gmres > 0:
        profile_gmres(h, sam, torch, dev, aks, a0, n, args.level, args.profile_gmres)
        h.close()
        return
    if args.profile_build > 0:
        pats = h.sam_pattern_build_batched(aks, args.level)
        prec = "fp64" if args.refine == 0 and args.fp64 else "fp32r"
        out = h.sam_build_batched(aks, a0, pats, prec, args.refine)
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(args.profile_build):
            h.sam_build_batched(aks, a0, pats, prec, args.refine, M_val=out[3])
        torch.cuda.synchronize()
        print("build: %d batched builds of %d maps, level %d, %s, %.3f ms per build" % (
            args.profile_build, K, args.level, prec, (time.perf_counter() - t) * 1e3 / args.profile_build))
        h.close()
        return
    if args.profile_sparsify > 0:
        for _ in range(2):
            h.sam_sparsify_batched(aks, "tau", 0.8)
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(args.profile_sparsify):
            h.sam_sparsify_batched(aks, "tau", 0.8)
        torch.cuda.synchronize()
        print("sparsify: %d batched calls, %.3f ms per call (%d maps)" % (
            args.profile_sparsify, (time.perf_counter() - t) * 1e3 / args.profile_sparsify, K))
        h.close()
        return
    if args.profile_adjoint > 0:
        pats = h.sam_pattern_build_batched(aks, args.level)
        tape = None
        if args.tape:
            tape = torch.empty((h.sam_factor_tape_bytes(pats, "fp32r") + 15) // 16 * 2, dtype=torch.float64,
                               device=dev)
            h.sam_set_factor_tape(sam.SAM_TAPE_RECORD, tape)
        offs_a, _, _, mv, _ = h.sam_build_batched(aks, a0, pats, "fp32r", args.refine)
        if tape is not None:
            h.sam_set_factor_tape(sam.SAM_TAPE_REPLAY, tape)
        gbar = torch.randn(mv.numel(), dtype=torch.float64, device=dev,
                           generator=torch.Generator(device=dev).manual_seed(3))
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(args.profile_adjoint):
            h.sam_build_backward_batched(aks, [a0] * K, pats, mv, gbar, "fp32r", args.refine, 1.0, offsets=offs_a)
        torch.cuda.synchronize()
        print("adjoint: %d steps, %.2f ms per step" % (args.profile_adjoint,
                                                      (time.perf_counter() - t) * 1e3 / args.profile_adjoint))
        h.close()
        return
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def make_outputs(level):
        pats = h.sam_pattern_build_batched(aks, level)
        offs = np.zeros(K + 1, np.int64)
        offs[1:] = np.cumsum([p.nnz for p in pats])
        out = (torch.empty(K * (n + 1), dtype=torch.int32, device=dev),
               torch.empty(int(offs[-1]), dtype=torch.int32, device=dev),
               torch.empty(int(offs[-1]), dtype=torch.float64, device=dev))
        for p in pats:
            p.destroy()
        return offs, out

    def step(level, precision, steps, offs, out):
        pats = h.sam_pattern_build_batched(aks, level)
        res = h.sam_build_batched(aks, a0, pats, precision, steps, M_row_ptr=out[0], M_col_idx=out[1],
                                  M_val=out[2], want_fro=True, offsets=offs)
        for p in pats:
            p.destroy()
        return res[4]

    def timed(level, precision, steps, nsteps, nwarm, profile=False):
        offs, out = make_outputs(level)
        for _ in range(nwarm):
            step(level, precision, steps, offs, out)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        if profile:
            h.sam_profile(True)
        ms = 0.0
        fro = None
        for _ in range(nsteps):
            flush.zero_()  # evict L2 between steps (outside the timed interval)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fro = step(level, precision, steps, offs, out)
            e1.record(stream)
            e1.synchronize()
            ms += e0.elapsed_time(e1)
        torch.cuda.synchronize()
        prof = h.sam_profile_read() if profile else None
        if profile:
            h.sam_profile(False)
        if world > 1:
            dist.barrier()
        return max_over_ranks(ms, world, dev) / nsteps, fro, prof, (offs, out)

    # ---- one-time tuning of the FP32 tile shapes on this workload (untimed)
    variants = [0] * sam.SAM_NUM_SIZE_CLASSES
    if not args.no_tune:
        pats = h.sam_pattern_build_batched(aks, args.level)
        variants = h.sam_tune(aks, a0, pats, "fp32r", args.refine)
        for p in pats:
            p.destroy()

    # ---- headline: FP32 QR + FP64 refinement, level 2
    with ClockSampler(local) as clk:
        ms, fro, prof, (offs, out) = timed(args.level, "fp32r", args.refine, args.steps, args.warmup, profile=True)
    clocks = clk.summary()
    cols_per_step = K * n
    value = job_value(cols_per_step, world, ms)
    launches_total, lsq_ms, lsq_n = prof
    gpu_launches = int(launches_total)

    extra = {}
    # the refinement guard's outcomes on the headline build (columns that kept
    # their solution after one step, re-solved in FP64)
    one, two, fp64c = h.sam_refine_stats()
    extra["refine_outcomes"] = {"one_step": one, "two_steps": two, "fp64_solved": fp64c}
    # accuracy: FP32+refine against the FP64 GPU build (all columns) and the oracle (a sample, below)
    v32 = out[2].clone()
    if not args.quick:
        ms64, fro64, _, (offs64, out64) = timed(args.level, "fp64", 0, max(2, args.steps // 3), 1)
        extra["fp64_columns_per_s"] = job_value(cols_per_step, world, ms64)
        extra["fp64_ms_per_step"] = ms64
        extra["speedup_fp32r_vs_fp64"] = value / extra["fp64_columns_per_s"]
        fro_e, col_e = error_stats(torch, out[1], offs, v32, out64[2], n)
        extra["max_rel_fro_vs_fp64_gpu"] = fro_e
        extra["max_col_rel_err_vs_fp64_gpu"] = col_e
        del out64
        # the automatic refinement mode on the same workload
        msa, _, _, _ = timed(args.level, "fp32r", "auto", max(2, args.steps // 2), 1)
        extra["auto_columns_per_s"] = job_value(cols_per_step, world, msa)
        extra["auto_ms_per_step"] = msa
        a1, a2, a3 = h.sam_refine_stats()
        extra["auto_refine_outcomes"] = {"one_step": a1, "two_steps": a2, "fp64_solved": a3}
        ms1, _, _, _ = timed(1, "fp32r", args.refine, max(2, args.steps // 2), 1)
        extra["level1_columns_per_s"] = job_value(cols_per_step, world, ms1)
        extra["rel_residual_per_map"] = [float(f) / float(np.linalg.norm(a0h.data)) for f in fro]

    # ---- numeric rebuild replayed from a captured CUDA graph (patterns fixed,
    #      values re-read from the same device buffers every replay)
    if not args.quick:
        pats = h.sam_pattern_build_batched(aks, args.level)
        plan = h.sam_plan_create(aks, a0, pats, "fp32r", args.refine)
        for p in pats:
            p.destroy()
        for _ in range(3):
            plan.execute()
        torch.cuda.synchronize()
        tg = 0.0
        ng = max(5, args.steps)
        for _ in range(ng):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            plan.execute()
            e1.record(stream)
            e1.synchronize()
            tg += e0.elapsed_time(e1)
        tg = max_over_ranks(tg / ng, world, dev)
        extra["graph_replay_columns_per_s"] = job_value(cols_per_step, world, tg)
        extra["graph_replay_ms"] = tg
        extra["graph_replay_launches"] = plan.launches()
        plan.destroy()

    # ---- adjoint of the same batched build (dL/dM random, residual term on)
    if not args.quick:
        pats = h.sam_pattern_build_batched(aks, args.level)
        offs_a, _, _, mv, _ = h.sam_build_batched(aks, a0, pats, "fp32r", args.refine)
        gbar = torch.randn(mv.numel(), dtype=torch.float64, device=dev,
                           generator=torch.Generator(device=dev).manual_seed(3))
        targets = [a0] * K

        def event_ms(fn, reps=3, warm=2):
            for _ in range(warm):
                fn()
            torch.cuda.synchronize()
            t = 0.0
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                fn()
                e1.record(stream)
                e1.synchronize()
                t += e0.elapsed_time(e1)
            return max_over_ranks(t / reps, world, dev)

        def backward():
            h.sam_build_backward_batched(aks, targets, pats, mv, gbar, "fp32r", args.refine, 1.0, offsets=offs_a)

        ta_re = event_ms(backward)
        # factor tape: the build records every column's R, the adjoint
        # replays it instead of recomputing the QR
        tape = torch.empty((h.sam_factor_tape_bytes(pats, "fp32r") + 15) // 16 * 2, dtype=torch.float64, device=dev)
        h.sam_set_factor_tape(sam.SAM_TAPE_RECORD, tape)
        tb_rec = event_ms(lambda: h.sam_build_batched(aks, a0, pats, "fp32r", args.refine, M_val=mv))
        h.sam_set_factor_tape(sam.SAM_TAPE_REPLAY, tape)
        ta = event_ms(backward)
        h.sam_set_factor_tape(sam.SAM_TAPE_OFF)
        extra["adjoint_columns_per_s"] = job_value(cols_per_step, world, ta_re)
        extra["adjoint_ms"] = ta_re
        extra["adjoint_roofline"] = adjoint_roofline(seq.mats, args.level, args.refine, ta_re)
        extra["adjoint_note"] = ("adjoint_ms: the batched adjoint recomputing each column's QR (nothing stored "
                                 "between forward and backward); adjoint_tape_ms: the same adjoint reading R from "
                                 "the build's factor tape (sam_set_factor_tape); build_with_tape_ms: the batched "
                                 "build recording the tape (patterns built beforehand)")
        extra["adjoint_tape_columns_per_s"] = job_value(cols_per_step, world, ta)
        extra["adjoint_tape_ms"] = ta
        extra["build_with_tape_ms"] = tb_rec
        extra["factor_tape_bytes"] = int(tape.numel() * 8)
        extra["adjoint_tape_roofline"] = adjoint_roofline(seq.mats, args.level, args.refine, ta, tape=True)
        del tape
        for p in pats:
            p.destroy()

    # ---- Sec. 4 sparsification of every source (column threshold tau = 0.8),
    #      all K in one batched call: HBM-bound, reported against the measured
    #      copy bandwidth (and the K single calls beside it)
    if not args.quick:
        for _ in range(2):
            h.sam_sparsify_batched(aks, "tau", 0.8)
        torch.cuda.synchronize()
        ts, tsingle, moved = 0.0, 0.0, 0.0
        nrep = 5
        for _ in range(nrep):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            outs = h.sam_sparsify_batched(aks, "tau", 0.8)
            e1.record(stream)
            e1.synchronize()
            ts += e0.elapsed_time(e1) / nrep
        for a, at in zip(aks, outs):
            # read the CSR once (+ column maxima), write the kept entries and a keep byte per entry
            moved += 12.0 * a.nnz + 4.0 * (n + 1) + 8.0 * n + 1.0 * a.nnz + 12.0 * at.nnz + 4.0 * (n + 1)
        for a in aks:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            h.sam_sparsify(a, "tau", 0.8)
            e1.record(stream)
            e1.synchronize()
            tsingle += e0.elapsed_time(e1)
        extra["sparsify_ms_per_map"] = ts / K
        extra["sparsify_single_call_ms_per_map"] = tsingle / K
        extra["sparsify_gbs"] = moved / (ts * 1e-3) / 1e9
        extra["sparsify_hbm_frac"] = extra["sparsify_gbs"] / measured_hbm_gbs()

    # ---- the map in use (Sec. 1-2): restarted GMRES(30) on A_{K-1} x = b with
    #      the right preconditioner M_{K-1} (P_0 v), P_0 a level-2 sparse
    #      approximate inverse of A_0 (the map of A_0 onto I), against P_0 alone
    if not args.quick:
        extra.update(krylov_measurement(h, sam, torch, dev, stream, aks, a0, offs, out[0], out[1], v32, n, K,
                                        world, rank))

    # ---- the other workloads of the same path (patterns + batched maps per step)
    if not args.quick and not args.no_configs and world == 1:
        extra["configs"] = config_figures(h, sam, torch, dev, stream)
        extra["cd2d_study"] = cd2d_study(h, sam, torch, dev, stream)

    # ---- roofline of the dominant kernel (largest least-squares size class)
    sizes = column_sizes(seq.mats, args.level)
    classes = size_classes()
    schedule = h.sam_get_bin_schedule()
    dom = int(np.argmax(lsq_ms))
    f32 = f64 = gathered = 0.0
    for (I, J, nB) in sizes:
        sel = bin_of(I, J, nB, classes, schedule) == dom
        a, b = algorithmic_flops(I[sel], J[sel], nB[sel], "fp32r", args.refine)
        f32 += float(np.sum(a))
        f64 += float(np.sum(b))
        # gathered bytes: every entry of B_j (FP64 value + int32 row) once per column
        gathered += 12.0 * float(np.sum(nB[sel]))
    t_launch = lsq_ms[dom] / max(lsq_n[dom], 1) * 1e-3
    nsteps_prof = args.steps
    f32_l, f64_l = f32, f64  # per launch: one launch per size class covers all maps of a step
    hbm_gbs = measured_hbm_gbs()
    t_hbm = gathered / (hbm_gbs * 1e9)
    t_roof = max(f32_l / PEAK_FP32, f64_l / PEAK_FP64, t_hbm)
    fp32_frac = f32_l / t_launch / PEAK_FP32
    fp64_frac = f64_l / t_launch / PEAK_FP64
    bound, unit = "alu", "TFLOP/s"
    if t_hbm >= max(f32_l / PEAK_FP32, f64_l / PEAK_FP64):
        bound, unit = "hbm", "GB/s"
        ach, peak = gathered / t_launch / 1e-3, hbm_gbs * 1e9 / 1e-3  # scaled by 1e12 below -> GB/s
    elif f32_l / PEAK_FP32 >= f64_l / PEAK_FP64:
        ach, peak = f32_l / t_launch, PEAK_FP32
    else:
        ach, peak = f64_l / t_launch, PEAK_FP64
    traffic = None
    tf = os.path.join(HERE, "profiles", "traffic.json")
    if os.path.exists(tf):
        try:
            import hashlib

            rec = json.load(open(tf))
            if (rec.get("kernel_sha256") == kernel_hash() and str(dom) in rec.get("bytes_per_column", {})
                    and rec.get("variant", {}).get(str(dom), 0) == variants[dom]):
                # traffic per column from the capture, times this launch's columns
                ncols = sum(int(np.sum(bin_of(I, J, nB, classes, schedule) == dom)) for (I, J, nB) in sizes)
                traffic = rec["bytes_per_column"][str(dom)] * ncols
        except Exception:
            traffic = None
    roofline = {"bound": bound, "achieved": ach / 1e12, "peak": peak / 1e12, "unit": unit,
                "frac": t_roof / t_launch, "traffic": traffic,
                "kernel": "lsq_kernel size class %d (|I|<=%d, |J|<=%d)" % (dom, classes["max_rows"][dom],
                                                                           classes["max_cols"][dom]),
                "launch_ms": t_launch * 1e3, "fp32_flops_per_launch": f32_l, "fp64_flops_per_launch": f64_l,
                "fp32_frac": fp32_frac, "fp64_frac": fp64_frac,
                "gathered_bytes_per_launch": gathered, "t_hbm_ms": t_hbm * 1e3, "hbm_gbs_measured": hbm_gbs,
                "peak_source": PEAK_SOURCE}
    if not args.quick:
        p32, p64 = h.sam_peak_flops(100.0)
        roofline["probe_fp32_tflops"] = p32 / 1e12
        roofline["probe_fp64_tflops"] = p64 / 1e12

    # ---- end to end through the C ABI with host buffers
    pin = lambda x: torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
    hk = [sam.Csr(pin(m.indptr), pin(m.indices), pin(m.data), n=n) for m in seq.mats]
    h0 = sam.Csr(pin(a0h.indptr), pin(a0h.indices), pin(a0h.data), n=n)
    hout = (torch.empty(K * (n + 1), dtype=torch.int32).pin_memory(),
            torch.empty(int(offs[-1]), dtype=torch.int32).pin_memory(),
            torch.empty(int(offs[-1]), dtype=torch.float64).pin_memory())
    h2d = sum(m.indptr.nbytes + m.indices.nbytes for m in seq.mats)  # pattern build
    h2d += sum(m.indptr.nbytes + m.indices.nbytes + m.data.nbytes for m in seq.mats)
    h2d += a0h.indptr.nbytes + a0h.indices.nbytes + a0h.data.nbytes
    d2h = sum(int(t.numel() * t.element_size()) for t in hout) + 8 * K

    def e2e_step():
        pats = h.sam_pattern_build_batched(hk, args.level)
        h.sam_build_batched(hk, h0, pats, "fp32r", args.refine, M_row_ptr=hout[0], M_col_idx=hout[1],
                            M_val=hout[2], want_fro=True, offsets=offs)
        for p in pats:
            p.destroy()

    for _ in range(3):
        e2e_step()
    torch.cuda.synchronize()
    # every step ends synchronised (host outputs): wall time per step, median
    # (host jitter), the mean beside it
    ne = max(10, args.steps)
    e2e_ms = []
    for _ in range(ne):
        t0 = time.perf_counter()
        e2e_step()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    torch.cuda.synchronize()
    e2e_med = max_over_ranks(statistics.median(e2e_ms), world, dev)
    e2e_mean = max_over_ranks(statistics.fmean(e2e_ms), world, dev)
    e2e_value = job_value(cols_per_step, world, e2e_med)

    # ---- CPU oracle baseline and sampled parity (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and world == 1:
        cpu, timed_maps = cpu_baseline(seq, args.level)
        if not args.quick:
            import oracle

            k = len(timed_maps) - 1
            ak = seq.mats[k]
            cp, ri = oracle.pattern(ak, args.level)
            rng = np.random.default_rng(0)
            cols = np.sort(rng.choice(n, 2000, replace=False)).astype(np.int32)
            ref = oracle.build_cols(ak, a0h, cp, ri, cols)
            import scipy.sparse as sp

            m = sp.csr_matrix((v32[offs[k]:offs[k + 1]].cpu().numpy(), out[1][offs[k]:offs[k + 1]].cpu().numpy(),
                               out[0][k * (n + 1):(k + 1) * (n + 1)].cpu().numpy()), shape=(n, n)).tocsc()
            m.sort_indices()
            idx = np.concatenate([np.arange(cp[j], cp[j + 1]) for j in cols])
            extra["sample_rel_fro_vs_oracle"] = float(np.linalg.norm(m.data[idx] - ref["mval"][idx]) /
                                                      np.linalg.norm(ref["mval"][idx]))
            cerr = [np.linalg.norm(m.data[cp[j]:cp[j + 1]] - ref["mval"][cp[j]:cp[j + 1]]) /
                    np.linalg.norm(ref["mval"][cp[j]:cp[j + 1]]) for j in cols]
            extra["max_col_rel_err_vs_oracle"] = float(max(cerr))
            extra["oracle_sample_columns"] = int(len(cols))

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                "config": {"workload": seq.name + "_seq%d_level%d" % (K, args.level), "n": n, "maps": K,
                           "level": args.level, "precision": "fp32 Householder QR + %d FP64 CSNE step(s), guarded (columns predicted above "
                                                       "1e-10 re-solved in FP64)" % args.refine,
                           "columns_per_step": cols_per_step, "tile_variants": variants,
                           "bin_schedule": schedule, "parallelism": "replicas" if world > 1 else "single",
                           "l2": "flushed between steps (256 MiB write outside the timed interval)"},
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                        "ms_per_step_median": e2e_med, "ms_per_step_mean": e2e_mean, "steps": ne,
                        "mean_value": job_value(cols_per_step, world, e2e_mean)},
                "gpu_launches": gpu_launches, "roofline": roofline, "clocks": clocks, "cpu_baseline": cpu,
                "maps_per_s": job_value(K, world, ms)}
        line.update(extra)
        print(json.dumps(line), flush=True)
    h.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
