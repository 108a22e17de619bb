"""Benchmark: SVDs/s of the mixed-precision Jacobi SVD on one GB300 (per rank), next to the
plain FP64 Jacobi on the same GPU and the CPU oracle.

Workload (one step = one full SVD, every stage of the hot path), by default the largest
single-GPU configuration: the 8192 x 8192 FP64 matrix A = B D, B with singular values
log-spaced 1 .. 1e-2 (Haar factors), D = diag(10^U(-10, 0)), seed 4, mixed path forced (the
paper's low-precision stage runs). ``--workload precision`` selects the 2048 x 1024 matrix
(B: 1 .. 1e-3, D = diag(10^U(-8, 0)), seed 1) instead; with the default workload it is also
timed as an extra. The plain path and the automatic branch choice are timed beside the mixed
one, and the 4096-matrix uneven batch (one persistent launch) is reported as an extra.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload large|precision] [--n N] [--m M]

Prints one JSON line (rank 0). Timing: CUDA events on the library's stream around each
step, L2 flushed (256 MiB write) before every timed step, max over ranks.

The reference arm (``--impl reference``) is the CPU oracle (plain C, one host core). Where one
complete oracle SVD of the workload takes more than about a minute (the 8192 x 8192 matrix:
hours), every step times a bounded sample of it and the SVD time is extrapolated from the
sample (the line says so: ``extrapolated``, with the parts).
"""
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

WORKLOADS = {
    "large": "large_%dx%d: A = B D, B = W1 diag(logspace(0,-2,n)) W2^T (Haar), D = diag(10^U(-10,0)), "
             "seed 4, FP64 column-major",
    "precision": "precision_%dx%d: A = B D, B = W1 diag(logspace(0,-3,n)) W2^T (Haar), "
                 "D = diag(10^U(-8,0)), seed 1, FP64 column-major",
}
BATCH_WORKLOAD = ("4096 matrices, n ~ U{16..256}, m = n + U{0..n}, kappa = 10^U(1,8), sigma "
                  "log-spaced, seed 2; mode mixed; one persistent launch")


def parse(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="large", choices=["large", "precision"])
    p.add_argument("--n", type=int, default=None, help="columns (large: also rows)")
    p.add_argument("--m", type=int, default=None, help="rows (precision workload)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-extras", action="store_true",
                   help="skip the plain/auto comparison, the 2048 x 1024 extra and the batch")
    p.add_argument("--batch-count", type=int, default=4096)
    p.add_argument("--batch-only", action="store_true",
                   help="time only the uneven batch (--batch-count matrices), one JSON line")
    p.add_argument("--no-e2e", action="store_true", help="skip the end-to-end (host buffers) measurement")
    p.add_argument("--low-kernel", default="auto", choices=["auto", "tc", "reg"],
                   help="kernel of the binary32 stage (auto: by size)")
    a = p.parse_args(argv)
    if a.workload == "large":
        a.n = a.n or 8192
        a.m = a.m or a.n
    else:
        a.n = a.n or 1024
        a.m = a.m or 2 * a.n
    return a


def workload(args):
    """(description, A as float64 Fortran-order numpy array)."""
    from paper_2209_04626_gb300 import inputs
    if args.workload == "large":
        A = inputs.large_8192(n=args.n, m=args.m)
    else:
        A = inputs.precision_2048x1024(m=args.m, n=args.n)
    return WORKLOADS[args.workload] % (args.m, args.n), A


# ------------------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while active (read-only)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
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
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------ oracle

# a complete oracle SVD is timed when it takes about a minute at most (2048 x 1024: 14 s);
# larger workloads are sampled and extrapolated
FULL_ORACLE_MAX_MN2 = 2048 * 1024 * 1024


def oracle_full(A):
    """One complete oracle SVD (Algorithm 4, low-precision stage forced) of A."""
    import oracle
    oracle.lib()
    t0 = time.perf_counter()
    _, _, _, st = oracle.svd(A, mode="mixed")
    return time.perf_counter() - t0, st


def oracle_sample(A):
    """The oracle's time for one SVD of A, extrapolated from a bounded sample (a few seconds):
      * the rate of its RRQR (Businger-Golub, binary64) on the first 192 columns of A, applied
        to the RRQR's 2 m n^2 - 2 n^3 / 3 flops;
      * the rate of its Householder QR on the same panel, applied to the switch (two triangular
        GEMMs of n^3 flops, the QR of B and the forming of Q, 4 n^3 / 3 each) and to the
        assembly of U (4 m n^2 - 2 n^3);
      * the time per column pair of one binary32 sweep and of one binary64 sweep with V, on n
        rows of the first 256 columns (the cost of a pair does not depend on the other columns;
        in a first sweep every pair rotates); the last sweep of each stage, which rotates
        (almost) nothing, is counted at the dot products' share of a pair's flops;
      * the sweep counts of the oracle's own complete SVD of the same recipe at n = 512.
    Returns a dict with the estimate and its parts."""
    import oracle
    from paper_2209_04626_gb300 import inputs
    oracle.lib()
    m, n = A.shape
    kq = min(192, n)
    t0 = time.perf_counter()
    oracle.geqp3(A[:, :kq])
    t_qp = time.perf_counter() - t0
    rate_qp = (2.0 * m * kq * kq - 2.0 * kq ** 3 / 3.0) / t_qp
    t0 = time.perf_counter()
    oracle.geqrf(A[:, :kq])
    t_qr = time.perf_counter() - t0
    rate_qr = (2.0 * m * kq * kq - 2.0 * kq ** 3 / 3.0) / t_qr
    ks = min(256, n)
    X = np.asfortranarray(A[:n, :ks])
    pairs_s = ks * (ks - 1) / 2.0
    V = np.zeros((n, ks), order="F")
    V[:ks, :ks] = np.eye(ks)
    t0 = time.perf_counter()
    oracle.jacobi(X, V, maxsweep=1)
    t64_rot = (time.perf_counter() - t0) / pairs_s
    t0 = time.perf_counter()
    oracle.jacobi_f32(X.astype(np.float32), maxsweep=1)
    t32_rot = (time.perf_counter() - t0) / pairs_s
    # sweep counts: the oracle's complete SVD of the same recipe at n = 512
    ns = min(512, n)
    As = inputs.large_8192(n=ns) if m == n else inputs.precision_2048x1024(m=2 * ns, n=ns)
    t0 = time.perf_counter()
    _, _, _, sts = oracle.svd(As, mode="mixed")
    t_small = time.perf_counter() - t0
    s32, s64 = max(1, sts["sweeps_low"]), max(1, sts["sweeps_work"])
    pairs = n * (n - 1) / 2.0
    t_precond = (2.0 * m * n * n - 2.0 * n ** 3 / 3.0) / rate_qp
    t_switch = (n ** 3 + 4.0 * n ** 3 / 3.0 + 4.0 * n ** 3 / 3.0 + n ** 3) / rate_qr
    t_final = (4.0 * m * n * n - 2.0 * n ** 3) / rate_qr
    # the last sweep of a stage rotates (almost) nothing: its pairs cost the dot product only,
    # 2n of the 2n + 6n flops of a rotated pair in binary32 and of 2n + 12n with V in binary64
    t_low = pairs * t32_rot * ((s32 - 1) + 0.25)
    t_work = pairs * t64_rot * ((s64 - 1) + 1.0 / 7.0)
    est = t_precond + t_switch + t_low + t_work + t_final
    return {"est_svd_s": est, "extrapolated": True,
            "parts_s": {"precond": t_precond, "low": t_low, "switch": t_switch, "work": t_work,
                        "final": t_final},
            "sweeps_used": [s32, s64], "sample_s": t_qp + t_qr + t_small,
            "sample": ("extrapolated from a timed sample of the single-threaded C oracle on this "
                       "matrix: RRQR and QR rates on its first %d columns, per-pair times of one "
                       "binary32 and one binary64 sweep (with V) on %d rows x %d columns, and the "
                       "sweep counts (%d + %d) of the oracle's complete SVD of the same recipe at "
                       "n = %d (%.1f s)" % (kq, n, ks, s32, s64, ns, t_small))}


def oracle_step(A):
    """One reference-arm step: (SVD seconds, info dict). A complete oracle SVD where it fits in
    about a minute, else the extrapolated sample."""
    m, n = A.shape
    if m * n * n <= FULL_ORACLE_MAX_MN2:
        dt, st = oracle_full(A)
        return dt, {"extrapolated": False, "sweeps_used": [st["sweeps_low"], st["sweeps_work"]],
                    "sample": ("one complete SVD of the %dx%d workload by the single-threaded C "
                               "oracle (Algorithm 4, low-precision stage forced; %d + %d sweeps), "
                               "%.1f s" % (m, n, st["sweeps_low"], st["sweeps_work"], dt))}
    r = oracle_sample(A)
    return r["est_svd_s"], r


# ------------------------------------------------------------------------------ dist

def max_over_ranks(value, device):
    """Maximum of a per-rank float over all ranks (the slowest rank's time); identity when
    torch.distributed is not initialized. Ends with a barrier."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return value
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def job_throughput(world, steps, max_ms):
    """Whole-job SVDs/s of `world` replicas that each ran `steps` SVDs in at most max_ms."""
    return world * steps / (max_ms / 1000.0)


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reference_arm(args):
    world, rank, local = dist_setup(args)
    if rank != 0:
        return 0
    desc, A = workload(args)
    for _ in range(args.warmup):
        oracle_step(A)
    times, infos = [], []
    t_all = time.perf_counter()
    for _ in range(args.steps):
        dt, info = oracle_step(A)
        times.append(dt)
        infos.append(info)
    wall = time.perf_counter() - t_all
    v = len(times) / sum(times)
    last = infos[-1]
    cb = {"value": v, "unit": "SVDs/s", "cores": 1, "kind": "oracle", "sample": last["sample"],
          "extrapolated": last["extrapolated"]}
    if last["extrapolated"]:
        cb["parts_s"] = last["parts_s"]
    line = {"impl": "reference", "metric": "SVDs/s", "value": v, "unit": "SVDs/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "m": args.m, "n": args.n, "mode": "mixed",
                       "parallelism": "replicas", "extrapolated": last["extrapolated"],
                       "sweeps_used": last["sweeps_used"]},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "SVDs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": wall}
    if last["extrapolated"]:
        line["sampled_wall_s_per_step"] = wall / len(times)
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------------------ ours

def flops_sweeps(n, sweeps, rotations, with_v=True):
    """Algorithmic flops of a Jacobi stage on an n x n matrix by the hot-path table's per-unit
    work: a dot product (2n flops) for every pair of every sweep, plus, for every rotation
    applied, the rotation of the pair's two columns of Y (6n: a multiply and an FMA per
    element) and, with V, of V's two columns (6n)."""
    return sweeps * n * (n - 1) / 2 * 2 * n + rotations * (12 if with_v else 6) * n


def flops_svd_fp64(m, n, sweeps_work, rot_work):
    """Algorithmic FP64 flops of the whole mixed SVD (RRQR, switch, refinement, U)."""
    qrcp = 2 * m * n * n - 2 * n ** 3 / 3
    switch = n ** 3 + 4 * n ** 3 / 3 + 4 * n ** 3 / 3 + n ** 3   # tri GEMM, QR, form Q, tri GEMM
    final = 4 * m * n * n - 2 * n ** 3
    return qrcp + switch + flops_sweeps(n, sweeps_work, rot_work) + final


FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12  # SMs x FP32 FMA/clk x 2 flop x max clock
FP64_PEAK_DERIVED = 152 * 2 * 2 * 2.07e9 / 1e12   # SMs x FP64 FMA/clk x 2 flop x max clock


def _measured_bf16_tflops():
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"])
    except Exception:
        return 1900.0  # the recipe's fallback burst figure


TF32_PEAK_TFLOPS = _measured_bf16_tflops() * 1.1 / 2.25


def time_calls(fn, steps, stream, flush):
    import torch
    out = []
    for k in range(steps):
        flush.fill_(float(k))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        out.append(e0.elapsed_time(e1))
    return out


def traffic_record(m, n, work_cluster=1):
    """DRAM bytes per launch of the refinement sweeps from a committed ncu summary, used only
    while the kernel's sources are the ones that were captured (sha256 recorded with each
    record) and for the same form of the kernel (CTAs per visit)."""
    tfile = os.path.join(ROOT, "profiles", "sweep_fp64_traffic.json")
    if not os.path.exists(tfile):
        return None, None
    try:
        tj = json.load(open(tfile))
        why = "no capture for this size and kernel form"
        for rec in tj.get("records", []):
            if rec.get("m") != m or rec.get("n") != n or rec.get("work_cluster", 1) != work_cluster:
                continue
            hh = hashlib.sha256()
            for f in rec.get("sources", []):
                hh.update(open(os.path.join(ROOT, f), "rb").read())
            if hh.hexdigest() != rec.get("sources_sha256"):
                why = "sources changed since the capture"
                continue
            return rec.get("bytes_per_launch"), rec.get("how")
    except Exception as ex:  # reported, not fatal
        return None, "unreadable: %s" % ex
    return None, why


def tensor_flops_low(m, n, sweeps):
    """Tensor-core flops of the blocked binary32 stage (64-column blocks, visits of 128 columns):
    per visit the Gram Z^T Z and the application Z W, each as three TF32 products (the split),
    2 m 128^2 flops each; every visit counted as rotating (an upper bound: a visit without
    rotations skips the application)."""
    k = (n + 63) // 64
    k += k & 1
    visits = sweeps * (k - 1) * (k // 2)
    return visits * 2 * 3 * 2.0 * m * 128 * 128


def measure_batched(args, dev, stream, flush):
    """The uneven batch (args.batch_count matrices) in one persistent launch: SVDs/s over three
    timed calls after a tuning call, and an upper-bound roofline of its binary64 work."""
    import torch
    from paper_2209_04626_gb300 import inputs, mpjsvd
    mats, _, bm, bn, bk = inputs.batch_matrices(count=args.batch_count)
    dmats = [mpjsvd.colmajor(torch.from_numpy(X), dev) for X in mats]
    hb = mpjsvd.Handle(mode="mixed")
    hb.svd_batched(dmats)
    torch.cuda.synchronize()
    binfo = [None]

    def bstep():
        binfo[0] = hb.svd_batched(dmats)[3]
    bms = time_calls(bstep, 3, stream, flush)
    # roofline of the batched launch (binary64 work by the hot-path table's counts, with three
    # refinement sweeps in which every pair rotates: an upper bound of the work done)
    fl_b = sum(flops_svd_fp64(int(mi), int(ni), 3, 3 * int(ni) * (int(ni) - 1) // 2)
               for mi, ni in zip(bm, bn))
    ach_b = fl_b / (statistics.mean(bms) / 1000.0) / 1e12
    out = {"workload": BATCH_WORKLOAD, "count": len(mats),
           "svds_per_s": len(mats) / (statistics.mean(bms) / 1000.0),
           "ms": statistics.mean(bms),
           "nonzero_info": int((binfo[0] != 0).sum().item()),
           "tuning": mpjsvd.mpjsvd_get_batched_tuning(hb.h),
           "roofline": {"bound": "alu", "achieved_upper": ach_b, "peak": FP64_PEAK_DERIVED,
                        "unit": "TFLOP/s", "frac_upper": ach_b / FP64_PEAK_DERIVED,
                        "flop_model": "per matrix: RRQR 2mn^2 - 2n^3/3, switch 14n^3/3, "
                                      "3 sweeps x n(n-1)/2 x 14n, U 4mn^2 - 2n^3 (upper bound)"}}
    hb.close()
    return out


def batch_only(args):
    """--batch-only: just the uneven batch (profiling and quick checks), one JSON line."""
    import torch
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    out = measure_batched(args, dev, torch.cuda.current_stream(dev), flush)
    print(json.dumps({"batched": out}))
    return 0


def ours(args):
    import torch
    world, rank, local = dist_setup(args)
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    from paper_2209_04626_gb300 import inputs, mpjsvd
    m, n = args.m, args.n
    desc, A_np = workload(args)
    A = mpjsvd.colmajor(torch.from_numpy(A_np), dev)
    U = mpjsvd.empty_colmajor(m, n, dev)
    S = torch.empty(n, dtype=torch.float64, device=dev)
    V = mpjsvd.empty_colmajor(n, n, dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    h = mpjsvd.Handle(mode="mixed", timing=1, low_kernel=args.low_kernel)

    def one(handle):
        handle.svd(A, out=(U, S, V))

    for _ in range(args.warmup):
        one(h)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()

    clocks = ClockSampler(dev.index)
    clocks.start()
    time.sleep(0.3)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    per_step_stats = []
    t_wall = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        one(h)
        ev[k][1].record(stream)
        per_step_stats.append(h.stats())  # synchronizes; outside the event pair
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall
    # the FP64 FMA microbenchmark right after the timed region (the GPU at its working clock)
    fp64_measured = mpjsvd.mpjsvd_measure_fp64_peak()
    clk = clocks.stop()
    ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(sum(ms), dev)
    st = per_step_stats[-1]
    value = job_throughput(world, args.steps, total_ms)
    assert all(s["status"] == 0 for s in per_step_stats), [s["status"] for s in per_step_stats]

    # roofline of the dominant kernel: the FP64 refinement sweeps (one cooperative launch per
    # SVD, its duration from CUDA events around it on the handle's stream)
    avg_work_ms = statistics.mean(s["ms_work"] for s in per_step_stats)
    fl_work = statistics.mean(flops_sweeps(n, s["sweeps_work"], s["rot_work"]) for s in per_step_stats)
    achieved = fl_work / (avg_work_ms / 1000.0) / 1e12
    avg_low_ms = statistics.mean(s["ms_low"] for s in per_step_stats)
    fl_low = statistics.mean(flops_sweeps(n, s["sweeps_low"], s["rot_low"], with_v=False)
                             for s in per_step_stats)
    phases = {k: statistics.mean(s[k] for s in per_step_stats)
              for k in ["ms_qr", "ms_branch", "ms_low", "ms_switch", "ms_work", "ms_final"]}
    wcl = st["work_cluster"]
    traffic, traffic_how = traffic_record(m, n, wcl)

    # accuracy of the timed outputs (torch FP64 matmuls, verification only)
    with torch.no_grad():
        bw = float(torch.linalg.norm(A - (U * S) @ V.t()) / torch.linalg.norm(A))
        eye = torch.eye(n, dtype=torch.float64, device=dev)
        orthU = float((U.t() @ U - eye).abs().max())
        orthV = float((V.t() @ V - eye).abs().max())
        del eye
    S_mixed = S.clone()

    compare = None
    if not args.no_extras:
        # plain FP64 Jacobi on the same GPU and the automatic branch choice
        Up, Sp, Vp = torch.empty_like(U), torch.empty_like(S), torch.empty_like(V)
        res = {}
        for mode in ("plain", "auto"):
            hm = mpjsvd.Handle(mode=mode, timing=1)
            tm = time_calls(lambda: hm.svd(A, out=(Up, Sp, Vp)), 1, stream, flush)
            sm_ = hm.stats()
            res[mode] = {"ms": tm[0], "branch": sm_["branch_name"], "sweeps_low": sm_["sweeps_low"],
                         "sweeps_work": sm_["sweeps_work"], "status": sm_["status"],
                         "max_rel_sigma_vs_mixed": float(((Sp - S_mixed).abs() / S_mixed).max())}
            hm.close()
        del Up, Sp, Vp
        compare = {"plain_ms": res["plain"]["ms"], "plain_svds_per_s": 1000.0 / res["plain"]["ms"],
                   "plain_sweeps_work": res["plain"]["sweeps_work"],
                   "mixed_over_plain": res["plain"]["ms"] / (total_ms / args.steps),
                   "auto_ms": res["auto"]["ms"], "auto_branch": res["auto"]["branch"],
                   "auto_sweeps": [res["auto"]["sweeps_low"], res["auto"]["sweeps_work"]],
                   "max_rel_sigma_plain_vs_mixed": res["plain"]["max_rel_sigma_vs_mixed"],
                   "max_rel_sigma_auto_vs_mixed": res["auto"]["max_rel_sigma_vs_mixed"]}

    # end to end through the public API: pinned host A -> device, SVD, U, S, V -> host
    e2e_value = None
    if not args.no_e2e:
        A_host = torch.from_numpy(np.asfortranarray(A_np).T.copy()).t().pin_memory()
        U_host = torch.empty((n, m), dtype=torch.float64).t().pin_memory()
        S_host = torch.empty(n, dtype=torch.float64).pin_memory()
        V_host = torch.empty((n, n), dtype=torch.float64).t().pin_memory()
        A_dev = mpjsvd.empty_colmajor(m, n, dev)

        def e2e_step():
            A_dev.copy_(A_host, non_blocking=True)
            h.svd(A_dev, out=(U, S, V))
            U_host.copy_(U, non_blocking=True)
            S_host.copy_(S, non_blocking=True)
            V_host.copy_(V, non_blocking=True)
        e2e_ms = time_calls(e2e_step, 2, stream, flush)
        e2e_value = world * len(e2e_ms) / (sum(e2e_ms) / 1000.0)
        del A_host, U_host, V_host, A_dev

    extras = {}
    if not args.no_extras and args.workload == "large":
        # the 2048 x 1024 precision workload: mixed, plain and the automatic choice
        P = mpjsvd.colmajor(torch.from_numpy(inputs.precision_2048x1024()), dev)
        Uq, Sq, Vq = mpjsvd.empty_colmajor(2048, 1024, dev), torch.empty(1024, dtype=torch.float64, device=dev), \
            mpjsvd.empty_colmajor(1024, 1024, dev)
        pr = {}
        for mode in ("mixed", "plain", "auto"):
            hm = mpjsvd.Handle(mode=mode, timing=1)
            hm.svd(P, out=(Uq, Sq, Vq))
            tm = time_calls(lambda: hm.svd(P, out=(Uq, Sq, Vq)), 5, stream, flush)
            sm_ = hm.stats()
            pr[mode] = {"ms": statistics.mean(tm), "branch": sm_["branch_name"],
                        "sweeps": [sm_["sweeps_low"], sm_["sweeps_work"]],
                        "phases_ms": {k: round(sm_[k], 2) for k in ["ms_qr", "ms_low", "ms_switch",
                                                                     "ms_work", "ms_final"]}}
            hm.close()
        pr["mixed_over_plain"] = pr["plain"]["ms"] / pr["mixed"]["ms"]
        extras["precision_2048x1024"] = pr
        del P, Uq, Sq, Vq
    if not args.no_extras:
        extras["batched"] = measure_batched(args, dev, stream, flush)

    h.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    if args.batch_only:
        return batch_only(args)
    return ours(args)


if __name__ == "__main__":
    sys.exit(main())
