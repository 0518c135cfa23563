"""Benchmark of the block-sparse x dense product Y = W.X on GB300.

Workload (the static sweep of Table 2, restricted as the paper's headline
comparisons are): m = k = 4096, n = 2048, FP16 values and X, FP32
accumulation, block size b in {1, 4, 8, 16} x density d in {1/32, 1/16, 1/8,
1/4}, uniform random block positions, N(0, 1) values.  One step runs all 16
products once through the library's public C ABI (AUTO kernel: b = 1 gather
kernel, b >= 4 tensor-core kernel).  The 16 problems' inputs total about
0.6 GB, more than twice L2, and each is touched once per step, so every
launch reads cold inputs.

Prints one JSON line (rank 0).  ``value`` is nonzero-FLOP throughput
(2 * nnz * n per product, Section 3) of the whole step in TFLOP/s, summed
over ranks; ``e2e`` is the same metric through ``spmm_run_host`` with X and Y
in pinned host memory; ``roofline`` describes the dominant kernel family;
``cpu_baseline`` times the FP64 oracle on a bounded sample.
``--impl reference`` times that oracle alone, as the reference arm.
"""
import argparse
import ctypes
import json
import math
import os
import statistics
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}
N_SMS = 152
# FP32 CUDA-core peak: 152 SMs x 128 FP32 lanes x 2 FLOP per FMA x 2.07 GHz
ALU_PEAK_TFLOPS = N_SMS * 128 * 2 * 2.070e9 / 1e12
METRIC = "effective TFLOP/s & %roofline, block-sparse vs plain FP32/dense; serve p50/p99"
SWEEP_B = (1, 4, 8, 16)
SWEEP_D = (1 / 32, 1 / 16, 1 / 8, 1 / 4)
M = K = 4096
N = 2048
E2E_WORKERS = 4           # host threads (one stream each) of the end-to-end leg


def load_peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return p, "measured"
    except Exception:
        return dict(FALLBACK), "fallback"


# ------------------------------------------------------------ clocks (NVML)
class ClockSampler:
    """Samples SM clock and clock-event reasons through NVML every few ms."""
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, bus_id=None):
        self.ok = False
        self.samples = []
        self.reasons = 0
        self.max_mhz = None
        try:
            nv = ctypes.CDLL("libnvidia-ml.so.1")
            if nv.nvmlInit_v2() != 0:
                return
            h = ctypes.c_void_p()
            got = False
            if bus_id:
                got = nv.nvmlDeviceGetHandleByPciBusId_v2(bus_id.encode(), ctypes.byref(h)) == 0
            if not got and nv.nvmlDeviceGetHandleByIndex_v2(0, ctypes.byref(h)) != 0:
                return
            self.nv, self.h = nv, h
            try:
                self._reasons_fn = nv.nvmlDeviceGetCurrentClocksEventReasons
            except AttributeError:
                self._reasons_fn = nv.nvmlDeviceGetCurrentClocksThrottleReasons
            mx = ctypes.c_uint()
            if nv.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0:
                self.max_mhz = mx.value
            self.ok = True
        except OSError:
            pass

    def _run(self):
        c = ctypes.c_uint()
        r = ctypes.c_ulonglong()
        while not self._stop.is_set():
            if self.nv.nvmlDeviceGetClockInfo(self.h, 1, ctypes.byref(c)) == 0:
                self.samples.append(c.value)
            if self._reasons_fn(self.h, ctypes.byref(r)) == 0:
                self.reasons |= r.value
            time.sleep(0.002)

    def __enter__(self):
        if self.ok:
            self._stop = threading.Event()
            self._t = threading.Thread(target=self._run, daemon=True)
            self._t.start()
        return self

    def __exit__(self, *a):
        if self.ok:
            self._stop.set()
            self._t.join()

    def summary(self):
        if not self.ok or not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": ["unavailable"]}
        names = [v for k, v in self.REASONS.items() if self.reasons & k]
        return {"sm_mhz": statistics.median(self.samples), "sm_max_mhz": self.max_mhz,
                "reasons": names, "samples": len(self.samples)}


# ----------------------------------------------------------- distributed
def dist_setup(gpus):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world, device="cuda"):
    """The slowest rank's time (every rank gets it)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(flop_per_rank_step, steps, world, seconds_max):
    """Whole-job TFLOP/s: every rank runs the same step (weak scaling), so
    the job did world x steps x the per-rank FLOPs in the slowest rank's
    time."""
    return flop_per_rank_step * steps * world / seconds_max / 1e12


# ---------------------------------------------------------- sweep points
def roof_of(b, nnzb, peaks, kernel, m=M):
    """Roofline of one product (m rows of Y; fewer for a row slice) on the
    kernel that runs it: nonzero FLOPs, compulsory bytes and the bound (the
    slower of compute-at-peak -- tensor cores for the TC kernel, FP32 lanes
    for the CUDA-core kernels -- and bytes-over-HBM)."""
    flops = 2.0 * nnzb * b * b * N
    es = 2
    vals = nnzb * b * b * es
    idx = nnzb * 4 + (m // b + 1) * 4
    xy = (K * N + m * N) * es
    bytes_ = vals + idx + xy
    t_hbm = bytes_ / (peaks["hbm_gbs"] * 1e9)
    if kernel != "tc":
        t_cmp, unit = flops / (ALU_PEAK_TFLOPS * 1e12), "alu"
    else:
        t_cmp, unit = flops / (peaks["bf16_tflops"] * 1e12), "tensor"
    bound = unit if t_cmp >= t_hbm else "hbm"
    return flops, bytes_, bound, max(t_cmp, t_hbm)


def roof_time(flops, bytes_, peaks, compute="tensor"):
    """Roofline time of one launch, max(FLOP / P_compute, bytes / HBM), and
    which of the two binds ("tensor" or "alu" for compute, else "hbm")."""
    pc = (peaks["bf16_tflops"] if compute == "tensor" else ALU_PEAK_TFLOPS) * 1e12
    t_c = flops / pc
    t_m = bytes_ / (peaks["hbm_gbs"] * 1e9)
    return (t_c, compute) if t_c >= t_m else (t_m, "hbm")


def roofline_obj(launches, peaks, compute="tensor", traffic=None, kernel=None):
    """Roofline of a set of launches of one kernel, each given as (FLOP,
    compulsory bytes, measured seconds): frac = sum of the launches'
    roofline times over the sum of their measured times (a launch's
    roofline time is max(FLOP / P_compute, bytes / HBM), Section 3's nonzero
    FLOPs 2 nnzb b^2 n); bound = the roof that holds most of the roofline
    time; achieved = frac x that roof's peak (the roofline-equivalent rate),
    with the plain nonzero-FLOP and compulsory-byte rates beside it.  Every
    input of frac is in the object, so it can be recomputed from it."""
    roofs = [roof_time(f, b, peaks, compute) for f, b, _ in launches]
    t_roof = sum(t for t, _ in roofs)
    t_meas = sum(t for _, _, t in launches)
    share = {}
    for t, bd in roofs:
        share[bd] = share.get(bd, 0.0) + t
    bound = max(share, key=share.get) if share else "hbm"
    if bound == "hbm":
        peak, unit = peaks["hbm_gbs"], "GB/s"
    elif bound == "alu":
        peak, unit = ALU_PEAK_TFLOPS, "TFLOP/s"
    else:
        peak, unit = peaks["bf16_tflops"], "TFLOP/s"
    frac = t_roof / t_meas if t_meas > 0 else None
    flops = sum(f for f, _, _ in launches)
    bytes_ = sum(b for _, b, _ in launches)
    out = {"bound": bound, "achieved": round(frac * peak, 2) if frac else None,
           "peak": round(peak, 1), "unit": unit, "frac": round(frac, 4) if frac else None,
           "traffic": traffic, "kernel": kernel, "launches": len(launches),
           "t_roof_us": round(t_roof * 1e6, 3), "t_meas_us": round(t_meas * 1e6, 3),
           "roof_share": {k: round(v / t_roof, 3) for k, v in share.items()} if t_roof else {},
           "flop_nz": flops, "bytes_compulsory": bytes_,
           "achieved_tflops_nz": round(flops / t_meas / 1e12, 2) if t_meas else None,
           "achieved_gbs_compulsory": round(bytes_ / t_meas / 1e9, 1) if t_meas else None,
           "definition": "frac = t_roof_us / t_meas_us, t_roof = sum over launches of "
                         "max(FLOP_nz / P_%s, compulsory bytes / P_hbm); achieved = frac x peak"
                         % compute}
    return out


def kernel_source_sha16(files=("csrc/k_tc.cu", "csrc/tc_ptx.cuh", "csrc/capi.cpp",
                               "csrc/plan_host.cpp")):
    """Hash of the sources that decide what the tensor-core launches read
    (the kernel and its planner): DRAM traffic taken by ncu stays valid
    only while this hash is unchanged."""
    import hashlib
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2303_16999_gb300", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


# DRAM traffic per tc_kernel launch of the static sweep step, from one ncu
# capture (dram__bytes_read.sum + dram__bytes_write.sum over the 16 launches
# of one step; the command and the per-launch table are in
# profiles/tc_kernel_sweep_dram.md).  Used only while the kernel and planner
# sources hash to `sha16`; otherwise the bench reports traffic null.
SWEEP_TRAFFIC = {"sha16": "d203c1bc4cd1969a", "bytes_per_launch": 38571792.0,
                 "source": "profiles/tc_kernel_sweep_dram.md"}


def sweep_traffic():
    if SWEEP_TRAFFIC["sha16"] and SWEEP_TRAFFIC["sha16"] == kernel_source_sha16():
        return SWEEP_TRAFFIC["bytes_per_launch"]
    return None


# DRAM traffic of one b = 1 gather launch at n = 1 (m = k = 16384, d = 1/16,
# L2 evicted), from one ncu capture (profiles/gather1_kernel_small_n.md);
# used only while the gather kernels and the planner hash to `sha16`.
GATHER_FILES = ("csrc/k_cudacore.cu", "csrc/capi.cpp", "csrc/plan_host.cpp")
GATHER_TRAFFIC = {"sha16": "b8c2e5b5ed61398c", "bytes_per_launch": 67988992.0,
                  "source": "profiles/gather1_kernel_small_n.md"}


def gather_traffic():
    if GATHER_TRAFFIC["sha16"] and GATHER_TRAFFIC["sha16"] == kernel_source_sha16(GATHER_FILES):
        return GATHER_TRAFFIC["bytes_per_launch"]
    return None


def row_range(rank, world, m=M, align=16):
    """This rank's rows of a product split by rows over ``world`` GPUs:
    near-equal slices on a 16-row grid (the first ones one unit larger)."""
    units = m // align
    lo = rank * (units // world) + min(rank, units % world)
    hi = lo + units // world + (1 if rank < units % world else 0)
    return lo * align, hi * align


def build_points(torch, S, wl, dev, only=None, rows=None):
    """The 16 sweep products; with ``rows`` each plan covers that slice of
    Y's rows only (strong scaling: the whole W's pattern and values are
    passed, the plan keeps its blocks)."""
    pts = []
    mr = M if rows is None else rows[1] - rows[0]
    for b in SWEEP_B:
        for d in SWEEP_D:
            if only is not None and (b, round(1 / d)) != only:
                continue
            c = wl.sweep_case(b, d)
            vals = torch.from_numpy(c["vals"]).half()
            X = torch.from_numpy(c["X"]).half()
            plan = S.Plan(M, K, N, b, w_dtype=S.F16, brow=c["brow"], bcol=c["bcol"], rows=rows)
            plan.pack(vals.to(dev))
            info = plan.info()
            pts.append(dict(b=b, d=d, nnzb=info["nnzb"], nnzb_whole=len(c["brow"]), m=mr,
                            plan=plan, X=X.to(dev),
                            Y=torch.empty((mr, N), dtype=torch.float16, device=dev),
                            Xh=X.pin_memory(),
                            Yh=torch.empty((mr, N), dtype=torch.float16).pin_memory(),
                            kernel=info["kernel"], c=c))
            del vals
    torch.cuda.synchronize()
    return pts


def launches_per_run(p):
    info = p["plan"].info()
    return 1 + (1 if info["n_reductions"] > 0 else 0)


# ------------------------------------------------------------ CPU oracle
_ORACLE_CASE = {}


def oracle_sample(target_s, b=16, d=1 / 16, threads=1):
    """Times the FP64 oracle on the first block rows of one sweep point,
    sized to about target_s seconds of work on ``threads`` host cores.  With
    several threads the sample's block rows are cut into that many
    contiguous slices and the unmodified oracle runs on each slice in its
    own thread at once (the C oracle releases the interpreter lock), i.e.
    the oracle parallelised over block rows; only the oracle calls are
    timed."""
    import concurrent.futures as cf
    import oracle
    import torch
    from paper_2303_16999_gb300 import workloads as wl
    key = (b, d)
    if key not in _ORACLE_CASE:
        c = wl.sweep_case(b, d)
        _ORACLE_CASE[key] = (c, torch.from_numpy(c["X"]).half(), torch.from_numpy(c["vals"]).half())
    c, X, vals = _ORACLE_CASE[key]
    Xf = oracle.to_f64(X)

    def slices(rows):
        cuts = [rows * t // threads for t in range(threads + 1)]
        out = []
        for lo, hi in zip(cuts[:-1], cuts[1:]):
            if hi <= lo:
                continue
            sel = (c["brow"] >= lo) & (c["brow"] < hi)
            out.append((hi - lo, (c["brow"][sel] - lo).astype(np.int32), c["bcol"][sel],
                        vals[sel], int(sel.sum())))
        return out

    def run(rows):
        parts = slices(rows)
        with cf.ThreadPoolExecutor(max_workers=len(parts)) as ex:
            t0 = time.perf_counter()
            list(ex.map(lambda q: oracle.spmm(q[0] * b, K, b, q[1], q[2], q[3], Xf), parts))
            dt = time.perf_counter() - t0
        return dt, 2.0 * sum(q[4] for q in parts) * b * b * N

    dt, fl = run(max(2, threads))
    rate = fl / max(dt, 1e-9)
    per_row = fl / max(2, threads)
    rows = int(min(M // b, max(threads, target_s * rate / max(per_row, 1))))
    dt, fl = run(rows)
    return dict(value=fl / dt / 1e12, unit="TFLOP/s", cores=threads, kind="oracle",
                sample="FP64 oracle (%s) on the first %d of %d block rows of the b=%d, d=1/%d, "
                       "m=k=4096, n=2048 point (%.2f GFLOP, %.1f s)"
                       % ("single thread" if threads == 1 else
                          "%d threads, one slice of block rows each" % threads,
                          rows, M // b, b, round(1 / d), fl / 1e9, dt),
                seconds=dt, gflop=fl / 1e9)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline_leg(target_s=8.0):
    """The oracle timed on this host: all cores (the reported baseline) and
    one core beside it."""
    par = oracle_sample(target_s, b=16, d=1 / 4, threads=host_cores())
    one = oracle_sample(target_s, b=16, d=1 / 4, threads=1)
    out = {k: par[k] for k in ("value", "unit", "cores", "kind", "sample")}
    out["single_thread"] = {k: one[k] for k in ("value", "unit", "cores", "sample")}
    try:
        import platform
        out["host"] = "%s, %d cores visible" % (platform.machine(), host_cores())
    except Exception:
        pass
    return out


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    total = args.steps + args.warmup
    per_step = max(0.05, min(2.0, 120.0 / max(total, 1)))
    cores = host_cores()
    for _ in range(args.warmup):
        oracle_sample(per_step, threads=cores)
    fl = 0.0
    dt = 0.0
    last = None
    for _ in range(args.steps):
        last = oracle_sample(per_step, threads=cores)
        fl += last["gflop"] * 1e9
        dt += last["seconds"]
    v = fl / dt / 1e12
    cpu = dict(value=v, unit="TFLOP/s", cores=cores, kind="oracle", sample=last["sample"])
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "TFLOP/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt * 1e3 / max(args.steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(), "cpu_baseline": cpu,
            "e2e": {"value": v, "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def workload_config(strong=False, world=1):
    return {"workload": "static sweep m=k=4096 n=2048 FP16, b in {1,4,8,16} x d in "
                        "{1/32,1/16,1/8,1/4}, 16 products per step",
            "m": M, "k": K, "n": N, "block_sizes": list(SWEEP_B),
            "densities": ["1/32", "1/16", "1/8", "1/4"], "mode": "static",
            "parallelism": ("row split over %d GPUs (X replicated, NCCL all-gather of the Y "
                            "slices after every product)" % world) if strong else
                           "replicas (weak)",
            "l2": "inputs larger than L2: 16 problems (~0.6 GB) each read once per step"}


# ------------------------------------------------------------------- main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-comparators", action="store_true")
    ap.add_argument("--no-dynamic", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-transposed", action="store_true")
    ap.add_argument("--no-sddmm", action="store_true")
    ap.add_argument("--no-refit", action="store_true",
                    help="skip the compact refit of the speed-up power law (m = k in {1024, "
                         "2048, 4096}, n in {1024, 4096}, every b and d; under a minute)")
    ap.add_argument("--refit-full", action="store_true",
                    help="refit on the full grid instead (m = k up to 8192, n up to 16384; a "
                         "few minutes)")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--scaling", default="weak", choices=["weak", "strong"],
                    help="weak: every rank runs the whole sweep (replicas); strong: every "
                         "product is split by rows over the ranks (X replicated) and the Y "
                         "slices are all-gathered after each product")
    ap.add_argument("--point", default=None,
                    help="run one sweep point only, 'b:1/d' e.g. 16:4 (profiling); the other "
                         "sections are then skipped unless named by --section")
    ap.add_argument("--section", action="append", default=[],
                    choices=["gather_small_n", "dynamic", "batched", "serving", "transposed",
                             "sddmm", "refit"],
                    help="with --point: also run this section (repeatable)")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)

    import torch
    from paper_2303_16999_gb300 import spmm as S
    from paper_2303_16999_gb300 import workloads as wl
    peaks, peak_src = load_peaks()
    rank, world, local = dist_setup(args.gpus)
    dev = torch.device("cuda", local)
    S.lib()
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline_leg()  # threads only, before the GPU work
    only = tuple(int(v) for v in args.point.split(":")) if args.point else None
    strong = args.scaling == "strong"
    rows = row_range(rank, world) if strong and world > 1 else None
    pts = build_points(torch, S, wl, dev, only, rows)
    gather = None
    if strong and world > 1:
        import torch.distributed as dist
        if M % (16 * world):
            raise SystemExit("--scaling strong needs m = %d to split into equal 16-row slices "
                             "over %d ranks" % (M, world))
        full = [torch.empty((M, N), dtype=torch.float16, device=dev) for _ in pts]

        def gather():
            for p, f in zip(pts, full):
                dist.all_gather_into_tensor(f, p["Y"])
    stream = torch.cuda.current_stream()

    # each product is captured once in its own CUDA graph; a step replays the
    # 16 graphs back to back with an event pair around each replay, so host
    # launch latency never enters the device timings
    cap_stream = torch.cuda.Stream()
    cap_stream.wait_stream(torch.cuda.current_stream())
    graphs = []
    with torch.cuda.stream(cap_stream):
        for _ in range(3):
            for p in pts:           # eager warm-up: module load, kernel attributes
                p["plan"].run(p["X"], p["Y"])
        cap_stream.synchronize()
        for p in pts:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=cap_stream):
                p["plan"].run(p["X"], p["Y"])
            graphs.append(g)
    torch.cuda.current_stream().wait_stream(cap_stream)

    def step(evs=None):
        for i, g in enumerate(graphs):
            if evs is not None:
                evs[i][0].record()
            g.replay()
            if evs is not None:
                evs[i][1].record()
        if gather is not None:
            gather()

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    evs = [[[torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)]
            for _ in pts] for _ in range(args.steps)]
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    try:
        bus = torch.cuda.get_device_properties(dev).pci_bus_id
    except Exception:
        bus = None
    sampler = ClockSampler(bus)
    barrier(world)
    torch.cuda.synchronize()
    with sampler:
        start.record()
        for s_ in range(args.steps):
            step(evs[s_])
        end.record()
        torch.cuda.synchronize()
    barrier(world)
    t_ms = start.elapsed_time(end)
    t_ms = max_over_ranks(t_ms, world)

    # per-launch durations over the timed steps (median per product)
    per = [statistics.median(evs[s_][i][0].elapsed_time(evs[s_][i][1])
                             for s_ in range(args.steps)) for i in range(len(pts))]
    flops_step = sum(2.0 * p["nnzb"] * p["b"] ** 2 * N for p in pts)
    if strong:
        # the whole problems once per step, whatever the number of ranks
        flops_job = sum(2.0 * p["nnzb_whole"] * p["b"] ** 2 * N for p in pts)
        value = flops_job * args.steps / (t_ms * 1e-3) / 1e12
    else:
        flops_job = flops_step * world
        value = job_throughput(flops_step, args.steps, world, t_ms * 1e-3)

    points, tc_launches = [], []
    for i, p in enumerate(pts):
        kern = {1: "plain", 2: "gather", 3: "tc", 4: "bgather"}[p["kernel"]]
        fl, by, bound, t_roof = roof_of(p["b"], p["nnzb"], peaks, kern, p["m"])
        us = per[i] * 1e3
        points.append({"b": p["b"], "d": "1/%d" % round(1 / p["d"]), "kernel": kern,
                       "us": round(us, 2),
                       "tflops_nz": round(fl / (us * 1e-6) / 1e12, 2),
                       "tflops_dense_equiv": round(2.0 * M * K * N / (us * 1e-6) / 1e12, 2),
                       "gbs_compulsory": round(by / (us * 1e-6) / 1e9, 1),
                       "bound": bound, "t_roof_us": round(t_roof * 1e6, 3),
                       "roof_frac": round(t_roof / (us * 1e-6), 3)})
        if kern == "tc":
            tc_launches.append((fl, by, us * 1e-6))
    # the dominant kernel: every product of the step runs on tc_kernel at
    # these sizes (AUTO takes b = 1 to the tensor cores at n = 2048)
    roofline = roofline_obj(tc_launches, peaks, "tensor", traffic=sweep_traffic(),
                            kernel="tc_kernel")
    roofline["share_of_step"] = round(sum(t for _, _, t in tc_launches) /
                                      max(sum(per) * 1e-3, 1e-12), 3)
    roofline["peak_source"] = "%s (MEASURED_PEAKS.json, burst)" % peak_src
    roofline["traffic_source"] = (SWEEP_TRAFFIC["source"] if roofline["traffic"] is not None
                                  else "null: no ncu capture of the current kernel sources")

    # end to end through the public API with host buffers: spmm_run_host
    # copies X in, runs, copies Y out and synchronises its own stream, so a
    # few host threads, each owning a share of the plans and its own stream,
    # let one product's copies overlap another's kernels
    workers = min(E2E_WORKERS, len(pts))
    e2e_streams = [torch.cuda.Stream(device=dev) for _ in range(workers)]

    def e2e_pass(steps):
        def work(w):
            for _ in range(steps):
                for j in range(w, len(pts), workers):
                    pts[j]["plan"].run_host(pts[j]["Xh"], pts[j]["Yh"], stream=e2e_streams[w])
        threads = [threading.Thread(target=work, args=(w,)) for w in range(workers)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()

    e2e_pass(1)   # untimed: each plan allocates its staging buffers on first use
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    e2e_pass(args.e2e_steps)
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, world)
    e2e = {"value": flops_job * args.e2e_steps / e2e_s / 1e12, "unit": "TFLOP/s",
           "h2d_bytes_per_step": sum(p["Xh"].numel() * 2 for p in pts),
           "d2h_bytes_per_step": sum(p["Yh"].numel() * 2 for p in pts),
           "steps": args.e2e_steps, "host_threads": workers}

    comparators = None
    if rank == 0 and not args.no_comparators and any(
            q["b"] == 16 and abs(q["d"] - 1 / 16) < 1e-12 for q in pts):
        comparators = run_comparators(torch, S, wl, dev, pts)

    dynamic = batched = serving = gsmall = transposed = sddmm = refit = None

    def want(name, off=False):
        return rank == 0 and not off and (args.point is None or name in args.section)
    if want("gather_small_n"):
        gsmall = run_gather_small_n(torch, S, wl, dev, peaks)
    if want("dynamic", args.no_dynamic):
        dynamic = run_dynamic(torch, S, wl, dev, peaks)
    if want("batched", args.no_batched):
        batched = run_batched(torch, S, wl, dev, peaks)
    if want("serving", args.no_serving):
        serving = run_serving(torch, S, wl, dev, peaks)
    if want("transposed", args.no_transposed):
        transposed = run_transposed(torch, S, wl, dev, peaks)
    if want("sddmm", args.no_sddmm):
        sddmm = run_sddmm(torch, S, wl, dev, peaks)
    if want("refit", args.no_refit):
        if args.refit_full:
            refit = run_refit(torch, S, wl, dev)
        else:
            refit = run_refit(torch, S, wl, dev, ms=(1024, 2048, 4096), ns=(1024, 4096))

    launches = sum(launches_per_run(p) for p in pts) * args.steps
    if rank == 0:
        line = {"metric": METRIC, "value": round(value, 3), "unit": "TFLOP/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(t_ms / args.steps, 4), "higher_is_better": True,
                "scaling": args.scaling, "vs_baseline": None, "dtype": "f16 (fp32 accumulate)",
                "data": "synthetic", "config": workload_config(strong, world),
                "e2e": e2e, "gpu_launches": launches, "clocks": sampler.summary(),
                "roofline": roofline, "cpu_baseline": cpu, "points": points,
                "comparators": comparators, "dynamic": dynamic, "batched": batched,
                "serving": serving, "gather_small_n": gsmall, "transposed": transposed,
                "sddmm": sddmm, "refit": refit}
        print(json.dumps(line))
    for p in pts:
        p["plan"].close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def graph_time_us(torch, fn, reps, inner=1):
    """Median device time of one fn() call: fn is captured ``inner`` times
    back to back in one CUDA graph (amortising launch latency for small
    kernels), the graph is replayed ``reps`` times."""
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(st):
        for _ in range(2):
            fn()
        st.synchronize()
        with torch.cuda.graph(g, stream=st):
            for _ in range(inner):
                fn()
    torch.cuda.current_stream().wait_stream(st)
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        g.replay()
        b.record()
        b.synchronize()
        ts.append(a.elapsed_time(b) * 1e3 / inner)
    return statistics.median(ts)


def run_dynamic(torch, S, wl, dev, peaks, calls=4, reps=10):
    """Dynamic mode, m = k = 8192, n = 1024, b = 16, d_max = 1/16, BF16: every
    call carries a fresh pattern (nnzb uniform in [8192, 16384]) and values,
    re-partitioned on the device.  Reports the per-call time, the
    re-partition + packing time alone (a call with n = 0), and the ratio to
    a static plan of the same pattern (the analogue of Table 3)."""
    m = k = 8192
    n = 1024
    cap = 16384
    bf = torch.bfloat16
    dplan = S.Plan(m, k, n, 16, w_dtype=S.BF16, mode=S.DYNAMIC, nnzb_max=cap)
    inputs = []
    for c in range(calls):
        cs = wl.dynamic_call(c)
        br = torch.zeros(cap, dtype=torch.int32)
        bc = torch.zeros(cap, dtype=torch.int32)
        br[:len(cs["brow"])] = torch.from_numpy(cs["brow"])
        bc[:len(cs["bcol"])] = torch.from_numpy(cs["bcol"])
        vd = torch.zeros((cap, 16, 16), dtype=bf)
        vd[:len(cs["vals"])] = torch.from_numpy(cs["vals"]).to(bf)
        inputs.append(dict(c=cs, pat=(torch.tensor([len(cs["brow"])], dtype=torch.int32, device=dev),
                                      br.to(dev), bc.to(dev)),
                           vals=vd.to(dev), X=torch.from_numpy(cs["X"]).to(bf).to(dev)))
    Y = torch.empty((m, n), dtype=bf, device=dev)
    Xe = torch.empty((k, 0), dtype=bf, device=dev)
    Ye = torch.empty((m, 0), dtype=bf, device=dev)
    flops = sum(2.0 * len(i["c"]["brow"]) * 256 * n for i in inputs)

    def calls_fn():
        for i in inputs:
            dplan.run(i["X"], Y, values=i["vals"], pattern=i["pat"])

    def part_fn():
        for i in inputs:
            dplan.run(Xe, Ye, values=i["vals"], pattern=i["pat"])

    t_dyn = graph_time_us(torch, calls_fn, reps) / calls
    t_part = graph_time_us(torch, part_fn, reps) / calls
    # the same calls with the re-partition as a chain of launches
    cplan = S.Plan(m, k, n, 16, w_dtype=S.BF16, mode=S.DYNAMIC, nnzb_max=cap, dyn_chain=True)

    def chain_fn():
        for i in inputs:
            cplan.run(i["X"], Y, values=i["vals"], pattern=i["pat"])
    t_chain = graph_time_us(torch, chain_fn, reps) / calls
    if cplan.status() != 0 or dplan.status() != 0:
        raise RuntimeError("dynamic status %d / %d" % (dplan.status(), cplan.status()))
    cplan.close()
    i0 = inputs[0]
    splan = S.Plan(m, k, n, 16, w_dtype=S.BF16, brow=i0["c"]["brow"], bcol=i0["c"]["bcol"])
    splan.pack(i0["vals"][:len(i0["c"]["brow"])].contiguous())
    t_static = graph_time_us(torch, lambda: splan.run(i0["X"], Y), reps)

    def one_dyn():
        dplan.run(i0["X"], Y, values=i0["vals"], pattern=i0["pat"])
    t_dyn0 = graph_time_us(torch, one_dyn, reps)
    fl0 = 2.0 * len(i0["c"]["brow"]) * 256 * n

    # the same calls in Blocked-ELL form (width = each pattern's longest row)
    for i in inputs:
        cols, src = wl.to_ell(i["c"]["brow"], i["c"]["bcol"], m // 16)
        ev = torch.zeros((m // 16, cols.shape[1], 16, 16), dtype=bf)
        sel = src >= 0
        ev[torch.from_numpy(sel)] = torch.from_numpy(i["c"]["vals"]).to(bf)[
            torch.from_numpy(src[sel])]
        i["ell"] = (torch.from_numpy(cols).to(dev), ev.to(dev))

    def ell_fn():
        for i in inputs:
            dplan.run_ell(i["ell"][0], i["ell"][1], i["X"], Y)
    t_ell = graph_time_us(torch, ell_fn, reps) / calls
    if dplan.status() != 0:
        raise RuntimeError("ELL status %d" % dplan.status())
    widths = [int(i["ell"][0].shape[1]) for i in inputs]
    out = {"workload": "dynamic m=k=8192 n=1024 b=16 d_max=1/16 BF16, fresh pattern per call",
           "us_per_call": round(t_dyn, 1), "tflops_nz": round(flops / calls / t_dyn / 1e6, 2),
           "repartition_pack_us": round(t_part, 1),
           "launch_chain_us_per_call": round(t_chain, 1),
           "repartition": "one cooperative launch (re-partition, packing, stage records), then "
                          "the product launch",
           "static_same_pattern_us": round(t_static, 1),
           "dynamic_same_pattern_us": round(t_dyn0, 1),
           "dynamic_over_static_time": round(t_dyn0 / t_static, 3),
           "static_tflops_nz": round(fl0 / t_static / 1e6, 2),
           "ell": {"us_per_call": round(t_ell, 1),
                   "tflops_nz": round(flops / calls / t_ell / 1e6, 2),
                   "widths": widths, "ell_over_csr_time": round(t_ell / t_dyn, 3),
                   "ell_over_static_time": round(t_ell / t_static, 3),
                   "launches_per_call": 2},
           # the cooperative re-partition, tc_kernel, reduce_kernel (it finds
           # its split rows on the device, so it is launched every call)
           "gpu_launches_per_call": 3}
    # compulsory bytes of a call: values, the pattern (8 B per block), the
    # block CSR written and read back (8 B per block each way), X and Y
    def dyn_bytes(nb):
        return nb * 256 * 2 + nb * 8 + nb * 16 + (k + m) * n * 2
    out["roofline"] = roofline_obj(
        [(2.0 * len(i["c"]["brow"]) * 256 * n, dyn_bytes(len(i["c"]["brow"])), t_dyn * 1e-6)
         for i in inputs], peaks, "tensor", kernel="dynamic call (re-partition + tc_kernel)")
    out["roofline_ell"] = roofline_obj(
        [(2.0 * len(i["c"]["brow"]) * 256 * n,
          int(i["ell"][0].numel()) * (256 * 2 + 4) + (k + m) * n * 2, t_ell * 1e-6)
         for i in inputs], peaks, "tensor", kernel="ell_kernel (padded slots read)")
    dplan.close()
    splan.close()
    return out


def run_batched(torch, S, wl, dev, peaks, reps=5):
    """48 uneven FFN-like products (W 4096 x 16384 / 16384 x 4096, b in {8, 16},
    d in {1/16, 1/8}, n log-uniform in [1, 512]) with E4M3 weights (one FP32
    scale per block) and BF16 X, in one persistent launch (CUDA graph),
    against the same 48 plans launched one after another and against the
    plain FP32 kernel run on FP32 copies, problem by problem."""
    bf = torch.bfloat16
    plans, p32, Xs, Ys, X32, Y32 = [], [], [], [], [], []
    flops = 0.0
    comp_bytes = 0
    # the autotuner: one tuning run per (b, density, n) bucket of the batch,
    # on that bucket's first problem; every plan below is AUTO and takes its
    # bucket's choice
    S.spmm_tune_clear()
    t_tune = time.perf_counter()
    tuned, seen = [], set()
    for i in range(48):
        sp = wl.batched_spec(i)
        key = (sp["m"], sp["k"], sp["b"], sp["d"], max(sp["n"] - 1, 0).bit_length())
        if key in seen:
            continue
        seen.add(key)
        c = wl.batched_case(i)
        codes, scales = S.quantize_e4m3(torch.from_numpy(c["vals"]).to(bf).to(dev))
        ld = (c["n"] + 7) // 8 * 8
        xb = torch.zeros((c["k"], ld), dtype=bf, device=dev)
        xb[:, :c["n"]] = torch.from_numpy(c["X"]).to(bf).to(dev)
        r = S.spmm_tune(c["m"], c["k"], c["b"], c["brow"], c["bcol"], codes.view(torch.uint8),
                        xb[:, :c["n"]], w_dtype=S.E4M3, x_dtype=S.BF16, scales=scales, reps=5)
        tuned.append({"m": c["m"], "k": c["k"], "b": c["b"], "d": "1/%d" % round(1 / sp["d"]),
                      "n_bucket": "(%d, %d]" % (2 ** (key[4] - 1) if key[4] else 0, 2 ** key[4]),
                      "tuned_on_n": c["n"], "choice": r["kernel"],
                      "stage_geometry": r["stage_geometry"],
                      "rows_per_group": r["rows_per_group"], "k_splits": r["k_splits"],
                      "col_tiles": r["col_tiles"],
                      "candidates": r["candidates"]})
        del codes, scales, xb
    t_tune = time.perf_counter() - t_tune
    for i in range(48):
        c = wl.batched_case(i)
        v = torch.from_numpy(c["vals"]).to(dev)
        codes, scales = S.quantize_e4m3(v.to(bf))
        p = S.Plan(c["m"], c["k"], c["n"], c["b"], w_dtype=S.E4M3, x_dtype=S.BF16,
                   brow=c["brow"], bcol=c["bcol"])
        p.pack(codes.view(torch.uint8), scales)
        n = c["n"]
        ld = (n + 7) // 8 * 8
        xb = torch.zeros((c["k"], ld), dtype=bf, device=dev)
        xb[:, :n] = torch.from_numpy(c["X"]).to(bf).to(dev)
        plans.append(p)
        Xs.append(xb[:, :n])
        Ys.append(torch.empty((c["m"], n), dtype=bf, device=dev))
        q = S.Plan(c["m"], c["k"], n, c["b"], w_dtype=S.F32, brow=c["brow"], bcol=c["bcol"],
                   kernel="plain")
        q.pack(v)
        p32.append(q)
        X32.append(xb[:, :n].float().contiguous())
        Y32.append(torch.empty((c["m"], n), dtype=torch.float32, device=dev))
        flops += 2.0 * len(c["brow"]) * c["b"] ** 2 * n
        nb = len(c["brow"])
        comp_bytes += nb * c["b"] ** 2 + 8 * nb + 4 * (c["m"] // c["b"] + 1) + \
            (c["k"] + c["m"]) * n * 2
        del v, codes, scales
    S.spmm_batch_run(plans, Xs, Ys)          # builds the cached schedule outside capture
    torch.cuda.synchronize()
    t_batch = graph_time_us(torch, lambda: S.spmm_batch_run(plans, Xs, Ys), reps)

    def seq():
        for p, x, y in zip(plans, Xs, Ys):
            p.run(x, y)
    t_seq = graph_time_us(torch, seq, reps)

    def seq32():
        for p, x, y in zip(p32, X32, Y32):
            p.run(x, y)
    t_32 = graph_time_us(torch, seq32, 2)
    infos = [p.info() for p in plans]
    w_bytes = sum(q["n_tiles"] * (256 + 64) if q["kernel"] == 3 else q["nnzb"] * (q["b"] ** 2 + 4)
                  for q in infos)
    kinds = [q["kernel"] for q in infos]
    n_bg = sum(1 for k_ in kinds if k_ == 4)
    n_red = sum(1 for q in infos if q["kernel"] == 3 and q["n_reductions"] > 0)
    wide = [q["kernel"] == 3 and q["col_tiles"] == 2 and y.shape[1] > 128 for q, y in zip(infos, Ys)]
    tc_launches = int(any(wide)) + int(any(q["kernel"] == 3 and not w for q, w in zip(infos, wide)))
    out = {"workload": "batched: 48 FFN-like products, E4M3 W + FP32 block scales, BF16 X",
           "us": round(t_batch, 1), "tflops_nz": round(flops / t_batch / 1e6, 2),
           "sequential_same_plans_us": round(t_seq, 1),
           "plain_fp32_sequential_us": round(t_32, 1),
           "speedup_vs_plain_fp32": round(t_32 / t_batch, 2),
           "speedup_vs_sequential": round(t_seq / t_batch, 3),
           "packed_weight_gb": round(w_bytes / 1e9, 3),
           "problems_on_bgather": n_bg, "problems_on_tc": len(kinds) - n_bg,
           # one BGATHER launch, one tensor-core launch per kind of CTA
           # (one or two column tiles; both stage geometries merged in each),
           # one reduction launch per split problem
           "gpu_launches": (1 if n_bg else 0) + tc_launches + n_red,
           "problems_on_tc_two_column_tiles": sum(wide),
           "tuner": {"buckets": len(tuned), "seconds": round(t_tune, 1), "table": tuned}}
    # the batch call as one unit: its roofline is that of all 48 problems
    # together, compulsory bytes = E4M3 values + one FP32 scale and one int32
    # column per block + row pointers + X once + Y once (BF16)
    out["roofline"] = roofline_obj([(flops, comp_bytes, t_batch * 1e-6)], peaks, "tensor",
                                   kernel="batch call: bgather_kernel (%d problems) + tc_kernel "
                                          "(%d problems), E4M3 weights" % (n_bg, len(kinds) - n_bg))
    for p in plans + p32:
        p.close()
    return out


def run_serving(torch, S, wl, dev, peaks, per_rate=4000,
                rates=(0.1, 0.25, 0.5, 0.75, 0.9, 1.0, 1.2)):
    """12 resident weights (m = k in {2048, 4096, 8192} x b in {8, 16} x 2
    seeds, d = 1/16, FP16); Poisson requests, n log-uniform in [1, 256],
    aimed uniformly at the weights.  Saturation throughput is measured with a
    closed burst, then each rate runs ``per_rate`` requests; the plain FP32
    kernel (one request per launch) serves the same streams as the baseline."""
    ws = wl.serve_weights()

    def make_server(fp32):
        srv = S.Server(hbm_budget_bytes=2 << 30, max_inflight=4, max_batch=64, max_batch_n=4096)
        plans, ids, xpool, ypool = [], [], [], []
        for w in ws:
            m, b = w["m"], w["b"]
            v = torch.from_numpy(w["vals"])
            if fp32:
                p = S.Plan(m, m, 256, b, w_dtype=S.F32, brow=w["brow"], bcol=w["bcol"],
                           kernel="plain")
                p.pack(v.to(dev))
                dt = torch.float32
            else:
                p = S.Plan(m, m, 256, b, w_dtype=S.F16, brow=w["brow"], bcol=w["bcol"])
                p.pack(v.half().to(dev))
                dt = torch.float16
            plans.append(p)
            ids.append(srv.register(p))
            xpool.append(torch.from_numpy(wl.request_x(w["seed"], m, 256)).to(dt).pin_memory())
            ypool.append(torch.empty((m, 256), dtype=dt).pin_memory())
        return srv, plans, ids, xpool, ypool

    def flat(t, rows, n):
        return t.view(-1)[:rows * n].view(rows, n)

    def run_stream(srv, ids, xpool, ypool, t_arr, wsel, ns):
        # native trace replay: submission times are kept by the library, not
        # by this interpreter; request contents do not matter for timing, so
        # every request of a weight reads one pinned X and writes one pinned Y
        return srv.replay(t_arr, [ids[w] for w in wsel], ns,
                          [xpool[w].data_ptr() for w in wsel], [ypool[w].data_ptr() for w in wsel])

    out = {"workload": "serving: 12 resident weights m=k in {2048,4096,8192}, b in {8,16}, "
                       "d=1/16, FP16; Poisson requests n log-uniform [1,256]"}
    for name, fp32 in (("tc_fp16", False), ("plain_fp32", True)):
        srv, plans, ids, xpool, ypool = make_server(fp32)
        # saturation: a closed burst of requests submitted at once
        tb, wb, nb = wl.serve_requests(per_rate, 1e9, len(ws), 4090)
        sat = run_stream(srv, ids, xpool, ypool, tb * 0, wb, nb)
        lam = sat["throughput_rps"]
        rows = []
        for ri, f in enumerate(rates):
            t_arr, wsel, ns = wl.serve_requests(per_rate, max(lam * f, 1.0), len(ws), 4000 + ri)
            st = run_stream(srv, ids, xpool, ypool, t_arr, wsel, ns)
            rows.append({"rate_x_sat": f, "offered_rps": round(lam * f, 1),
                         "p50_us": round(st["p50_us"], 1), "p99_us": round(st["p99_us"], 1),
                         "throughput_rps": round(st["throughput_rps"], 1),
                         "tflops_nz": round(st["tflops_nz"], 3),
                         "mean_requests_per_launch": round(st["mean_requests_per_launch"], 2)})
        out[name] = {"saturation_rps": round(lam, 1), "saturation_tflops_nz": round(sat["tflops_nz"], 3),
                     "rates": rows}
        # the burst's roofline: every request's nonzero FLOPs against the
        # tensor peak (FP32 lanes for the plain kernel), and as compulsory
        # bytes each weight read once for the whole burst plus every
        # request's X and Y once (host-link time not counted)
        es = 4 if fp32 else 2
        used = set(int(w) for w in wb)
        fl = sum(2.0 * len(ws[w]["brow"]) * ws[w]["b"] ** 2 * int(nn) for w, nn in zip(wb, nb))
        by = sum(len(ws[w]["brow"]) * (ws[w]["b"] ** 2 * es + 4) + 4 * (ws[w]["m"] // ws[w]["b"] + 1)
                 for w in used)
        by += sum((ws[w]["k"] + ws[w]["m"]) * int(nn) * es for w, nn in zip(wb, nb))
        out[name]["roofline_saturation"] = roofline_obj(
            [(fl, by, len(wb) / max(lam, 1e-9))], peaks, "alu" if fp32 else "tensor",
            kernel="serving loop at saturation (%d requests)" % len(wb))
        srv.close()
        for p in plans:
            p.close()
    return out


def run_gather_small_n(torch, S, wl, dev, peaks, reps=15):
    """The b = 1 gather kernel (CUDA cores) at small n, where it is bound by
    HBM: m = k = 16384, d = 1/16 (16.8 M non-zeros: 34 MB of FP16 values and
    34 MB of 16-bit or 67 MB of int32 column indices), FP16.  Each timed run
    follows a 256 MB write and read-back that evict L2 (the read-back lets
    the written lines drain first); the events bracket the product alone.
    Compulsory bytes (values, the indices the kernel reads, row pointers, X
    once, Y once) over the measured time, against the measured HBM copy
    bandwidth."""
    m = k = 16384
    nnzb = wl.nnzb_for(m, k, 1, 1 / 16)
    c = wl.problem(7, m, k, 32, 1, nnzb)
    plan = S.Plan(m, k, 32, 1, w_dtype=S.F16, brow=c["brow"], bcol=c["bcol"], kernel="gather")
    plan.pack(torch.from_numpy(c["vals"].reshape(-1)).half().to(dev))
    # bytes per column index each point's kernel reads: the plan's 16-bit
    # copy where X stays in shared memory (n = 1 and 4 at this k), else int32
    ib16 = plan.info()["index_bytes"]

    def idx_bytes(n):
        return ib16 if n in (1, 4) else 4
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    out = []
    for n in (1, 4, 16, 32):
        X = torch.from_numpy(c["X"][:, :n].copy()).half().to(dev)
        Y = torch.empty((m, n), dtype=torch.float16, device=dev)
        for _ in range(3):
            plan.run(X, Y)
        ts = []
        for _ in range(reps):
            # evict L2: write a buffer twice its size, then read it back, so
            # the dirty lines are written back before the timed launch
            flush.zero_()
            flush.max()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            plan.run(X, Y)
            b.record()
            b.synchronize()
            ts.append(a.elapsed_time(b) * 1e3)
        us = statistics.median(ts)
        by = nnzb * 2 + nnzb * idx_bytes(n) + (m + 1) * 4 + (k + m) * n * 2
        gbs = by / us / 1e3
        out.append({"n": n, "us": round(us, 2), "gbs": round(gbs, 1), "index_bytes": idx_bytes(n),
                    "frac_of_hbm": round(gbs / peaks["hbm_gbs"], 3),
                    "tflops_nz": round(2.0 * nnzb * n / us / 1e6, 3)})
    plan.close()
    del flush
    launches = [(2.0 * nnzb * q["n"],
                 nnzb * 2 + nnzb * q["index_bytes"] + (m + 1) * 4 + (k + m) * q["n"] * 2,
                 q["us"] * 1e-6) for q in out]
    return {"workload": "b=1 gather kernel, m=k=16384, d=1/16 (16.8 M non-zeros), FP16, small n; "
                        "L2 evicted (256 MB written and read back) before every timed run",
            "points": out,
            "roofline_n1": dict(roofline_obj(launches[:1], peaks, "alu", traffic=gather_traffic(),
                                             kernel="gather1_kernel n=1"),
                                traffic_source=GATHER_TRAFFIC["source"]
                                if gather_traffic() is not None else None),
            "roofline": roofline_obj(launches, peaks, "alu", kernel="gather kernels n in {1,4,16,32}")}


def run_transposed(torch, S, wl, dev, peaks, reps=15,
                   cases=((16, 1 / 16), (16, 1 / 4), (8, 1 / 16), (4, 1 / 16), (1, 1 / 16))):
    """Z = W^T.Y against Y = W.X on the same W (sweep points, m = k = 4096,
    n = 2048, FP16; the sweep's X serves as Y).  Both plans run from cold L2
    (256 MB written and read back before every timed run); the events
    bracket the product alone."""
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    out, tr_launches = [], []
    for b, d in cases:
        c = wl.sweep_case(b, d)
        vals = torch.from_numpy(c["vals"]).half().to(dev)
        X = torch.from_numpy(c["X"]).half().to(dev)
        Y = torch.empty((M, N), dtype=torch.float16, device=dev)
        row = {"b": b, "d": "1/%d" % round(1 / d)}
        for name, tr in (("forward", False), ("transposed", True)):
            plan = S.Plan(M, K, N, b, w_dtype=S.F16, brow=c["brow"], bcol=c["bcol"],
                          transposed=tr)
            plan.pack(vals)
            for _ in range(3):
                plan.run(X, Y)
            ts = []
            for _ in range(reps):
                flush.zero_()
                flush.max()
                a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                plan.run(X, Y)
                e.record()
                e.synchronize()
                ts.append(a.elapsed_time(e) * 1e3)
            if plan.status() != 0:
                raise RuntimeError("plan status %d" % plan.status())
            us = statistics.median(ts)
            row[name] = {"us": round(us, 2), "kernel": {1: "plain", 2: "gather", 3: "tc", 4: "bgather"}[
                plan.info()["kernel"]],
                "tflops_nz": round(2.0 * len(c["brow"]) * b * b * N / us / 1e6, 2)}
            plan.close()
        row["transposed_over_forward_time"] = round(row["transposed"]["us"] /
                                                    row["forward"]["us"], 3)
        out.append(row)
        fl, by, _, _ = roof_of(b, len(c["brow"]), peaks, "tc")
        tr_launches.append((fl, by, row["transposed"]["us"] * 1e-6))
        del vals, X, Y
    del flush
    return {"workload": "Z = W^T.Y vs Y = W.X on one W, m=k=4096, n=2048, FP16; L2 evicted "
                        "(256 MB written and read back) before every timed run", "points": out,
            "roofline": roofline_obj(tr_launches, peaks, "tensor",
                                     kernel="transposed products (square W: same bytes)")}


def run_sddmm(torch, S, wl, dev, peaks, reps=10,
              cases=((16, 1 / 16), (16, 1 / 4), (8, 1 / 16), (4, 1 / 16), (1, 1 / 16))):
    """The sampled product dW = (dY.X^T) on the block mask, m = k = 4096,
    n = 2048, BF16 inputs, FP32 dW; each timed run follows an L2 eviction
    (256 MB written and read back) and the events bracket the call alone.
    Useful FLOPs 2 nnzb b^2 n; the dense-tile kernel computes every 128 x 256
    tile, so its roofline is the tensor peak on 2 m k n (reported for both
    forms as the dense-equivalent rate)."""
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    out, sd_launches = [], []
    for b, d in cases:
        c = wl.sddmm_problem(sweep_seed_sd(b, d), M, K, N, b, wl.nnzb_for(M, K, b, d))
        dY = torch.from_numpy(c["dY"]).bfloat16().to(dev)
        X = torch.from_numpy(c["X"]).bfloat16().to(dev)
        plan = S.Plan(M, K, N, b, w_dtype=S.BF16, brow=c["brow"], bcol=c["bcol"])
        dW = torch.empty((len(c["brow"]), b, b), dtype=torch.float32, device=dev)
        for _ in range(3):
            plan.sddmm(dY, X, dW)
        ts = []
        for _ in range(reps):
            flush.zero_()
            flush.max()
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            plan.sddmm(dY, X, dW)
            e.record()
            e.synchronize()
            ts.append(a.elapsed_time(e) * 1e3)
        if plan.status() != 0:
            raise RuntimeError("plan status %d" % plan.status())
        us = statistics.median(ts)
        dense = 2.0 * M * K * N / us / 1e6
        gathered = plan.info()["sddmm_form"] == 1
        row = {"b": b, "d": "1/%d" % round(1 / d),
               "kernel": "sddmm_gather" if gathered else "sddmm_dense", "us": round(us, 2),
               "tflops_nz": round(2.0 * len(c["brow"]) * b * b * N / us / 1e6, 2)}
        if gathered:
            # rows moved from L2: each block's 16 X rows plus one block row of
            # dY per item of up to 8 blocks (items counted as in the kernel)
            counts = np.bincount(c["brow"], minlength=M // 16)
            items = int(np.sum((counts + 7) // 8))
            moved = (len(c["brow"]) + items) * 16 * N * 2
            row["l2_to_sm_tbs"] = round(moved / us / 1e6, 2)
        else:
            row["tflops_dense_equiv"] = round(dense, 1)
            row["frac_of_tensor_peak"] = round(dense / peaks["bf16_tflops"], 3)
        # useful work: 2 nnzb b^2 n FLOPs; compulsory bytes dY and X once
        # (BF16) and dW once (FP32)
        fl_u = 2.0 * len(c["brow"]) * b * b * N
        by_u = (M + K) * N * 2 + len(c["brow"]) * b * b * 4 + len(c["brow"]) * 8
        t_r, bd = roof_time(fl_u, by_u, peaks, "tensor")
        row["bound"] = bd
        row["roof_frac"] = round(t_r / (us * 1e-6), 3)
        sd_launches.append((fl_u, by_u, us * 1e-6))
        out.append(row)
        plan.close()
        del dY, X, dW
    del flush
    return {"workload": "dW = (dY.X^T) on the block mask, m=k=4096, n=2048, BF16 in, FP32 out; "
                        "L2 evicted before every timed run", "points": out,
            "roofline": roofline_obj(sd_launches, peaks, "tensor",
                                     kernel="sddmm kernels (useful FLOPs)")}


def fit_power_law(rows):
    """Least squares in log space: log S = log c + alpha log m + beta log d +
    gamma log b over rows (m, d, b, S), the form of the speed-up model of
    Section 5 ("Will my application speed up?").  Returns (c, alpha, beta,
    gamma, r2)."""
    A = np.array([[1.0, math.log(m), math.log(d), math.log(b)] for m, d, b, _ in rows])
    y = np.array([math.log(r[3]) for r in rows])
    coef, *_ = np.linalg.lstsq(A, y, rcond=None)
    res = y - A @ coef
    tot = y - y.mean()
    r2 = 1.0 - float(res @ res) / float(tot @ tot) if float(tot @ tot) > 0 else 1.0
    return math.exp(coef[0]), float(coef[1]), float(coef[2]), float(coef[3]), r2


def run_refit(torch, S, wl, dev, ms=(1024, 2048, 4096, 8192), ns=(256, 1024, 4096, 16384),
              bs=(1, 4, 8, 16), ds=(1 / 32, 1 / 16, 1 / 8, 1 / 4), reps=5):
    """The paper's static sweep on this GPU (Table 2's m = k, n, b, d grid,
    FP16): speed-up S = best-over-n sparse TFLOP/s / best-over-n dense
    TFLOP/s, both counting the useful 2 m k n d FLOPs, i.e. cuBLAS dense
    time over sparse time at each side's best n; then the power law of
    Section 5 refitted to S, the largest density with S > 1 per (b, m), and
    cuSPARSE CSR / BSR context at m = k = 4096, n = 2048, d = 1/16 (the
    library's generic SpMM called directly).  Timed
    with CUDA events (median of reps after two warm-up runs), L2 warm on
    both sides alike."""
    def med_us(fn):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            e.record()
            e.synchronize()
            ts.append(a.elapsed_time(e) * 1e3)
        return statistics.median(ts)

    t0 = time.perf_counter()
    rows, grid = [], []
    for m in ms:
        rng = np.random.default_rng(m)
        Xs = {n: torch.from_numpy(rng.standard_normal((m, n), dtype=np.float32)).half().to(dev)
              for n in ns}
        Ys = {n: torch.empty((m, n), dtype=torch.float16, device=dev) for n in ns}
        Wd = torch.from_numpy(rng.standard_normal((m, m), dtype=np.float32)).half().to(dev)
        dense = max(2.0 * m * m * n / med_us(lambda: torch.matmul(Wd, Xs[n], out=Ys[n])) / 1e6
                    for n in ns)
        del Wd
        for b in bs:
            for d in ds:
                c = wl.problem(90000 + m + 100 * b + int(round(1 / d)), m, m, 0, b,
                               wl.nnzb_for(m, m, b, d))
                plan = S.Plan(m, m, max(ns), b, w_dtype=S.F16, brow=c["brow"], bcol=c["bcol"])
                plan.pack(torch.from_numpy(c["vals"]).half().to(dev))
                best, best_n = 0.0, 0
                for n in ns:
                    us = med_us(lambda: plan.run(Xs[n], Ys[n]))
                    tf = 2.0 * len(c["brow"]) * b * b * n / us / 1e6
                    if tf > best:
                        best, best_n = tf, n
                if plan.status() != 0:
                    raise RuntimeError("plan status %d" % plan.status())
                plan.close()
                sp = best / (d * dense)
                rows.append((m, d, b, sp))
                grid.append({"m": m, "b": b, "d": "1/%d" % round(1 / d),
                             "sparse_tflops_nz": round(best, 2), "best_n": best_n,
                             "dense_tflops": round(dense, 1), "speedup": round(sp, 3)})
        del Xs, Ys
    cfit, al, be, ga, r2 = fit_power_law(rows)
    thresholds = {}
    for label, bset in (("b=1", (1,)), ("b>=4", (4, 8, 16)), ("b>=8", (8, 16))):
        for m in ms:
            ok = [d for d in ds if all(sp > 1.0 for (mm, dd, bb, sp) in rows
                                      if mm == m and dd == d and bb in bset)]
            thresholds["%s, m=k=%d" % (label, m)] = ("d <= 1/%d" % round(1 / max(ok))) if ok else None
    context = {}
    try:
        m, n, d = 4096, 2048, 1 / 16
        lib = _cusparse()
        X = torch.from_numpy(np.random.default_rng(5).standard_normal((m, n), dtype=np.float32))
        Xd = X.half().cuda()
        for b, label in ((1, "cusparse_csr_fp16"), (16, "cusparse_bsr_fp16")):
            c = wl.problem(777 + b, m, m, 0, b, wl.nnzb_for(m, m, b, d))
            try:
                if lib is None:
                    raise RuntimeError("libcusparse.so.12 not found")
                us = cusparse_spmm_us(torch, lib, m, m, n, b, c["brow"], c["bcol"],
                                      torch.from_numpy(c["vals"]).half(), Xd)
                context[label] = {"us": round(us, 1),
                                  "tflops_nz": round(2.0 * len(c["brow"]) * b * b * n / us / 1e6, 2)}
            except Exception as ex:  # context only
                context[label] = "unavailable: %s" % str(ex).splitlines()[0][:160]
        context["point"] = "m=k=4096, n=2048, d=1/16, FP16 values and X, FP32 compute"
        context["call"] = "cusparseSpMM (generic API; CSR default algorithm, BSR_ALG1)"
    except Exception as ex:  # context only: never fail the benchmark over it
        context["error"] = str(ex).splitlines()[0][:200]
    return {"workload": "static sweep m=k in %s, n in %s (best over n), b in %s, d in %s, FP16; "
                        "speed-up = sparse TFLOP/s / dense (cuBLAS) TFLOP/s, useful FLOPs both"
                        % (list(ms), list(ns), list(bs), ["1/%d" % round(1 / v) for v in ds]),
            "fit": {"c": cfit, "alpha_m": round(al, 3), "beta_d": round(be, 3),
                    "gamma_b": round(ga, 3), "r2": round(r2, 3),
                    "condition": "%.3g * m^%.2f * d^%.2f * b^%.2f > 1" % (cfit, al, be, ga)},
            "thresholds": thresholds, "grid": grid, "cusparse_context": context,
            "seconds": round(time.perf_counter() - t0, 1)}


def _cusparse():
    """libcusparse through ctypes (context numbers only; None if absent)."""
    import glob
    cands = ["libcusparse.so.12", "/usr/local/cuda/lib64/libcusparse.so.12"]
    cands += glob.glob("/usr/local/cuda*/targets/*/lib/libcusparse.so.12")
    for c in cands:
        try:
            return ctypes.CDLL(c)
        except OSError:
            continue
    return None


def cusparse_spmm_us(torch, lib, m, k, n, b, brow, bcol, vals, X, reps=10):
    """Median time of one cusparseSpMM call (generic API, FP16 values and
    X, FP32 compute, row-major dense operands) with W in CSR (b = 1) or BSR
    (b > 1, row-major blocks) form, on torch's current stream.  Context
    for the paper's GPU comparison system (Section 5), not part of the
    product."""
    vp = ctypes.c_void_p
    i64 = ctypes.c_int64
    order = np.lexsort((bcol, brow))
    mb = m // b
    rp = np.zeros(mb + 1, np.int32)
    np.add.at(rp, np.asarray(brow, np.int64) + 1, 1)
    rp = np.cumsum(rp).astype(np.int32)
    d_rp = torch.from_numpy(rp).cuda()
    d_ci = torch.from_numpy(np.asarray(bcol, np.int32)[order]).cuda()
    d_v = vals[torch.from_numpy(order)].contiguous().cuda()
    Y = torch.empty((m, n), dtype=torch.float16, device="cuda")
    h, A, Bd, Cd = vp(), vp(), vp(), vp()
    chk = []

    def ok(st, what):
        if st != 0:
            raise RuntimeError("%s returned %d" % (what, st))
    ok(lib.cusparseCreate(ctypes.byref(h)), "cusparseCreate")
    try:
        ok(lib.cusparseSetStream(h, vp(torch.cuda.current_stream().cuda_stream)), "SetStream")
        R16F, R32F, I32, BASE0, ROW = 2, 0, 2, 0, 2
        if b == 1:
            ok(lib.cusparseCreateCsr(ctypes.byref(A), i64(m), i64(k), i64(len(brow)),
                                     vp(d_rp.data_ptr()), vp(d_ci.data_ptr()),
                                     vp(d_v.data_ptr()), I32, I32, BASE0, R16F), "CreateCsr")
            alg = 0
        else:
            ok(lib.cusparseCreateBsr(ctypes.byref(A), i64(mb), i64(k // b), i64(len(brow)),
                                     i64(b), i64(b), vp(d_rp.data_ptr()), vp(d_ci.data_ptr()),
                                     vp(d_v.data_ptr()), I32, I32, BASE0, R16F, ROW),
               "CreateBsr")
            alg = 14   # CUSPARSE_SPMM_BSR_ALG1
        ok(lib.cusparseCreateDnMat(ctypes.byref(Bd), i64(k), i64(n), i64(n),
                                   vp(X.data_ptr()), R16F, ROW), "CreateDnMat B")
        ok(lib.cusparseCreateDnMat(ctypes.byref(Cd), i64(m), i64(n), i64(n),
                                   vp(Y.data_ptr()), R16F, ROW), "CreateDnMat C")
        one, zero = ctypes.c_float(1.0), ctypes.c_float(0.0)
        sz = ctypes.c_size_t()
        ok(lib.cusparseSpMM_bufferSize(h, 0, 0, ctypes.byref(one), A, Bd, ctypes.byref(zero), Cd,
                                       R32F, alg, ctypes.byref(sz)), "SpMM_bufferSize")
        buf = torch.empty(max(int(sz.value), 16), dtype=torch.uint8, device="cuda")

        def call():
            ok(lib.cusparseSpMM(h, 0, 0, ctypes.byref(one), A, Bd, ctypes.byref(zero), Cd, R32F,
                                alg, vp(buf.data_ptr())), "SpMM")
        for _ in range(2):
            call()
        torch.cuda.synchronize()
        for _ in range(reps):
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            call()
            e.record()
            e.synchronize()
            chk.append(a.elapsed_time(e) * 1e3)
    finally:
        for d, f in ((A, "cusparseDestroySpMat"), (Bd, "cusparseDestroyDnMat"),
                     (Cd, "cusparseDestroyDnMat")):
            if d.value:
                getattr(lib, f)(d)
        lib.cusparseDestroy(h)
    return statistics.median(chk)


def sweep_seed_sd(b, d):
    return 7000 + 10 * b + int(round(math.log2(1 / d)))


def run_comparators(torch, S, wl, dev, pts):
    """Context on the same GPU for b = 16, d = 1/16: the plain FP32 kernel on
    FP32 copies of the inputs, and cuBLAS dense FP16 GEMM on the densified W."""
    p = next(q for q in pts if q["b"] == 16 and abs(q["d"] - 1 / 16) < 1e-12)
    c = p["c"]
    out = {}

    def timeit(fn, reps=20):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ts = []
        for _ in range(reps):
            a.record()
            fn()
            b.record()
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts) * 1e3

    fl = 2.0 * p["nnzb"] * 256 * N
    plan32 = S.Plan(M, K, N, 16, w_dtype=S.F32, brow=c["brow"], bcol=c["bcol"], kernel="plain")
    plan32.pack(torch.from_numpy(c["vals"]).half().float().to(dev))
    X32 = p["X"].float()
    Y32 = torch.empty((M, N), dtype=torch.float32, device=dev)
    us = timeit(lambda: plan32.run(X32, Y32))
    out["plain_fp32_kernel"] = {"us": round(us, 1), "tflops_nz": round(fl / us / 1e6, 3)}
    plan32.close()
    Wd = torch.zeros((M, K), dtype=torch.float16, device=dev)
    v = torch.from_numpy(c["vals"]).half().to(dev)
    r = torch.from_numpy(c["brow"]).long().to(dev)
    cc = torch.from_numpy(c["bcol"]).long().to(dev)
    Wd.view(M // 16, 16, K // 16, 16).permute(0, 2, 1, 3)[r, cc] = v
    us = timeit(lambda: torch.matmul(Wd, p["X"]))
    out["cublas_dense_fp16"] = {"us": round(us, 1), "tflops_nz": round(fl / us / 1e6, 2),
                                "tflops_dense": round(2.0 * M * K * N / us / 1e6, 1)}
    out["point"] = "b=16, d=1/16, m=k=4096, n=2048"
    # AUTO's kernel for b = 1 at n = 2048: the CUDA-core gather kernel against
    # the tensor-core plan the sweep runs, same pattern, values and X (warm L2)
    b1 = []
    for q in pts:
        if q["b"] != 1 or q["m"] != M:    # (row-split plans cover a slice of Y)
            continue
        cq = q["c"]
        pg = S.Plan(M, K, N, 1, w_dtype=S.F16, brow=cq["brow"], bcol=cq["bcol"], kernel="gather")
        pg.pack(torch.from_numpy(cq["vals"].reshape(-1)).half().to(dev))
        Yg = torch.empty((M, N), dtype=torch.float16, device=dev)
        g_us = timeit(lambda: pg.run(q["X"], Yg), reps=5)
        t_us = timeit(lambda: q["plan"].run(q["X"], q["Y"]), reps=5)
        b1.append({"d": "1/%d" % round(1 / q["d"]), "gather_us": round(g_us, 1),
                   "tc_us": round(t_us, 1), "auto": {2: "gather", 3: "tc"}[q["kernel"]]})
        pg.close()
    out["b1_gather_vs_tc_n2048"] = b1
    return out


if __name__ == "__main__":
    sys.exit(main())
