"""The benchmark's multi-rank logic on CPU: two gloo ranks (the GPU launch
uses NCCL over one process per GPU; every GPU run here has one GPU).
Checks the barrier, the max-over-ranks timing, the whole-job throughput
and that the reference arm prints on rank 0 only."""
import importlib.util
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    b = _bench()
    b.barrier(world)
    t = 1.0 + rank                       # rank 1 is the slow one
    tmax = b.max_over_ranks(t, world, device="cpu")
    value = b.job_throughput(2.0e12, 3, world, tmax)
    out[rank] = (tmax, value)
    b.barrier(world)
    dist.destroy_process_group()


def test_two_gloo_ranks():
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as man:
        out = man.dict()
        mp.start_processes(_rank, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
        res = dict(out)
    assert res[0][0] == res[1][0] == 2.0                  # max over ranks
    assert res[0][1] == res[1][1] == pytest.approx(6.0)   # 2 ranks x 3 steps x 2 TFLOP / 2 s


def test_single_rank_is_identity():
    b = _bench()
    assert b.max_over_ranks(1.5, 1) == 1.5
    assert b.job_throughput(1e12, 4, 1, 2.0) == pytest.approx(2.0)


@pytest.mark.parametrize("rank,prints", [("0", True), ("1", False)])
def test_reference_arm_prints_on_rank0_only(rank, prints):
    env = dict(os.environ, RANK=rank, WORLD_SIZE="2", LOCAL_RANK=rank)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0", "--gpus", "2"],
                       env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert bool(lines) == prints
    if prints:
        import json
        d = json.loads(lines[-1])
        assert d["impl"] == "reference" and d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"


def test_power_law_fit_recovers_exponents():
    """The speed-up model refit: exact power-law data gives back its
    coefficient and exponents, and R^2 = 1."""
    bench = _bench()
    rows = []
    for m in (1024, 2048, 4096, 8192):
        for d in (1 / 32, 1 / 16, 1 / 8, 1 / 4):
            for b in (1, 4, 8, 16):
                rows.append((m, d, b, 0.0013 * m ** 0.59 * d ** -0.54 * b ** 0.50))
    c, al, be, ga, r2 = bench.fit_power_law(rows)
    assert abs(c - 0.0013) < 1e-9 and abs(al - 0.59) < 1e-9
    assert abs(be + 0.54) < 1e-9 and abs(ga - 0.50) < 1e-9 and abs(r2 - 1.0) < 1e-12


def test_roofline_fraction_is_recomputable():
    """frac = sum of per-launch roofline times (max(FLOP / P_tensor,
    bytes / P_hbm)) over the sum of measured times; the object carries both
    sums, and the bound is the roof that holds most of the roofline time."""
    bench = _bench()
    peaks = {"hbm_gbs": 1000.0, "bf16_tflops": 100.0}
    # launch 1: tensor-bound, t_roof = 1e12 / 1e14 = 10 ms; launch 2: HBM-bound,
    # t_roof = 5e9 / 1e12 = 5 ms; measured 20 ms and 25 ms
    r = bench.roofline_obj([(1e12, 1e9, 0.020), (1e9, 5e9, 0.025)], peaks, "tensor")
    assert r["t_roof_us"] == pytest.approx(15000.0)
    assert r["t_meas_us"] == pytest.approx(45000.0)
    assert r["frac"] == pytest.approx(r["t_roof_us"] / r["t_meas_us"], abs=1e-4)
    assert r["bound"] == "tensor" and r["peak"] == 100.0
    assert r["achieved"] == pytest.approx(r["frac"] * r["peak"], abs=0.01)
    assert r["roof_share"] == {"tensor": pytest.approx(2 / 3, abs=1e-3),
                               "hbm": pytest.approx(1 / 3, abs=1e-3)}


def test_sweep_traffic_only_for_the_captured_sources():
    """DRAM traffic from an ncu capture is reported only while the kernel and
    planner sources hash to the captured value."""
    bench = _bench()
    saved = dict(bench.SWEEP_TRAFFIC)
    try:
        bench.SWEEP_TRAFFIC.update(sha16=bench.kernel_source_sha16(), bytes_per_launch=123.0)
        assert bench.sweep_traffic() == 123.0
        bench.SWEEP_TRAFFIC.update(sha16="0" * 16)
        assert bench.sweep_traffic() is None
    finally:
        bench.SWEEP_TRAFFIC.clear()
        bench.SWEEP_TRAFFIC.update(saved)


def test_strong_scaling_row_ranges_match_the_oracle_split():
    """The benchmark's per-rank rows (strong scaling) are the oracle's row
    split of m on the 16-row grid, for the rank counts the benchmark takes."""
    from oracle import plan as P
    bench = _bench()
    for world in (1, 2, 3, 4, 8):
        assert [bench.row_range(r, world) for r in range(world)] == P.row_split(4096, 1, world)
