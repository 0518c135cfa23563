"""Row-split sharding on CPU (the multi-GPU form of the product: each
worker owns a slice of W's rows and the whole of X, Section 3.2's
distribution of the non-zeros over workers).

* Host-only slice plans against the oracle's plan of the same slice, bit
  for bit (block CSR, items, tile structure, the index of each kept block
  in the whole pattern).
* Two gloo ranks: each plans its slice (checked as above) and computes its
  rows with the oracle on integer operands; the all-gathered rows equal the
  whole product bit for bit.
* The option's errors.
"""
import os
import socket

import numpy as np
import pytest

import oracle
from oracle import plan as P
from paper_2303_16999_gb300 import spmm as S
from paper_2303_16999_gb300 import workloads as wl

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

TC_KEYS = ["grp_row0", "grp_rows", "grp_ebeg", "ent_col", "ent_tbeg", "ent_cover", "tile_row",
           "blk_slot", "blk_off", "ws_row0"]


def check_slice_plan(m, k, n, b, brow, bcol, rb, re, kernel):
    """A host-only plan of rows [rb, re) against the oracle's plan of the
    slice; returns the oracle's slice (brow, bcol, src_index)."""
    p = S.Plan(m, k, n, b, brow=brow, bcol=bcol, kernel=kernel, host_only=True, rows=(rb, re))
    info = p.info()
    sb, sc, src = P.row_slice(brow, bcol, b, rb, re)
    assert info["m"] == re - rb and info["nnzb"] == len(sb)
    assert (info["row_begin"], info["row_end"]) == (rb, re)
    assert np.array_equal(p.array("src_index"), src)
    rp, ci, pm = P.csr((re - rb) // b, sb, sc)
    assert np.array_equal(p.array("row_ptr"), rp)
    assert np.array_equal(p.array("col_idx"), ci)
    assert np.array_equal(p.array("perm"), pm)
    if info["kernel"] == 3:   # TC
        want = P.tc_plan(re - rb, k, b, sb, sc, info["rows_per_group"], info["max_per_item"],
                         groups=info["n_groups"])
        for key in TC_KEYS:
            assert np.array_equal(p.array(key), want[key]), key
    else:
        want = P.row_plan((re - rb) // b, rp, info["max_per_item"], sort_items=True)
    assert np.array_equal(p.array("items").reshape(-1, 6), want["items"])
    assert np.array_equal(p.array("red").reshape(-1, 3), want["red"])
    p.close()
    return sb, sc, src


@pytest.mark.parametrize("b,kernel", [(16, "tc"), (8, "tc"), (4, "tc"), (1, "tc"), (1, "gather")])
@pytest.mark.parametrize("workers", [2, 3, 8])
def test_slice_plans_bit_exact(b, kernel, workers):
    m, k, n = 1024, 512, 256
    c = wl.problem(600 + b, m, k, 0, b, wl.nnzb_for(m, k, b, 1 / 8))
    seen = []
    for rb, re in P.row_split(m, b, workers):
        _, _, src = check_slice_plan(m, k, n, b, c["brow"], c["bcol"], rb, re, kernel)
        seen.append(src)
    # every block of the whole pattern is kept by exactly one slice
    allsrc = np.concatenate(seen)
    assert np.array_equal(np.sort(allsrc), np.arange(len(c["brow"])))


def test_row_split_ranges():
    assert P.row_split(4096, 16, 2) == [(0, 2048), (2048, 4096)]
    assert P.row_split(96, 16, 4) == [(0, 32), (32, 64), (64, 80), (80, 96)]
    r = P.row_split(4096, 1, 3)
    assert r[0][0] == 0 and r[-1][1] == 4096 and all(a % 16 == 0 for a, _ in r)


def test_slice_option_errors():
    brow = np.array([0, 5, 9], np.int32)
    bcol = np.array([1, 2, 3], np.int32)
    for rows, code in (((0, 0 + 8), S.ERR_SHAPE), ((16, 8), S.ERR_SHAPE), ((0, 4096), S.ERR_SHAPE),
                       ((-16, 16), S.ERR_SHAPE)):
        with pytest.raises(S.SpmmError) as e:
            S.Plan(256, 256, 64, 16, brow=brow, bcol=bcol, host_only=True, rows=rows)
        assert e.value.status == code, rows
    # a repeated block outside the slice is still an error of the pattern
    with pytest.raises(S.SpmmError) as e:
        S.Plan(256, 256, 64, 16, brow=np.array([0, 9, 9], np.int32),
               bcol=np.array([1, 3, 3], np.int32), host_only=True, rows=(0, 64))
    assert e.value.status == S.ERR_PATTERN


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    m, k, n, b = 512, 768, 40, 8
    c = wl.integer_problem(4242, m, k, n, b, wl.nnzb_for(m, k, b, 1 / 4))
    rb, re = P.row_split(m, b, world)[rank]
    sb, sc, src = check_slice_plan(m, k, n, b, c["brow"], c["bcol"], rb, re, "tc")
    # this rank's rows through the oracle on its slice, from the whole W's
    # values picked by src_index
    Yr = oracle.spmm(re - rb, k, b, sb, sc, c["vals"][src], c["X"])
    parts = [torch.zeros((hi - lo, n), dtype=torch.float64) for lo, hi in P.row_split(m, b, world)]
    dist.all_gather(parts, torch.from_numpy(Yr))
    if rank == 0:
        out["Y"] = torch.cat(parts).numpy()
        out["Y_whole"] = oracle.spmm(m, k, b, c["brow"], c["bcol"], c["vals"], c["X"])
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_row_split():
    port = _free_port()
    with mp.get_context("spawn").Manager() as man:
        out = man.dict()
        mp.start_processes(_rank, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
        res = dict(out)
    assert np.array_equal(res["Y"], res["Y_whole"])
