"""Host-side merge of independent jobs' checkpoints (Sec. 3.4), on CPU.

The jobs of the paper's third parallel strategy each accumulate a subset of
the snapshots and are merged before Step 3.  Here each job's partial sums are
a checkpoint file; paper_1910_06409_gb300.merge adds them on the host.  The
two-rank test runs the jobs as gloo processes that meet only at a barrier
(the data path has no collective) and checks the merged file and the
max-over-ranks timing reduction used by bench.py.
"""
import os
import socket

import numpy as np
import pytest

from paper_1910_06409_gb300 import merge as M


def _fake(rank, ny=7, nacc=50):
    rng = np.random.default_rng(100 + rank)
    hdr = {"nx": 16, "nz": 8, "ny": ny, "precision": 0, "pair_domain": 0, "nzt": 0, "nxt": 0, "term_set": 127,
           "mean_count": 2.0 + rank, "snap_count": 2.0 + rank, "Lx": 12.5, "Lz": 6.25, "nu": 0.005}
    # every job took its spectra about the same Step-1 mean
    mean = np.random.default_rng(7).standard_normal(4 * ny)
    return {"header": hdr, "mean_sum": rng.standard_normal(4 * ny), "stats": rng.standard_normal(M.NSTAT * ny),
            "mean": mean, "acc": rng.standard_normal(nacc) + 1j * rng.standard_normal(nacc)}


def test_merge_sums(tmp_path):
    parts = [_fake(r) for r in range(3)]
    paths = []
    for r, ck in enumerate(parts):
        p = str(tmp_path / f"p{r}.ckpt")
        M.write(p, ck)
        paths.append(p)
    out = str(tmp_path / "m.ckpt")
    M.merge(paths, out)
    got = M.read(out)
    assert np.array_equal(got["mean_sum"], parts[0]["mean_sum"] + parts[1]["mean_sum"] + parts[2]["mean_sum"])
    assert np.array_equal(got["stats"], parts[0]["stats"] + parts[1]["stats"] + parts[2]["stats"])
    assert np.array_equal(got["acc"], parts[0]["acc"] + parts[1]["acc"] + parts[2]["acc"])
    assert got["header"]["snap_count"] == 9.0 and got["header"]["mean_count"] == 9.0
    assert got["header"]["have_acc"] == 1


def test_merge_rejects_mismatch_and_truncation(tmp_path):
    a, b = _fake(0), _fake(1)
    b["header"]["nu"] = 0.001
    pa, pb = str(tmp_path / "a.ckpt"), str(tmp_path / "b.ckpt")
    M.write(pa, a)
    M.write(pb, b)
    with pytest.raises(M.CheckpointError):
        M.merge([pa, pb], str(tmp_path / "m.ckpt"))
    c = _fake(2)
    c["header"]["term_set"] = 1                 # accumulators of another term set
    pc = str(tmp_path / "c.ckpt")
    M.write(pc, c)
    with pytest.raises(M.CheckpointError):
        M.merge([pa, pc], str(tmp_path / "m.ckpt"))
    d = _fake(3)
    d["header"]["acc_kind"] = 1                 # plane spectra of the split path
    pd = str(tmp_path / "d.ckpt")
    M.write(pd, d)
    with pytest.raises(M.CheckpointError):
        M.merge([pa, pd], str(tmp_path / "m.ckpt"))
    with open(pb, "wb") as f:
        f.write(b"GKECKPT")
    with pytest.raises(M.CheckpointError):
        M.read(pb)


def test_merge_refuses_jobs_with_their_own_means(tmp_path):
    # two jobs that each froze the mean of their own snapshot subset: their
    # spectra are about different means and do not add (Step 1 precedes Step 2)
    a, b = _fake(0), _fake(1)
    b["mean"] = b["mean"] * (1.0 + 1e-6)
    pa, pb = str(tmp_path / "a.ckpt"), str(tmp_path / "b.ckpt")
    M.write(pa, a)
    M.write(pb, b)
    with pytest.raises(M.CheckpointError, match="mean"):
        M.merge([pa, pb], str(tmp_path / "m.ckpt"))
    # a difference at the rounding level of the sums is the same mean
    b["mean"] = a["mean"] * (1.0 + 1e-15)
    M.write(pb, b)
    M.merge([pa, pb], str(tmp_path / "m.ckpt"))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, d, results):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        M.write(os.path.join(d, f"part{rank}.ckpt"), _fake(rank))      # this job's partial sums
        dist.barrier()
        ms = torch.tensor([10.0 + rank])                               # per-rank step time
        dist.all_reduce(ms, op=dist.ReduceOp.MAX)
        if rank == 0:
            M.merge([os.path.join(d, f"part{r}.ckpt") for r in range(world)], os.path.join(d, "merged.ckpt"))
        dist.barrier()
        results[rank] = float(ms.item())
    finally:
        dist.destroy_process_group()


def test_two_rank_jobs_and_merge(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mgr = mp.get_context("spawn").Manager()
    results = mgr.dict()
    mp.spawn(_rank, args=(world, _free_port(), str(tmp_path), results), nprocs=world, join=True)
    assert dict(results) == {0: 11.0, 1: 11.0}
    got = M.read(str(tmp_path / "merged.ckpt"))
    want = [_fake(r) for r in range(world)]
    assert np.array_equal(got["acc"], want[0]["acc"] + want[1]["acc"])
    assert got["header"]["snap_count"] == 5.0
