"""The multi-rank paths on CPU with the gloo backend (world size 2).

* block-sharded A x: partial P_r^T W_r P_r x per rank plus one all-reduce
  equals the whole product;
* a PCG whose products and inner products are reduced over ranks gives the
  single-process solution;
* the bench's replica timing takes the maximum over ranks.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import oracle as O  # noqa: E402
import synth  # noqa: E402
from paper_1801_08937_gb300 import sharding as SH  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _scan():
    return synth.make_scan(nx=8, ny=8, n_det=4, n_t=2048, n_int=4, half_bw=40, f_knee=1.0, seed=31,
                           flag_frac=0.01)


def _worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    scan = _scan()
    b0, b1 = SH.partition_blocks(scan.block_off, world)[rank]
    pix, psi, off, band_idx, _ = SH.shard(scan.pix, scan.psi, scan.block_off, scan.block_band, b0, b1)
    local = O.Problem(pix, psi, off, scan.band, band_idx, scan.n_pix)

    def allsum(a):
        t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64))
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        return t.numpy()

    x = np.random.default_rng(5).standard_normal((scan.n_pix, 3))
    Ax = allsum(O.apply_A(local, x))
    # M_BD blocks are sums over blocks too
    blocks, hits = O.bd_blocks(local)
    blocks = allsum(blocks)
    hits = allsum(hits.astype(np.float64))
    good = O.select_pixels(blocks, hits)
    mbd = O.bd_inverse(blocks, good)
    d = synth.make_tod(scan, synth.make_sky(scan.n_pix, 6), synth.make_noise(scan, 6))
    t0, t1 = int(scan.block_off[b0]), int(scan.block_off[b1])
    b = allsum(O.rhs(local, d[t0:t1])).reshape(-1)
    xs, info = O.pcg(lambda v: allsum(O.apply_A(local, v)).reshape(-1),
                     lambda v: O.bd_apply(mbd, v).reshape(-1), b, tol=1e-10, max_iter=2000)
    tmax = SH.max_over_ranks(1.0 + rank, dist)
    np.savez(os.path.join(out_dir, f"r{rank}.npz"), Ax=Ax, x=xs, iters=info["iters"], tmax=tmax,
             b0=b0, b1=b1)
    dist.destroy_process_group()


def test_partition_is_balanced_and_complete():
    off = np.array([0, 10, 30, 35, 90, 100, 160])
    parts = SH.partition_blocks(off, 3)
    assert parts[0][0] == 0 and parts[-1][1] == 6
    assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))
    assert SH.partition_blocks(off, 1) == [(0, 6)]


def test_two_rank_sharded_product_and_solve(tmp_path):
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    r = [np.load(tmp_path / f"r{i}.npz") for i in range(world)]
    scan = _scan()
    prob = O.Problem.from_scan(scan)
    x = np.random.default_rng(5).standard_normal((scan.n_pix, 3))
    np.testing.assert_allclose(r[0]["Ax"], O.apply_A(prob, x), rtol=1e-12, atol=1e-9)
    np.testing.assert_allclose(r[1]["Ax"], r[0]["Ax"], rtol=0, atol=0)
    assert int(r[0]["b1"]) == int(r[1]["b0"])
    # single-process solve of the same system
    blocks, hits = O.bd_blocks(prob)
    good = O.select_pixels(blocks, hits)
    mbd = O.bd_inverse(blocks, good)
    d = synth.make_tod(scan, synth.make_sky(scan.n_pix, 6), synth.make_noise(scan, 6))
    b = O.rhs(prob, d).reshape(-1)
    xs, info = O.pcg(lambda v: O.apply_A(prob, v).reshape(-1), lambda v: O.bd_apply(mbd, v).reshape(-1), b,
                     tol=1e-10, max_iter=2000)
    np.testing.assert_allclose(r[0]["x"], xs, rtol=1e-8, atol=1e-10)
    assert int(r[0]["iters"]) == info["iters"]
    assert float(r[0]["tmax"]) == 2.0 and float(r[1]["tmax"]) == 2.0
