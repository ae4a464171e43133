"""A solve whose timeline is split across processes (mm_set_reduction) equals the single-process solve.

A and b are sums over stationary blocks (Sect. 3, Eq. linearsystem): two ranks each set up the
pointing of half of the detectors, sum every partial product with a gloo all-reduce on the host,
and must reproduce the map of one process holding the whole timeline, for M_BD and for the
two-level preconditioner.  Both ranks run on the one GPU of the test box (no kernel of one rank
waits on the other: the sums happen on the host between launches); the multi-GPU path is not
measured on hardware.
"""
import os
import socket

import numpy as np
import pytest

import synth
from helpers import assert_close

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_1801_08937_gb300")
MM = P.mapmaker

CFG = dict(nx=8, ny=8, n_det=4, n_t=4096, n_int=4, half_bw=64, f_knee=1.0)


def _local(scan, d, rank, world):
    """The detectors of one rank: pixel, angle, blocks and timeline of its contiguous detector range."""
    per = scan.n_det // world
    t0, t1 = rank * per * scan.n_t, (rank + 1) * per * scan.n_t
    b0 = int(np.searchsorted(scan.block_off, t0))
    b1 = int(np.searchsorted(scan.block_off, t1))
    return (scan.pix[t0:t1], scan.psi[t0:t1], scan.block_off[b0:b1 + 1] - t0, scan.block_band[b0:b1],
            d[t0:t1], per)


def _rank_main(rank, world, port, out_dir, prec):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    scan = synth.make_scan(seed=61, flag_frac=0.01, **CFG)
    d = synth.make_tod(scan, synth.make_sky(scan.n_pix, 61), synth.make_noise(scan, 61))
    pix, psi, bo, bb, dl, n_det = _local(scan, d, rank, world)
    c = MM.Context(0, None, prec)
    c.set_reduction(lambda arr: dist.all_reduce(torch.from_numpy(arr)))
    c.setup_pointing(pix, psi, bo, bb, scan.band, scan.n_pix, n_det=n_det)
    dropped = c.build_bd()
    tod = dl.astype(c.tod_dtype)
    xb, ib = c.solve(tod, MM.MM_PRECOND_BD, tol=1e-10, max_iter=2000)
    k = c.build_coarse(None, m_max=30, eps_arn=1e-10, k=8)
    x2, i2 = c.solve(tod, MM.MM_PRECOND_2L, tol=1e-10, max_iter=2000)
    np.savez(os.path.join(out_dir, f"rank{rank}.npz"), xb=xb[0], x2=x2[0], ib=ib[0]["iters"], i2=i2[0]["iters"],
             sb=ib[0]["status"], s2=i2[0]["status"], dropped=dropped, k=k)
    c.close()
    dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


@pytest.mark.parametrize("prec", [MM.MM_FP64, MM.MM_FP32_MIXED])
def test_two_rank_solve_equals_single_process(tmp_path, prec):
    import torch.multiprocessing as mp
    mp.spawn(_rank_main, args=(2, _free_port(), str(tmp_path), prec), nprocs=2, join=True)
    r0 = np.load(tmp_path / "rank0.npz")
    r1 = np.load(tmp_path / "rank1.npz")
    # every rank follows the same iterations and holds the same map
    assert int(r0["ib"]) == int(r1["ib"]) and int(r0["i2"]) == int(r1["i2"])
    assert np.array_equal(r0["xb"], r1["xb"]) and np.array_equal(r0["x2"], r1["x2"])
    assert str(r0["sb"]) == "MM_OK" and str(r0["s2"]) == "MM_OK"
    # against one process with the whole timeline
    scan = synth.make_scan(seed=61, flag_frac=0.01, **CFG)
    d = synth.make_tod(scan, synth.make_sky(scan.n_pix, 61), synth.make_noise(scan, 61))
    c = MM.Context(0, None, prec)
    c.setup_scan(scan)
    assert c.build_bd() == int(r0["dropped"])
    tod = d.astype(c.tod_dtype)
    xb, ib = c.solve(tod, MM.MM_PRECOND_BD, tol=1e-10, max_iter=2000)
    assert c.build_coarse(None, m_max=30, eps_arn=1e-10, k=8) == int(r0["k"])
    x2, i2 = c.solve(tod, MM.MM_PRECOND_2L, tol=1e-10, max_iter=2000)
    c.close()
    assert abs(ib[0]["iters"] - int(r0["ib"])) <= 1 and abs(i2[0]["iters"] - int(r0["i2"])) <= 2
    assert_close(r0["xb"], xb[0], 1e-8, "two ranks vs one process, M_BD")
    assert_close(r0["x2"], x2[0], 1e-8, "two ranks vs one process, M_2l")


def test_reduction_failure_is_reported():
    """A reduction that fails (here: raises) fails the call with MM_ERR_REDUCE instead of going on."""
    scan = synth.make_scan(seed=62, **CFG)
    c = MM.Context(0, None, MM.MM_FP64)

    def broken(arr):
        raise RuntimeError("rank lost")
    c.set_reduction(broken)
    c.setup_scan(scan)
    with pytest.raises(MM.MapMakerError) as e:
        c.build_bd()
    assert e.value.status == MM.MM_ERR_REDUCE
    c.set_reduction(None)
    c.build_bd()
    with pytest.raises(MM.MapMakerError) as e:
        c.set_reduction(lambda a: None)
        c.solve(np.zeros((2, scan.n_samples)), MM.MM_PRECOND_BD, rhs_len=[100, 200])
    assert e.value.status == MM.MM_ERR_ARG
    c.close()
