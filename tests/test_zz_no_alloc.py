"""The allocation-free M_2l entry point agrees with mm_apply_precond.

mm_apply_precond_2l_noalloc exists for callers that may not allocate device
memory while they run (latency-critical serving loops, plug-ins inside a host
application that owns the device memory).  It keeps its reduction scratch in
a fixed device array inside the library instead of allocating temporaries.
This file is collected last so that a failure here leaves every other test
already run.
"""
import numpy as np
import pytest

import synth
from helpers import assert_close

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_1801_08937_gb300")
MM = P.mapmaker


def test_noalloc_m2l_matches_allocating_entry_point_twice():
    scan = synth.make_scan(nx=8, ny=8, n_det=4, n_t=4096, n_int=4, half_bw=64, f_knee=1.0, seed=21)
    d = synth.make_tod(scan, synth.make_sky(scan.n_pix, 21), synth.make_noise(scan, 21))
    c = MM.Context(0, None, MM.MM_FP64)
    c.setup_scan(scan)
    c.build_bd()
    b = c.rhs(d)
    k = c.build_coarse(b[0], m_max=20, eps_arn=1e-12, k=6)
    assert k == 6
    rng = np.random.default_rng(21)
    for call in range(2):
        nrhs = 3
        x = torch.from_numpy(rng.standard_normal((nrhs, scan.n_pix, 3))).cuda()
        ref = c.apply_precond(MM.MM_PRECOND_2L, x)
        out = torch.full_like(x, float("nan"))
        c.apply_precond_2l_noalloc(x, out)
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        assert np.isfinite(o).all()
        assert_close(o, ref.cpu().numpy(), 1e-11, f"call {call}")


def test_noalloc_rejects_oversized_batches():
    scan = synth.make_scan(nx=4, ny=4, n_det=2, n_t=512, n_int=2, half_bw=8, f_knee=1.0, seed=22)
    c = MM.Context(0, None, MM.MM_FP64)
    c.setup_scan(scan)
    c.build_bd()
    c.build_coarse(c.rhs(synth.make_tod(scan, synth.make_sky(scan.n_pix, 22), None))[0], m_max=10,
                   eps_arn=1e-12, k=4)
    x = torch.zeros((129, scan.n_pix, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(MM.MapMakerError) as e:
        c.apply_precond_2l_noalloc(x, torch.empty_like(x))
    assert e.value.status == MM.MM_ERR_ARG


def _ctx_with_basis(prec, k, seed, nx=12):
    """A context whose coarse space is a random k-vector basis installed with mm_set_coarse."""
    scan = synth.make_scan(nx=nx, ny=nx, n_det=4, n_t=4096, n_int=4, half_bw=32, f_knee=1.0, seed=seed)
    c = MM.Context(0, None, prec)
    c.setup_scan(scan)
    c.build_bd()
    Z = np.random.default_rng(seed).standard_normal((k, scan.n_pix, 3))
    c.set_coarse(Z)
    return c, scan


@pytest.mark.parametrize("prec", [MM.MM_FP64, MM.MM_FP32_MIXED])
def test_noalloc_largest_coarse_space_and_batch(prec):
    """k = 128 (the shared-array limit of the kernels) and 128 right-hand sides: the partial sums
    of Z^T x no longer fit one CTA row per pixel chunk, so the call runs fewer CTAs than the
    allocating path; results agree on two calls in a row, in both context precisions."""
    c, scan = _ctx_with_basis(prec, 128, 41)
    rng = np.random.default_rng(41)
    for call in range(2):
        x = torch.from_numpy(rng.standard_normal((128, scan.n_pix, 3))).cuda()
        ref = c.apply_precond(MM.MM_PRECOND_2L, x)
        out = torch.full_like(x, float("nan"))
        c.apply_precond_2l_noalloc(x, out)
        torch.cuda.synchronize()
        assert_close(out.cpu().numpy(), ref.cpu().numpy(), 1e-11, f"k=128 nrhs=128 call {call}")


def test_noalloc_refuses_a_larger_coarse_space_and_aliased_arrays():
    c, scan = _ctx_with_basis(MM.MM_FP64, 129, 42)
    x = torch.zeros((1, scan.n_pix, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(MM.MapMakerError) as e:
        c.apply_precond_2l_noalloc(x, torch.empty_like(x))
    assert e.value.status == MM.MM_ERR_ARG
    c.close()
    c, scan = _ctx_with_basis(MM.MM_FP64, 8, 43)
    x = torch.ones((2, scan.n_pix, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(MM.MapMakerError) as e:
        c.apply_precond_2l_noalloc(x, x)                     # in place
    assert e.value.status == MM.MM_ERR_ARG
    flat = torch.ones(3 * 3 * scan.n_pix, dtype=torch.float64, device="cuda")
    with pytest.raises(MM.MapMakerError) as e:                # y starts inside x
        c.apply_precond_2l_noalloc(flat[:2 * 3 * scan.n_pix], flat[3 * scan.n_pix:])
    assert e.value.status == MM.MM_ERR_ARG
    assert torch.all(x == 1)


def test_noalloc_restores_the_current_device():
    c, scan = _ctx_with_basis(MM.MM_FP64, 4, 44)
    x = torch.ones((1, scan.n_pix, 3), dtype=torch.float64, device="cuda")
    before = torch.cuda.current_device()
    c.apply_precond_2l_noalloc(x, torch.empty_like(x))
    assert torch.cuda.current_device() == before
