"""The coarse products of M_2l on the tensor cores (option "tc_coarse") against the oracle and the
float64 CUDA-core kernels, at the shapes of the batched Monte Carlo workload (32x32 patch, k = 32,
64 right-hand sides) and of the large map (512x512 patch, k = 64, 64 right-hand sides).

The tensor-core path splits its operands into TF32 pairs (high part + remainder, about 22 bits),
accumulates in float32 and forms M_BD (R - AZ U) + Z U in float32, so M_2l x agrees with the float64
result to a few 1e-7 (an element near a cancellation to a few 1e-6); the tolerance below is 2e-5.
A two-level PCG solve with it converges to the same maps in the same number of products.
"""
import numpy as np
import pytest

import oracle as O
import synth
from helpers import assert_close, oracle_problem

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_1801_08937_gb300")
MM = P.mapmaker

TOL_TC = 2e-5


def _ctx(scan, tc):
    """tc: 2 puts every eligible batch on the tensor cores (1 would keep small maps on the CUDA cores)."""
    c = MM.Context(0, None, MM.MM_FP64)
    c.set_option("tc_coarse", 2 if tc else 0)
    c.setup_scan(scan)
    c.build_bd()
    return c


def test_tc_m2l_matches_oracle_at_the_batched_shape():
    """32x32 patch, k = 32 (a seeded random basis installed with mm_set_coarse), 64 right-hand
    sides: tensor-core M_2l x against the oracle's Eq. m2l with its own A Z, E and M_BD."""
    scan = synth.make_scan(nx=32, ny=32, n_det=8, n_t=16384, n_int=4, half_bw=32, f_knee=1.0, seed=71)
    prob, mbd, good = oracle_problem(scan)
    rng = np.random.default_rng(71)
    Z = rng.standard_normal((32, scan.n_pix, 3))
    Z[:, ~good] = 0.0
    x = rng.standard_normal((64, scan.n_pix, 3))
    x[:, ~good] = 0.0
    Zf = Z.reshape(32, -1).T
    A = lambda v: O.apply_A(prob, v.reshape(-1, 3)).reshape(-1)  # noqa: E731
    M = lambda v: O.bd_apply(mbd, v).reshape(-1)  # noqa: E731
    AZ, _, L = O.coarse_space(A, Zf)
    ref = np.stack([O.m2l_apply(x[r].reshape(-1), M, Zf, AZ, L).reshape(-1, 3) for r in range(64)])
    c = _ctx(scan, 1)
    c.set_coarse(Z)
    xd = torch.from_numpy(x).cuda()
    y_tc = c.apply_precond(MM.MM_PRECOND_2L, xd).cpu().numpy()
    assert_close(y_tc, ref, TOL_TC, "tensor-core M_2l vs oracle, 64 RHS, k = 32")
    c.set_option("tc_coarse", 0)
    y64 = c.apply_precond(MM.MM_PRECOND_2L, xd).cpu().numpy()
    assert_close(y64, ref, 1e-11, "float64 M_2l vs oracle, 64 RHS, k = 32")
    # eight right-hand sides, the smallest batch the tensor-core path takes
    c.set_option("tc_coarse", 2)
    y8 = c.apply_precond(MM.MM_PRECOND_2L, xd[:8].contiguous()).cpu().numpy()
    assert_close(y8, ref[:8], TOL_TC, "tensor-core M_2l vs oracle, 8 RHS")
    # the default (1) keeps a map this small (1024 pixels) on the float64 CUDA-core kernels
    c.set_option("tc_coarse", 1)
    y_auto = c.apply_precond(MM.MM_PRECOND_2L, xd).cpu().numpy()
    assert_close(y_auto, ref, 1e-11, "default tc_coarse on a 1024-pixel map: float64 M_2l vs oracle")
    with pytest.raises(MM.MapMakerError) as e:
        c.set_option("tc_coarse", 3)
    assert e.value.status == MM.MM_ERR_ARG
    c.close()


def test_tc_m2l_large_map_against_float64_kernels_and_identity():
    """512x512 patch (786432 unknowns), k = 64, 64 right-hand sides: tensor-core against float64
    CUDA-core M_2l, and M_2l A Z = Z (Sect. 3.2, Eq. ident) through the tensor-core path."""
    scan = synth.make_scan(nx=512, ny=512, n_det=16, n_t=1 << 18, n_int=4, half_bw=16, f_knee=1.0, seed=72)
    c = _ctx(scan, 1)
    rng = np.random.default_rng(72)
    c.set_coarse(rng.standard_normal((64, scan.n_pix, 3)))
    Z, _ = c.get_coarse()
    x = torch.from_numpy(rng.standard_normal((64, scan.n_pix, 3))).cuda()
    y_tc = c.apply_precond(MM.MM_PRECOND_2L, x).cpu().numpy()
    c.set_option("tc_coarse", 0)
    y64 = c.apply_precond(MM.MM_PRECOND_2L, x).cpu().numpy()
    assert_close(y_tc, y64, TOL_TC, "tensor-core vs float64 M_2l, 512x512, k = 64, 64 RHS")
    c.set_option("tc_coarse", 2)
    # here U = E^-1 (Z^T A Z) is the identity: the float32-accumulated Z^T A Z (about 1e-6) is amplified by
    # the condition number of E, and (A Z - A Z U) cancels, so the identity holds to about 1e-5 of Z
    AZ = c.apply_A(torch.from_numpy(Z).cuda())
    MAZ = c.apply_precond(MM.MM_PRECOND_2L, AZ).cpu().numpy()
    assert_close(MAZ, Z, 1e-4, "M_2l A Z = Z through the tensor-core path", elem_tol=1e-3)
    c.close()


def test_tc_two_level_batch_solves_like_float64():
    """A batch of 16 maps on one operator: two-level PCG with the tensor-core coarse products reaches
    the tolerance and the same maps as with the float64 ones."""
    cfg = dict(nx=16, ny=16, n_det=4, n_t=8192, n_int=4, half_bw=64, f_knee=2.0)
    scan = synth.make_scan(seed=73, **cfg)
    tods = np.stack([synth.make_tod(scan, synth.make_sky(scan.n_pix, 700 + i), synth.make_noise(scan, 700 + i))
                     for i in range(16)])
    res = {}
    for tc in (0, 1):
        c = _ctx(scan, tc)
        k = c.build_coarse(c.rhs(tods[:1])[0], m_max=60, eps_arn=1e-12, k=24)
        assert k == 24
        x, info = c.solve(tods, MM.MM_PRECOND_2L, tol=1e-10, max_iter=2000)
        res[tc] = (x, info)
        c.close()
    for r in range(16):
        assert res[1][1][r]["status"] == "MM_OK" and res[1][1][r]["true_rel_res"] <= 1e-9
        assert abs(res[1][1][r]["iters"] - res[0][1][r]["iters"]) <= 2
        assert_close(res[1][0][r], res[0][0][r], 1e-8, f"map {r}: tensor-core vs float64 coarse products")


def test_tc_m2l_matches_oracle_at_the_mixed_precision_map_shape():
    """The 512x512 patch of the mixed-precision workload (786432 unknowns), k = 64, 64 right-hand
    sides: tensor-core M_2l x against the oracle's Eq. m2l element by element, with the oracle's own
    A Z (a short 8-detector scan keeps the 64 oracle products A z_i to seconds), E and M_BD."""
    scan = synth.make_scan(nx=512, ny=512, n_det=8, n_t=1 << 18, n_int=4, half_bw=16, f_knee=1.0, seed=74)
    prob, mbd, good = oracle_problem(scan)
    rng = np.random.default_rng(74)
    k, nrhs = 64, 64
    Z = rng.standard_normal((k, scan.n_pix, 3))
    Z[:, ~good] = 0.0
    x = rng.standard_normal((nrhs, scan.n_pix, 3))
    x[:, ~good] = 0.0
    Zf = Z.reshape(k, -1).T
    A = lambda v: O.apply_A(prob, v.reshape(-1, 3)).reshape(-1)  # noqa: E731
    M = lambda v: O.bd_apply(mbd, v).reshape(-1)  # noqa: E731
    AZ, _, L = O.coarse_space(A, Zf)
    c = _ctx(scan, 1)
    c.set_coarse(Z)
    y_tc = c.apply_precond(MM.MM_PRECOND_2L, torch.from_numpy(x).cuda()).cpu().numpy()
    c.close()
    ref = np.stack([O.m2l_apply(x[r].reshape(-1), M, Zf, AZ, L).reshape(-1, 3) for r in range(nrhs)])
    assert_close(y_tc, ref, TOL_TC, "tensor-core M_2l vs oracle, 512x512, k = 64, 64 RHS")
