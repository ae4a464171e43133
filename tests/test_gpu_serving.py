"""Continuous-batching server: each map is the same alone and in the mix.

Requests on a handful of scans (some repeated, so their coarse space is
reused) arrive while others are still iterating; every result must match
the same request solved alone through the plain C ABI within the solve
tolerance, and must match the FP64 oracle on the small scans.
"""
import time

import numpy as np
import pytest

import oracle as O
import synth
from helpers import assert_close, oracle_problem

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_1801_08937_gb300")
MM = P.mapmaker
from paper_1801_08937_gb300 import serving as S  # noqa: E402


def _scan(i):
    shapes = [dict(nx=8, ny=8, n_det=4, n_t=2048, n_int=2, half_bw=64, f_knee=1.0),
              dict(nx=12, ny=12, n_det=3, n_t=4096, n_int=4, half_bw=32, f_knee=0.5),
              dict(nx=6, ny=6, n_det=2, n_t=3072, n_int=3, half_bw=100, f_knee=2.0)]
    return synth.make_scan(seed=40 + i, **shapes[i % 3])


def _spec(scan):
    return S.ScanSpec(scan.pix, scan.psi, scan.block_off, scan.block_band, scan.band, scan.n_pix, scan.n_det)


def _alone(scan, tod, precision, precond, k, m_max):
    c = MM.Context(0, None, precision)
    c.setup_scan(scan)
    c.build_bd(1e-3)
    if precond == MM.MM_PRECOND_2L:
        c.build_coarse(c.rhs(tod)[0], m_max=m_max, eps_arn=1e-6, k=k)
    x, info = c.solve(tod, precond, tol=1e-9, max_iter=800)
    c.close()
    return x[0], info[0]


@pytest.mark.parametrize("precision", [MM.MM_FP64, MM.MM_FP32_MIXED])
def test_results_same_alone_and_in_mix(precision):
    scans = [_scan(i) for i in range(3)]
    dtype = np.float32 if precision == MM.MM_FP32_MIXED else np.float64
    reqs = []
    for j in range(9):
        i = j % 3
        sc = scans[i]
        tod = synth.make_tod(sc, synth.make_sky(sc.n_pix, 100 + j), synth.make_noise(sc, 100 + j)).astype(dtype)
        reqs.append((f"scan{i}", sc, tod))
    srv = S.MapServer(device=0, precision=precision, iters_per_tick=1, m_max=30, k=6, reserve_bytes=0).start()
    futs = []
    for j, (sid, sc, tod) in enumerate(reqs):
        futs.append(srv.submit(S.MapRequest(sid, _spec(sc), tod, MM.MM_PRECOND_2L, tol=1e-9, max_iter=800)))
        if j == 5:
            time.sleep(0.01)            # later arrivals join while earlier solves run
    res = [f.result(timeout=120) for f in futs]
    st = srv.stats()
    srv.stop()
    assert st["completed"] == 9 and st["max_concurrent"] >= 2
    # a repeat finds its scan resident or shares the scan's first solve
    assert all(r.scan_cached or r.batch_size > 1 for r in res[3:])
    for (sid, sc, tod), r in zip(reqs, res):
        assert r.info["status"] == "MM_OK"
        # the coarse space of a repeated scan comes from its first request's b, so
        # compare against the exact solution rather than bit-for-bit
        prob, mbd, good = oracle_problem(sc)
        b = O.rhs(prob, tod.astype(np.float64)).reshape(-1)
        xo = O.pcg(lambda v: O.apply_A(prob, v).reshape(-1), lambda v: O.bd_apply(mbd, v).reshape(-1), b,
                   tol=1e-13, max_iter=5000)[0]
        assert_close(r.map, xo, 1e-6)
    # the first request of each scan has exactly the set-up of a standalone solve
    for j in range(3):
        sid, sc, tod = reqs[j]
        xa, ia = _alone(sc, tod, precision, MM.MM_PRECOND_2L, 6, 30)
        assert_close(res[j].map, xa, 1e-7)


def test_admission_waits_for_memory_and_evicts_idle_scans():
    scans = [_scan(i) for i in range(3)]
    per_scan = max(MM.estimate_bytes(s.n_samples, s.n_pix, s.n_bands, s.half_bw, 1, 30, 6, MM.MM_FP64)
                   for s in scans)
    # room for about two resident scans: the third must wait and evict
    srv = S.MapServer(device=0, precision=MM.MM_FP64, iters_per_tick=4, m_max=30, k=6, reserve_bytes=0,
                      budget_bytes=int(2.5 * per_scan)).start()
    futs = []
    for j in range(6):
        sc = scans[j % 3]
        tod = synth.make_tod(sc, synth.make_sky(sc.n_pix, 200 + j), synth.make_noise(sc, 200 + j))
        futs.append(srv.submit(S.MapRequest(f"s{j % 3}", _spec(sc), tod, MM.MM_PRECOND_BD, tol=1e-9)))
    res = [f.result(timeout=120) for f in futs]
    st = srv.stats()
    srv.stop()
    assert all(r.info["status"] == "MM_OK" for r in res)
    assert st["evictions"] >= 1


def test_harvest_mode_first_request_bd_then_two_level():
    """A new scan's first request runs M_BD and seeds the coarse space for the next ones."""
    sc = _scan(0)
    tods = [synth.make_tod(sc, synth.make_sky(sc.n_pix, 500 + j), synth.make_noise(sc, 500 + j)) for j in range(3)]
    srv = S.MapServer(device=0, precision=MM.MM_FP64, iters_per_tick=2, m_max=40, k=6, reserve_bytes=0,
                      coarse="harvest").start()
    first = srv.submit(S.MapRequest("h", _spec(sc), tods[0], MM.MM_PRECOND_2L, tol=1e-9)).result(timeout=120)
    time.sleep(0.05)
    later = [srv.submit(S.MapRequest("h", _spec(sc), t, MM.MM_PRECOND_2L, tol=1e-9)) for t in tods[1:]]
    later = [f.result(timeout=120) for f in later]
    srv.stop()
    prob, mbd, good = oracle_problem(sc)
    for t, r in zip(tods, [first] + later):
        assert r.info["status"] == "MM_OK"
        b = O.rhs(prob, t).reshape(-1)
        xo = O.pcg(lambda v: O.apply_A(prob, v).reshape(-1), lambda v: O.bd_apply(mbd, v).reshape(-1), b,
                   tol=1e-13, max_iter=5000)[0]
        assert_close(r.map, xo, 1e-6)
    assert all(r.info["iters"] < first.info["iters"] for r in later)


def test_requests_on_a_busy_scan_fold_into_one_multi_rhs_solve():
    """Requests that arrive while their scan is being set up or solved wait and then run together as
    one multi-right-hand-side PCG solve on the scan's context; each map is the one the same request
    gets alone with that scan's coarse space (built from the first request's timeline)."""
    sc = _scan(1)
    tods = [synth.make_tod(sc, synth.make_sky(sc.n_pix, 600 + j), synth.make_noise(sc, 600 + j)) for j in range(6)]
    srv = S.MapServer(device=0, precision=MM.MM_FP64, iters_per_tick=1, m_max=30, k=6, reserve_bytes=0,
                      max_batch=4).start()
    futs = [srv.submit(S.MapRequest("b", _spec(sc), t, MM.MM_PRECOND_2L, tol=1e-10, max_iter=800)) for t in tods]
    # a request with another tolerance is not folded into the same run
    other = srv.submit(S.MapRequest("b", _spec(sc), tods[0], MM.MM_PRECOND_2L, tol=1e-8, max_iter=800))
    res = [f.result(timeout=120) for f in futs]
    r_other = other.result(timeout=120)
    st = srv.stats()
    srv.stop()
    assert st["completed"] == 7
    assert st["largest_batch"] == 4 and st["batched_requests"] >= 4
    assert max(r.batch_size for r in res) == 4 and r_other.info["status"] == "MM_OK"
    c = MM.Context(0, None, MM.MM_FP64)
    c.setup_scan(sc)
    c.build_bd(1e-3)
    c.build_coarse(c.rhs(tods[0])[0], m_max=30, eps_arn=1e-6, k=6)
    for j, (t, r) in enumerate(zip(tods, res)):
        assert r.info["status"] == "MM_OK"
        xa, ia = c.solve(t, MM.MM_PRECOND_2L, tol=1e-10, max_iter=800)
        assert abs(r.info["iters"] - ia[0]["iters"]) <= 1
        assert_close(r.map, xa[0], 1e-9, f"request {j} (batch of {r.batch_size}) vs alone")
    c.close()
