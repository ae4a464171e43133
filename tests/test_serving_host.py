"""The map server's scheduling logic on the host (CPU): admission by device memory, resident
per-scan state with LRU eviction, the harvest mode of the coarse space, per-scan set-up errors and
the cap on concurrent solves.  The library context and the CUDA calls are replaced by fakes that
record what the scheduler asks of them; the arithmetic itself is covered by the GPU tests.
"""
import contextlib
import threading

import numpy as np
import pytest

pytest.importorskip("torch")
from paper_1801_08937_gb300 import serving as S  # noqa: E402

M = S.M


class FakeStream:
    cuda_stream = 0

    def synchronize(self):
        pass


class FakeCuda:
    def __init__(self, free):
        self.free = free

    def Stream(self, device=None):
        return FakeStream()

    def stream(self, s):
        return contextlib.nullcontext()

    def mem_get_info(self, device):
        return self.free, self.free

    def set_device(self, device):
        pass

    def synchronize(self, device=None):
        pass

    def empty_cache(self):
        pass


class FakeTorch:
    class Tensor:                     # no timeline in these tests is a tensor
        pass

    def __init__(self, free=1 << 40):
        self.cuda = FakeCuda(free)


class FakeContext:
    """Records calls; a solve finishes after three polls (and once gate[n_pix], if any, is set) with
    map i filled by the sum of timeline i."""
    lock = threading.Lock()
    log = []
    fail_npix = set()
    fail_poll = set()
    gate = {}
    oom_begin = set()
    iters_for = {}                    # (n_pix, precond) -> products reported
    live = 0
    max_live = 0

    def __init__(self, device, stream, precision):
        self.opts = {}
        self.harvested = 0
        self.n_pix = None
        with FakeContext.lock:
            FakeContext.live += 1
            FakeContext.max_live = max(FakeContext.max_live, FakeContext.live)

    def _rec(self, *what):
        with FakeContext.lock:
            FakeContext.log.append(what)

    def setup_pointing(self, pix, psi, block_off, block_band, band, n_pix, n_det=1):
        self.n_pix = n_pix
        self._rec("setup", n_pix)
        if n_pix in FakeContext.fail_npix:
            raise RuntimeError(f"bad scan {n_pix}")

    def build_bd(self, rcond):
        return 0

    def rhs(self, tod):
        return np.zeros((1, self.n_pix, 3))

    def build_coarse(self, b, m_max, eps_arn, k):
        self._rec("coarse", self.n_pix)
        return k

    def build_coarse_from_solve(self, k):
        self._rec("coarse_from_solve", self.n_pix)
        return k

    def set_option(self, name, value):
        self.opts[name] = value

    def get_option(self, name):
        return self.harvested if name == "harvested" else self.opts.get(name, 0)

    def solve_begin(self, tod, precond, tol=1e-8, max_iter=500):
        if self.n_pix in FakeContext.oom_begin:
            FakeContext.oom_begin.discard(self.n_pix)      # out of memory once
            self._rec("oom", self.n_pix)
            raise M.MapMakerError(M.MM_ERR_OOM, "out of memory")
        self.tod, self.precond, self.polls = np.atleast_2d(np.asarray(tod)), precond, 0
        self.tol = tol
        if self.opts.get("harvest", 0) > 0:
            self.harvested = self.opts["harvest"]
        self._rec("begin", self.n_pix, precond, self.tod.shape[0], tol)

    def solve_launch(self, n_iter):
        pass

    def solve_poll(self):
        self.polls += 1
        if self.n_pix in FakeContext.fail_poll:
            FakeContext.fail_poll.discard(self.n_pix)       # fails once
            raise RuntimeError(f"breakdown on {self.n_pix}")
        g = FakeContext.gate.get(self.n_pix)
        return True, self.polls >= 3 and (g is None or g.is_set())

    def solve_end(self, out=None, like=None):
        x = np.repeat(self.tod.sum(axis=1)[:, None, None], self.n_pix, axis=1).repeat(3, axis=2)
        its = FakeContext.iters_for.get((self.n_pix, self.precond), self.polls)
        return x, [{"iters": its, "status": "MM_OK", "precond": self.precond, "tol": self.tol}
                   for _ in range(self.tod.shape[0])]

    def close(self):
        self._rec("close", self.n_pix)
        with FakeContext.lock:
            FakeContext.live -= 1


@pytest.fixture
def fake(monkeypatch):
    FakeContext.log = []
    FakeContext.fail_npix = set()
    FakeContext.fail_poll = set()
    FakeContext.gate = {}
    FakeContext.oom_begin = set()
    FakeContext.iters_for = {}
    FakeContext.live = 0
    FakeContext.max_live = 0
    monkeypatch.setattr(M, "Context", FakeContext)
    monkeypatch.setattr(M, "estimate_bytes", lambda *a, **k: 1000)
    return FakeContext


def spec(n_pix, n_samples=64):
    return S.ScanSpec(np.zeros(n_samples, np.int32), np.zeros(n_samples, np.float32),
                      np.array([0, n_samples]), np.zeros(1, np.int32), np.ones((1, 2)), n_pix)


def server(**kw):
    free = kw.pop("free", 1 << 40)
    srv = S.MapServer(device=0, precision=M.MM_FP64, reserve_bytes=0, **kw)
    srv.torch = FakeTorch(free)
    return srv.start()


def request(n_pix, value, **kw):
    return S.MapRequest(f"scan{n_pix}", spec(n_pix), np.full(64, value, np.float64), **kw)


def test_repeated_scans_hit_the_resident_state_and_results_route_to_their_requests(fake):
    srv = server()
    order = [(10, 1.0), (20, 2.0), (10, 3.0), (20, 4.0), (10, 5.0)]
    futs = []
    for n, v in order:
        futs.append(srv.submit(request(n, v)))
    res = [f.result(timeout=20) for f in futs]
    srv.stop()
    for (n, v), r in zip(order, res):
        assert r.map.shape == (n, 3) and np.all(r.map == 64 * v)
        assert r.info["precond"] == M.MM_PRECOND_2L
    st = srv.stats()
    assert st["completed"] == 5
    assert sum(1 for e in fake.log if e[0] == "setup") == 2
    assert sum(1 for e in fake.log if e[0] == "coarse") == 2     # one Arnoldi basis per scan
    # each repeat either found its scan resident or shared its first solve
    assert not res[0].scan_cached and not res[1].scan_cached
    assert all(r.scan_cached or r.batch_size > 1 for r in res[2:])


def test_memory_budget_evicts_the_least_recently_used_idle_scan(fake):
    # a scan holds 1000 B; a solve needs 8 B per sample + 512 B per pixel (64 samples, 3-5 pixels):
    # the budget fits one resident scan and its solve, never two scans
    srv = server(budget_bytes=4100)
    futs = [srv.submit(request(n, 1.0)) for n in (3, 4, 5)]
    for f in futs:
        f.result(timeout=20)
    srv.stop()
    assert srv.stats()["evictions"] == 2
    closes = [e[1] for e in fake.log if e[0] == "close"]
    assert closes[:2] == [3, 4]                                  # evicted in arrival (LRU) order
    assert fake.max_live == 1


def test_harvest_mode_solves_a_new_scan_with_m_bd_then_deflates_later_requests(fake):
    srv = server(coarse="harvest", m_max=40)
    r1 = srv.submit(request(7, 1.0)).result(timeout=20)
    assert r1.info["precond"] == M.MM_PRECOND_BD
    for _ in range(2000):                                         # the basis is built off the critical path
        if any(e[0] == "coarse_from_solve" for e in fake.log):
            break
        threading.Event().wait(0.005)
    r2 = srv.submit(request(7, 2.0)).result(timeout=20)
    srv.stop()
    assert r2.info["precond"] == M.MM_PRECOND_2L
    assert not any(e[0] == "coarse" for e in fake.log)            # no separate Arnoldi run
    begins = [e for e in fake.log if e[0] == "begin"]
    assert [b[2] for b in begins] == [M.MM_PRECOND_BD, M.MM_PRECOND_2L]


def test_a_failing_scan_set_up_fails_its_requests_only(fake):
    fake.fail_npix = {30}
    srv = server()
    bad = [srv.submit(request(30, 1.0)) for _ in range(2)]
    good = srv.submit(request(31, 2.0))
    for f in bad:
        with pytest.raises(RuntimeError, match="bad scan 30"):
            f.result(timeout=20)
    assert np.all(good.result(timeout=20).map == 128.0)
    srv.stop()
    assert srv.error is None


def test_concurrent_solves_are_capped(fake):
    srv = server(max_active=1)
    futs = [srv.submit(request(n, float(n))) for n in (40, 41, 42, 43)]
    for n, f in zip((40, 41, 42, 43), futs):
        assert np.all(f.result(timeout=20).map == 64.0 * n)
    srv.stop()
    assert srv.stats()["max_concurrent"] == 1


def test_a_failing_solve_fails_its_request_only_and_its_scan_is_set_up_again(fake):
    fake.fail_poll = {50}
    srv = server()
    bad = srv.submit(request(50, 1.0))
    good = srv.submit(request(51, 2.0))
    with pytest.raises(RuntimeError, match="breakdown on 50"):
        bad.result(timeout=20)
    assert np.all(good.result(timeout=20).map == 128.0)
    again = srv.submit(request(50, 3.0)).result(timeout=20)        # the scan's context was dropped: fresh set-up
    srv.stop()
    assert np.all(again.map == 192.0) and not again.scan_cached
    assert srv.error is None and srv.stats()["failed"] == 1
    assert sum(1 for e in fake.log if e[:2] == ("setup", 50)) == 2
    assert ("close", 50) in fake.log


def _wait_for(pred, what):
    for _ in range(4000):
        if pred():
            return
        threading.Event().wait(0.005)
    raise AssertionError(f"timed out waiting for {what}")


def test_requests_on_a_busy_scan_fold_into_its_next_multi_rhs_solve(fake):
    fake.gate = {60: threading.Event()}
    srv = server(max_batch=4)
    first = srv.submit(request(60, 1.0))
    _wait_for(lambda: any(e[0] == "begin" for e in fake.log), "the first solve")
    later = [srv.submit(request(60, float(v))) for v in (2, 3, 4, 5, 6)]
    other = srv.submit(request(60, 7.0, tol=1e-6))               # another run: not folded in
    threading.Event().wait(0.05)
    assert sum(1 for e in fake.log if e[0] == "begin") == 1      # all wait while the scan is busy
    fake.gate[60].set()
    res = [f.result(timeout=20) for f in [first] + later]
    r_other = other.result(timeout=20)
    srv.stop()
    for v, r in zip((1, 2, 3, 4, 5, 6), res):
        assert np.all(r.map == 64.0 * v)                          # results route to their own requests
    assert np.all(r_other.map == 64.0 * 7) and r_other.info["tol"] == 1e-6 and r_other.batch_size == 1
    begins = [e for e in fake.log if e[0] == "begin"]
    assert [b[3] for b in begins] == [1, 4, 1, 1]                 # max_batch caps the fold
    assert [r.batch_size for r in res] == [1, 4, 4, 4, 4, 1]
    st = srv.stats()
    assert st["batched_requests"] == 4 and st["largest_batch"] == 4 and st["completed"] == 7
    assert sum(1 for e in fake.log if e[0] == "setup") == 1


def test_requests_arriving_during_a_scan_set_up_share_its_first_solve(fake):
    srv = server(max_batch=8)
    futs = [srv.submit(request(70, float(v))) for v in (1, 2, 3)]
    res = [f.result(timeout=20) for f in futs]
    srv.stop()
    for v, r in zip((1, 2, 3), res):
        assert np.all(r.map == 64.0 * v)
    begins = [e for e in fake.log if e[0] == "begin"]
    assert sum(b[3] for b in begins) == 3 and len(begins) <= 2   # at most the first one ran alone


def test_a_solve_out_of_memory_waits_for_the_work_in_flight_and_is_retried(fake):
    fake.gate = {80: threading.Event()}
    fake.oom_begin = {81}
    srv = server()
    held = srv.submit(request(80, 1.0))
    _wait_for(lambda: ("begin", 80) in [e[:2] for e in fake.log], "the first solve")
    retried = srv.submit(request(81, 2.0))
    _wait_for(lambda: ("oom", 81) in fake.log, "the failed allocation")
    threading.Event().wait(0.05)
    assert not any(e[:2] == ("begin", 81) for e in fake.log)     # waits while scan 80 runs
    fake.gate[80].set()
    assert np.all(retried.result(timeout=20).map == 128.0)
    assert np.all(held.result(timeout=20).map == 64.0)
    srv.stop()
    assert srv.stats()["oom_requeued"] == 1 and srv.stats()["failed"] == 0


def test_harvest_mode_drops_a_coarse_space_that_saves_too_few_products(fake):
    """Scan 92's M_2l run takes 19 products after a 20-product M_BD run: later requests use M_BD.
    Scan 93's takes 10: it keeps M_2l."""
    fake.iters_for = {(92, M.MM_PRECOND_BD): 20, (92, M.MM_PRECOND_2L): 19,
                      (93, M.MM_PRECOND_BD): 20, (93, M.MM_PRECOND_2L): 10}
    srv = server(coarse="harvest", m_max=40)
    for n in (92, 93):
        for v in (1.0, 2.0, 3.0):
            if v == 2.0:
                _wait_for(lambda: ("coarse_from_solve", n) in fake.log, "the basis")
            assert np.all(srv.submit(request(n, v)).result(timeout=20).map == 64.0 * v)
    srv.stop()
    begins = {n: [e[2] for e in fake.log if e[0] == "begin" and e[1] == n] for n in (92, 93)}
    assert begins[92] == [M.MM_PRECOND_BD, M.MM_PRECOND_2L, M.MM_PRECOND_BD]
    assert begins[93] == [M.MM_PRECOND_BD, M.MM_PRECOND_2L, M.MM_PRECOND_2L]
    assert srv.stats()["coarse_disabled"] == 1


def test_release_idle_closes_idle_scans_until_memory_is_free(fake):
    """A host application asks for memory back: idle resident scans are closed, least recently used
    first, until the device reports enough free; a busy scan is kept."""
    fake.gate = {101: threading.Event()}
    srv = server(free=1 << 20)
    for n in (100, 102):
        srv.submit(request(n, 1.0)).result(timeout=20)
    busy = srv.submit(request(101, 1.0))
    _wait_for(lambda: ("begin", 101) in [e[:2] for e in fake.log], "the busy solve")
    srv.torch.cuda.free = 0                        # nothing free until scans are closed
    srv.release_idle(1 << 10)
    _wait_for(lambda: ("close", 102) in fake.log, "the second idle scan to close")
    closes = [e[1] for e in fake.log if e[0] == "close"]
    assert closes == [100, 102] and 101 not in closes   # LRU order; the busy scan stays
    fake.gate[101].set()
    busy.result(timeout=20)
    srv.stop()
