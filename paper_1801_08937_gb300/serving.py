"""Continuous-batching map-making server on one GPU.

Requests (a scan -- pointing, stationary blocks, noise bands -- plus a
timeline) are admitted while device memory allows.  Each scan keeps its own
context resident: pointing, M_BD and the two-level coarse space are built
once per scan_id (the paper's "simplified" reuse of one deflation basis for
later data, Sect. 7) and every later request on that scan only pays for
b = P^T W d and the PCG iterations.  Admitted solves advance together: each
tick enqueues a few PCG iterations on every active context (its own CUDA
stream) without waiting, then polls them, so their kernels overlap on the
device and a request that arrives while others run joins at the next tick.
New scans are set up on worker threads, also on their own streams.

All arithmetic runs in libmapmaker.so; this module only schedules.
"""
from __future__ import annotations

import collections
import threading
import time
from concurrent.futures import Future, ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

from . import mapmaker as M


@dataclass
class ScanSpec:
    """Pointing and weight of one scan (host numpy or device torch arrays)."""
    pix: object
    psi: object
    block_off: np.ndarray
    block_band: np.ndarray
    band: np.ndarray
    n_pix: int
    n_det: int = 1

    @property
    def n_samples(self) -> int:
        return int(self.block_off[-1])


@dataclass
class MapRequest:
    scan_id: str
    scan: ScanSpec
    tod: object                        # [n_samples] timeline, dtype of the server precision
    precond: int = M.MM_PRECOND_2L
    tol: float = 1e-8
    max_iter: int = 500
    arrival: float = field(default_factory=time.perf_counter)


@dataclass
class MapResult:
    map: np.ndarray                    # [n_pix, 3]
    info: dict
    latency_s: float
    queued_s: float
    scan_cached: bool


class _ScanEntry:
    def __init__(self, ctx, stream, nbytes, spec):
        self.ctx = ctx
        self.stream = stream
        self.nbytes = nbytes
        self.spec = spec
        self.busy = False
        self.ready = False
        self.error = None
        self.has_coarse = False
        self.harvesting = False
        self.last_used = time.perf_counter()


class _Active:
    def __init__(self, req, fut, entry, t_start, cached):
        self.req = req
        self.fut = fut
        self.entry = entry
        self.t_start = t_start
        self.cached = cached
        self.launched = False


class MapServer:
    """Admission by device memory, resident per-scan state, interleaved solves."""

    def __init__(self, device: int = 0, precision: int = M.MM_FP32_MIXED, budget_bytes: int | None = None,
                 iters_per_tick: int = 4, max_active: int = 16, m_max: int = 60, k: int = 16,
                 eps_arn: float = 1e-6, setup_workers: int = 2, reserve_bytes: int = 2 << 30,
                 coarse: str = "arnoldi"):
        """coarse: "arnoldi" builds each new scan's deflation basis before its
        first solve; "harvest" solves the first request of a scan with M_BD,
        keeping the Lanczos vectors of that run, and builds the basis from
        them afterwards, so later requests on the scan use M_2l."""
        import torch
        self.torch = torch
        self.device = device
        self.precision = precision
        self.iters_per_tick = iters_per_tick
        self.max_active = max_active
        self.m_max, self.k, self.eps_arn = m_max, k, eps_arn
        self.coarse_mode = coarse
        self.reserve = reserve_bytes
        self.budget = budget_bytes
        self._pending = collections.deque()
        self._active: list[_Active] = []
        self._setting_up: dict[str, list] = {}
        self._scans: collections.OrderedDict[str, _ScanEntry] = collections.OrderedDict()
        self._lock = threading.Lock()
        self._pool = ThreadPoolExecutor(max_workers=setup_workers)
        self._stop = threading.Event()
        self._thread = None
        self.latencies = []
        self.completed = 0
        self.cache_hits = 0
        self.evictions = 0
        self.admitted = 0
        self.rejected = 0
        self.failed = 0
        self.max_concurrent = 0
        self.t0 = None
        self.error = None

    # ---------------- public API ----------------
    def start(self):
        self.t0 = time.perf_counter()
        self._thread = threading.Thread(target=self._loop, daemon=True)
        self._thread.start()
        return self

    def stop(self, wait: bool = True):
        self._stop.set()
        if wait and self._thread is not None:
            self._thread.join()
        self._pool.shutdown(wait=True)
        for e in self._scans.values():
            e.ctx.close()
        self._scans.clear()

    def submit(self, req: MapRequest) -> Future:
        fut = Future()
        with self._lock:
            self._pending.append((req, fut))
        return fut

    def stats(self) -> dict:
        lat = np.array(self.latencies) if self.latencies else np.zeros(1)
        wall = (time.perf_counter() - self.t0) if self.t0 else 0.0
        return {"completed": self.completed, "p50_s": float(np.percentile(lat, 50)),
                "p99_s": float(np.percentile(lat, 99)), "mean_s": float(lat.mean()),
                "maps_per_s": self.completed / wall if wall > 0 else 0.0, "cache_hits": self.cache_hits,
                "evictions": self.evictions, "admitted": self.admitted, "max_concurrent": self.max_concurrent,
                "resident_scans": len(self._scans), "failed": self.failed}

    # ---------------- memory accounting ----------------
    def _free_bytes(self) -> int:
        free, total = self.torch.cuda.mem_get_info(self.device)
        if self.budget is not None:
            used = sum(e.nbytes for e in self._scans.values())
            free = min(free, self.budget - used)
        return free - self.reserve

    def _scan_bytes(self, spec: ScanSpec, nrhs=1) -> int:
        lam = int(np.asarray(spec.band).shape[-1] - 1)
        nb = int(np.asarray(spec.band).reshape(-1, lam + 1).shape[0])
        return M.estimate_bytes(spec.n_samples, spec.n_pix, nb, lam, nrhs, self.m_max, self.k, self.precision)

    def _solve_bytes(self, spec: ScanSpec) -> int:
        esz = 4 if self.precision == M.MM_FP32_MIXED else 8
        return spec.n_samples * esz + spec.n_pix * 32 * 16

    def _evict_idle(self, need: int, keep_id: str | None = None) -> bool:
        for sid in list(self._scans.keys()):
            if self._free_bytes() >= need:
                return True
            if sid == keep_id:
                continue
            e = self._scans[sid]
            if not e.busy and e.ready and sid not in self._setting_up:
                e.ctx.close()
                del self._scans[sid]
                self.evictions += 1
                self.torch.cuda.synchronize(self.device)
        return self._free_bytes() >= need

    # ---------------- scan set-up (worker threads) ----------------
    def _setup(self, sid: str, entry: _ScanEntry, want_coarse: bool, tod):
        try:
            torch = self.torch
            torch.cuda.set_device(self.device)
            with torch.cuda.stream(entry.stream):
                s = entry.spec
                entry.ctx.setup_pointing(s.pix, s.psi, s.block_off, s.block_band, s.band, s.n_pix, n_det=s.n_det)
                entry.ctx.build_bd(1e-3)
                if want_coarse and self.coarse_mode == "arnoldi":
                    b = entry.ctx.rhs(tod)
                    entry.ctx.build_coarse(b[0], m_max=self.m_max, eps_arn=self.eps_arn, k=self.k)
                    entry.has_coarse = True
            entry.stream.synchronize()
        except Exception as ex:  # reported to every waiting request
            entry.error = ex
        entry.ready = True

    def _coarse_from_solve(self, entry: _ScanEntry):
        try:
            self.torch.cuda.set_device(self.device)
            if entry.ctx.get_option("harvested") >= 2:
                entry.ctx.build_coarse_from_solve(k=self.k)
                entry.has_coarse = True
            entry.stream.synchronize()
        except Exception:
            entry.has_coarse = False   # later requests fall back to M_BD
        entry.busy = False

    # ---------------- scheduler ----------------
    def _admit(self):
        with self._lock:
            pending = list(self._pending)
        keep = []
        for req, fut in pending:
            # requests waiting for their scan's set-up start solving when it ends: they count too
            in_flight = len(self._active) + sum(len(w) for w in self._setting_up.values())
            if in_flight >= self.max_active:
                keep.append((req, fut))
                continue
            e = self._scans.get(req.scan_id)
            if e is not None and (e.busy or not e.ready):
                keep.append((req, fut))
                continue
            if e is not None and e.error is not None:
                fut.set_exception(e.error)
                continue
            need = self._solve_bytes(req.scan) + (0 if e is not None else self._scan_bytes(req.scan))
            if self._free_bytes() < need and not self._evict_idle(need, keep_id=req.scan_id):
                keep.append((req, fut))
                continue
            if e is None:
                stream = self.torch.cuda.Stream(device=self.device)
                ctx = M.Context(self.device, stream.cuda_stream, self.precision)
                e = _ScanEntry(ctx, stream, self._scan_bytes(req.scan), req.scan)
                e.busy = True
                self._scans[req.scan_id] = e
                self._pool.submit(self._setup, req.scan_id, e, req.precond == M.MM_PRECOND_2L, req.tod)
                self._setting_up.setdefault(req.scan_id, []).append((req, fut))
                self.admitted += 1
                continue
            self.cache_hits += 1
            self._start_solve(req, fut, e, cached=True)
        with self._lock:
            newer = list(self._pending)[len(pending):]
            self._pending = collections.deque(keep + newer)

    def _start_solve(self, req, fut, e, cached):
        e.busy = True
        e.last_used = time.perf_counter()
        self._scans.move_to_end(req.scan_id)
        precond = req.precond if (req.precond != M.MM_PRECOND_2L or e.has_coarse) else M.MM_PRECOND_BD
        e.harvesting = (req.precond == M.MM_PRECOND_2L and not e.has_coarse and self.coarse_mode == "harvest")
        try:
            e.ctx.set_option("harvest", self.m_max if e.harvesting else 0)
            e.ctx.solve_begin(req.tod, precond, tol=req.tol, max_iter=req.max_iter)
        except Exception as ex:
            e.busy = False
            fut.set_exception(ex)
            return
        self.admitted += 0 if not cached else 1
        self._active.append(_Active(req, fut, e, time.perf_counter(), cached))
        self.max_concurrent = max(self.max_concurrent, len(self._active))

    def _finish_setups(self):
        for sid in list(self._setting_up.keys()):
            e = self._scans.get(sid)
            if e is None or not e.ready:
                continue
            waiting = self._setting_up.pop(sid)
            e.busy = False
            for req, fut in waiting:
                if e.error is not None:
                    fut.set_exception(e.error)
                else:
                    self._start_solve(req, fut, e, cached=False)

    def _drop_failed(self, a, ex):
        """A solve that raised fails its own request; its scan's context is closed and forgotten (its
        state is unknown), so a later request on the scan sets it up again."""
        if not a.fut.done():
            a.fut.set_exception(ex)
        sid = a.req.scan_id
        if self._scans.get(sid) is a.entry:
            del self._scans[sid]
            try:
                a.entry.ctx.close()
            except Exception:
                pass
        self.failed += 1

    def _tick(self) -> bool:
        progressed = False
        failed = set()
        for a in self._active:
            if not a.launched:
                try:
                    a.entry.ctx.solve_launch(self.iters_per_tick)
                except Exception as ex:
                    self._drop_failed(a, ex)
                    failed.add(id(a))
                    continue
                a.launched = True
        still = []
        for a in self._active:
            if id(a) in failed:
                continue
            try:
                ready, done = a.entry.ctx.solve_poll()
                x, info = a.entry.ctx.solve_end() if done else (None, None)
            except Exception as ex:
                self._drop_failed(a, ex)
                progressed = True
                continue
            if ready:
                a.launched = False
                progressed = True
            if done:
                now = time.perf_counter()
                if a.entry.harvesting:
                    # deflation basis from this M_BD run's Lanczos vectors, off the critical path
                    a.entry.harvesting = False
                    self._pool.submit(self._coarse_from_solve, a.entry)
                else:
                    a.entry.busy = False
                a.entry.last_used = now
                self.latencies.append(now - a.req.arrival)
                self.completed += 1
                a.fut.set_result(MapResult(x[0], info[0], now - a.req.arrival, a.t_start - a.req.arrival, a.cached))
            else:
                still.append(a)
        self._active = still
        return progressed

    def _fail_all(self, ex):
        with self._lock:
            pending = list(self._pending)
            self._pending.clear()
        for _, fut in pending:
            if not fut.done():
                fut.set_exception(ex)
        for a in self._active:
            if not a.fut.done():
                a.fut.set_exception(ex)
        for waiting in self._setting_up.values():
            for _, fut in waiting:
                if not fut.done():
                    fut.set_exception(ex)
        self._active = []
        self._setting_up = {}

    def _loop(self):
        self.torch.cuda.set_device(self.device)
        while not self._stop.is_set():
            try:
                self._finish_setups()
                self._admit()
                progressed = self._tick() if self._active else False
            except Exception as ex:   # a scheduler fault fails every request instead of hanging them
                self._fail_all(ex)
                self.error = ex
                return
            if not progressed:
                time.sleep(0.0002)
