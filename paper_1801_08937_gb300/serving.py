"""Continuous-batching map-making server on one GPU.

Requests (a scan -- pointing, stationary blocks, noise bands -- plus a
timeline) are admitted while device memory allows.  Each scan keeps its own
context resident: pointing, M_BD and the two-level coarse space are built
once per scan_id (the paper's "simplified" reuse of one deflation basis for
later data, Sect. 7) and every later request on that scan only pays for
b = P^T W d and the PCG iterations.  Requests on one scan that wait while the
scan's context is busy (or still being set up) are folded into its next
solve: one multi-right-hand-side PCG run (the paper's Monte Carlo case of many
maps on one operator, Sect. 7), up to max_batch maps, for requests that ask
for the same preconditioner, tolerance and iteration cap.  Admitted solves
advance together: each
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
    batch_size: int = 1                # maps solved together in the request's PCG run


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
        self.bd_iters = None           # products of this scan's harvested M_BD solve
        self.coarse_checked = False    # the first M_2l solve has been compared with it
        self.coarse_useless = False    # M_2l saved too little here: requests use M_BD
        self.last_used = time.perf_counter()


class _Active:
    def __init__(self, batch, entry, t_start, cached, precond=None):
        self.batch = batch             # [(request, future)] solved as one multi-right-hand-side run
        self.precond = precond         # the preconditioner the run uses
        self.entry = entry
        self.t_start = t_start
        self.cached = cached
        self.launched = False


class MapServer:
    """Admission by device memory, resident per-scan state, interleaved solves."""

    def __init__(self, device: int = 0, precision: int = M.MM_FP32_MIXED, budget_bytes: int | None = None,
                 iters_per_tick: int = 4, max_active: int = 16, m_max: int = 60, k: int = 16,
                 eps_arn: float = 1e-6, setup_workers: int = 2, reserve_bytes: int = 2 << 30,
                 coarse: str = "arnoldi", max_batch: int = 16, min_coarse_gain: float = 0.1):
        """coarse: "arnoldi" builds each new scan's deflation basis before its
        first solve; "harvest" solves the first request of a scan with M_BD,
        keeping the Lanczos vectors of that run, and builds the basis from
        them afterwards, so later requests on the scan use M_2l.
        max_active bounds the requests in flight (set-ups and solves, counted
        per map); max_batch the maps folded into one solve.  In harvest mode
        the first M_2l solve of a scan is compared with the scan's M_BD run:
        if it saved less than min_coarse_gain of the products, later requests
        on the scan use M_BD (a coarse space does not pay on every operator)."""
        import torch
        self.torch = torch
        self.device = device
        self.precision = precision
        self.iters_per_tick = iters_per_tick
        self.max_active = max_active
        self.max_batch = max(1, int(max_batch))
        self.min_coarse_gain = float(min_coarse_gain)
        self.coarse_disabled = 0
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
        self._release = 0
        self._reserved = {}            # scan_id -> bytes promised to a set-up that has not allocated yet
        self._oom_wait = False         # a solve ran out of memory: start none until another ends
        self.oom_requeued = 0
        self.batched = 0               # requests that shared their PCG run with others
        self.largest_batch = 0
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

    def release_idle(self, need_bytes: int):
        """Ask the scheduler to close idle resident scans (least recently used first) until
        need_bytes of device memory are free, for a host application that needs memory back."""
        with self._lock:
            self._release = max(self._release, int(need_bytes))

    def stats(self) -> dict:
        lat = np.array(self.latencies) if self.latencies else np.zeros(1)
        wall = (time.perf_counter() - self.t0) if self.t0 else 0.0
        return {"completed": self.completed, "p50_s": float(np.percentile(lat, 50)),
                "p99_s": float(np.percentile(lat, 99)), "mean_s": float(lat.mean()),
                "maps_per_s": self.completed / wall if wall > 0 else 0.0, "cache_hits": self.cache_hits,
                "evictions": self.evictions, "admitted": self.admitted, "max_concurrent": self.max_concurrent,
                "resident_scans": len(self._scans), "failed": self.failed, "batched_requests": self.batched,
                "largest_batch": self.largest_batch, "oom_requeued": self.oom_requeued,
                "coarse_disabled": self.coarse_disabled}

    # ---------------- memory accounting ----------------
    def _free_bytes(self) -> int:
        """Device memory that admission may still hand out: what the device reports free, less the
        reserve and what set-ups in flight will allocate."""
        free, total = self.torch.cuda.mem_get_info(self.device)
        if self.budget is not None:
            used = sum(e.nbytes for e in self._scans.values())
            free = min(free, self.budget - used)
        return free - self.reserve - sum(self._reserved.values())

    def _scan_bytes(self, spec: ScanSpec, nrhs=1) -> int:
        lam = int(np.asarray(spec.band).shape[-1] - 1)
        nb = int(np.asarray(spec.band).reshape(-1, lam + 1).shape[0])
        return M.estimate_bytes(spec.n_samples, spec.n_pix, nb, lam, nrhs, self.m_max, self.k, self.precision)

    def _tod_bytes(self, spec: ScanSpec) -> int:
        return spec.n_samples * (4 if self.precision == M.MM_FP32_MIXED else 8)

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
    @staticmethod
    def _key(req):
        """Requests solved together must agree on what the run computes."""
        return (req.precond, float(req.tol), int(req.max_iter))

    def _in_flight(self) -> int:
        """Requests being solved or waiting for their scan's set-up."""
        return sum(len(a.batch) for a in self._active) + sum(len(w) for w in self._setting_up.values())

    def _admit(self):
        with self._lock:
            pending = list(self._pending)
        keep = []
        taken = set()
        for j, (req, fut) in enumerate(pending):
            if j in taken:
                continue
            room = self.max_active - self._in_flight()
            if room <= 0 or self._oom_wait:
                keep.append((req, fut))
                continue
            e = self._scans.get(req.scan_id)
            if e is not None and e.error is not None:
                fut.set_exception(e.error)
                continue
            if e is not None and (e.busy or not e.ready):
                keep.append((req, fut))     # folded into the scan's next solve
                continue
            # this request and the later ones on the same scan that ask for the same run
            batch, idx = [(req, fut)], [j]
            for j2 in range(j + 1, len(pending)):
                if len(batch) >= min(self.max_batch, room):
                    break
                r2 = pending[j2][0]
                if j2 not in taken and r2.scan_id == req.scan_id and self._key(r2) == self._key(req):
                    batch.append(pending[j2])
                    idx.append(j2)
            def need_of(n):
                # solve state, plus the stacked timelines of a batch, plus a new scan's resident state
                b = self._solve_bytes(req.scan) * n + (self._tod_bytes(req.scan) * n if n > 1 else 0)
                return b + (self._scan_bytes(req.scan, n) if e is None else 0)
            free = self._free_bytes()
            while len(batch) > 1 and free < need_of(len(batch)):
                batch.pop()                 # a smaller batch that fits; the rest wait for the scan
                idx.pop()
            need = need_of(len(batch))
            if free < need and not self._evict_idle(need, keep_id=req.scan_id):
                keep.append((req, fut))     # the others are tried on their own turn
                continue
            taken.update(idx)
            if e is None:
                stream = self.torch.cuda.Stream(device=self.device)
                ctx = M.Context(self.device, stream.cuda_stream, self.precision)
                e = _ScanEntry(ctx, stream, self._scan_bytes(req.scan, len(batch)), req.scan)
                e.busy = True
                self._scans[req.scan_id] = e
                self._reserved[req.scan_id] = e.nbytes
                self._pool.submit(self._setup, req.scan_id, e, req.precond == M.MM_PRECOND_2L, req.tod)
                self._setting_up.setdefault(req.scan_id, []).extend(batch)
                self.admitted += len(batch)
                continue
            self.cache_hits += len(batch)
            self.admitted += len(batch)
            self._start_solve(batch, e, cached=True)
        with self._lock:
            newer = list(self._pending)[len(pending):]
            self._pending = collections.deque(keep + newer)

    def _stack_tods(self, batch, e):
        """The batch's timelines as one [nrhs, n_samples] array, made on the context's stream."""
        tods = [r.tod for r, _ in batch]
        if len(tods) == 1:
            return tods[0]
        torch = self.torch
        if all(isinstance(t, torch.Tensor) and t.is_cuda for t in tods):
            with torch.cuda.stream(e.stream):
                return torch.stack([t.reshape(-1) for t in tods])
        return np.stack([t.cpu().numpy().reshape(-1) if isinstance(t, torch.Tensor) else np.asarray(t).reshape(-1)
                         for t in tods])

    def _start_solve(self, batch, e, cached):
        req = batch[0][0]
        e.busy = True
        e.last_used = time.perf_counter()
        self._scans.move_to_end(req.scan_id)
        precond = req.precond if (req.precond != M.MM_PRECOND_2L or e.has_coarse) else M.MM_PRECOND_BD
        e.harvesting = (req.precond == M.MM_PRECOND_2L and not e.has_coarse and not e.coarse_useless
                        and self.coarse_mode == "harvest")
        try:
            e.ctx.set_option("harvest", self.m_max if e.harvesting else 0)
            e.ctx.solve_begin(self._stack_tods(batch, e), precond, tol=req.tol, max_iter=req.max_iter)
        except Exception as ex:
            e.busy = False
            e.harvesting = False
            busy = bool(self._active or self._setting_up)
            if getattr(ex, "status", None) == M.MM_ERR_OOM and (busy or not getattr(req, "_oom_retried", False)):
                if busy:
                    # memory comes back when the work in flight ends: wait for it at the head of the queue
                    self._oom_wait = True
                else:
                    # nothing in flight: give back every idle scan's memory and try once more
                    self._evict_idle(1 << 62, keep_id=req.scan_id)
                    req._oom_retried = True
                self.oom_requeued += len(batch)
                self.torch.cuda.empty_cache()
                with self._lock:
                    self._pending.extendleft(reversed(batch))
                return
            for _, fut in batch:
                fut.set_exception(ex)
            return
        self._active.append(_Active(batch, e, time.perf_counter(), cached, precond))
        self.max_concurrent = max(self.max_concurrent, sum(len(a.batch) for a in self._active))
        self.largest_batch = max(self.largest_batch, len(batch))
        if len(batch) > 1:
            self.batched += len(batch)

    def _finish_setups(self):
        for sid in list(self._setting_up.keys()):
            e = self._scans.get(sid)
            if e is None or not e.ready:
                continue
            waiting = self._setting_up.pop(sid)
            e.busy = False
            if (getattr(e.error, "status", None) == M.MM_ERR_OOM and (self._active or self._setting_up)):
                # set up again once the work in flight has given memory back
                self._reserved.pop(sid, None)
                del self._scans[sid]
                e.ctx.close()
                self._oom_wait = True
                self.oom_requeued += len(waiting)
                with self._lock:
                    self._pending.extendleft(reversed(waiting))
                continue
            if e.error is not None:
                self._reserved.pop(sid, None)
                for _, fut in waiting:
                    fut.set_exception(e.error)
                continue
            # the requests that ask for the same run as the first go now; the rest wait for the scan
            k0 = self._key(waiting[0][0])
            first = [w for w in waiting if self._key(w[0]) == k0][:self.max_batch]
            rest = [w for w in waiting if all(w is not f for f in first)]
            if rest:
                with self._lock:
                    self._pending.extendleft(reversed(rest))
            self._start_solve(first, e, cached=False)
            self._reserved.pop(sid, None)          # the first solve has allocated its state

    def _drop_failed(self, a, ex):
        """A solve that raised fails its own requests; its scan's context is closed and forgotten (its
        state is unknown), so a later request on the scan sets it up again."""
        for _, fut in a.batch:
            if not fut.done():
                fut.set_exception(ex)
        sid = a.batch[0][0].scan_id
        if self._scans.get(sid) is a.entry:
            del self._scans[sid]
            try:
                a.entry.ctx.close()
            except Exception:
                pass
        self.failed += len(a.batch)

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
                self._oom_wait = False
                self._judge_coarse(a, info)
                if a.entry.harvesting:
                    # deflation basis from this M_BD run's Lanczos vectors, off the critical path
                    a.entry.harvesting = False
                    self._pool.submit(self._coarse_from_solve, a.entry)
                else:
                    a.entry.busy = False
                a.entry.last_used = now
                for i, (req, fut) in enumerate(a.batch):
                    self.latencies.append(now - req.arrival)
                    self.completed += 1
                    fut.set_result(MapResult(x[i], info[i], now - req.arrival, a.t_start - req.arrival, a.cached,
                                             len(a.batch)))
            else:
                still.append(a)
        self._active = still
        return progressed

    def _judge_coarse(self, a, info):
        """Harvest mode: remember the products of the scan's M_BD run, and compare the first M_2l
        run with them; a coarse space that saves less than min_coarse_gain is dropped."""
        e = a.entry
        its = [float(i.get("iters", 0)) for i in info if i.get("status") == "MM_OK"]
        if not its or self.coarse_mode != "harvest":
            return
        mean = sum(its) / len(its)
        if a.precond == M.MM_PRECOND_BD and e.bd_iters is None:
            e.bd_iters = mean
        elif a.precond == M.MM_PRECOND_2L and not e.coarse_checked and e.bd_iters:
            e.coarse_checked = True
            if mean > (1.0 - self.min_coarse_gain) * e.bd_iters:
                e.has_coarse = False
                e.coarse_useless = True
                self.coarse_disabled += 1

    def _fail_all(self, ex):
        with self._lock:
            pending = list(self._pending)
            self._pending.clear()
        for _, fut in pending:
            if not fut.done():
                fut.set_exception(ex)
        for a in self._active:
            for _, fut in a.batch:
                if not fut.done():
                    fut.set_exception(ex)
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
                if self._oom_wait and not self._active and not self._setting_up:
                    self._oom_wait = False     # nothing left to give memory back: try again
                if self._release:
                    with self._lock:
                        need, self._release = self._release, 0
                    self._evict_idle(need)
                self._finish_setups()
                self._admit()
                progressed = self._tick() if self._active else False
            except Exception as ex:   # a scheduler fault fails every request instead of hanging them
                self._fail_all(ex)
                self.error = ex
                return
            if not progressed:
                time.sleep(0.0002)
