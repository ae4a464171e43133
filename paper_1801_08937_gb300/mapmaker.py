"""ctypes binding of libmapmaker.so (include/mapmaker.h).

Argument marshalling only: every computation runs in the library's CUDA
kernels.  Arrays may be numpy arrays (host memory, passed as MM_HOST) or
torch tensors (device memory on the context's GPU, passed as MM_DEVICE; CPU
tensors are passed as host memory).  The library must have been built
(``paper_1801_08937_gb300.build.build()``); loading fails loudly otherwise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmapmaker.so")

MM_OK, MM_ERR_ARG, MM_ERR_OOM, MM_ERR_CUDA, MM_ERR_STATE = 0, 1, 2, 3, 4
MM_ERR_NOT_CONVERGED, MM_ERR_BREAKDOWN, MM_ERR_SINGULAR, MM_ERR_TIMEOUT, MM_ERR_REDUCE = 5, 6, 7, 8, 9
MM_FP64, MM_FP32_MIXED = 0, 1
MM_PRECOND_BD, MM_PRECOND_2L = 0, 1
MM_HOST, MM_DEVICE = 0, 1

STATUS_NAMES = {0: "MM_OK", 1: "MM_ERR_ARG", 2: "MM_ERR_OOM", 3: "MM_ERR_CUDA", 4: "MM_ERR_STATE",
                5: "MM_ERR_NOT_CONVERGED", 6: "MM_ERR_BREAKDOWN", 7: "MM_ERR_SINGULAR", 8: "MM_ERR_TIMEOUT",
                9: "MM_ERR_REDUCE"}


class mm_solve_info(C.Structure):
    _fields_ = [("iters", C.c_int32), ("status", C.c_int32), ("rel_res", C.c_double),
                ("true_rel_res", C.c_double), ("t_solve_ms", C.c_double),
                ("refinements", C.c_int32), ("precond_used", C.c_int32)]


# (name, restype, argtypes) for every entry point of include/mapmaker.h
_VP, _I32, _I64, _D = C.c_void_p, C.c_int32, C.c_int64, C.c_double
SIGNATURES = [
    ("mm_create", C.c_int, [C.POINTER(C.c_void_p), C.c_int, _VP, C.c_int]),
    ("mm_destroy", C.c_int, [_VP]),
    ("mm_last_error", C.c_char_p, [_VP]),
    ("mm_setup_pointing", C.c_int, [_VP, _I64, _I32, _I32, _VP, _VP, _I32, _VP, _VP, _I32, _I32, _VP, C.c_int]),
    ("mm_build_bd", C.c_int, [_VP, _D, C.POINTER(_I32)]),
    ("mm_rhs", C.c_int, [_VP, _VP, _VP, _I32, C.c_int]),
    ("mm_apply_A", C.c_int, [_VP, _VP, _VP, _I32, C.c_int]),
    ("mm_apply_precond", C.c_int, [_VP, C.c_int, _VP, _VP, _I32, C.c_int]),
    ("mm_build_coarse", C.c_int, [_VP, _VP, _I32, _D, _I32, _D, C.POINTER(_I32), C.c_int]),
    ("mm_set_coarse", C.c_int, [_VP, _I32, _VP, C.c_int]),
    ("mm_get_coarse", C.c_int, [_VP, _VP, _VP, C.POINTER(_I32)]),
    ("mm_solve", C.c_int, [_VP, _VP, _VP, _I32, _VP, C.c_int, _D, _I32, C.POINTER(mm_solve_info), C.c_int]),
    ("mm_set_option", C.c_int, [_VP, C.c_char_p, _D]),
    ("mm_get_option", C.c_int, [_VP, C.c_char_p, C.POINTER(_D)]),
    ("mm_solve_begin", C.c_int, [_VP, _VP, _I32, _VP, C.c_int, _D, _I32, C.c_int]),
    ("mm_solve_step", C.c_int, [_VP, _I32, C.POINTER(_I32)]),
    ("mm_solve_end", C.c_int, [_VP, _VP, C.POINTER(mm_solve_info), C.c_int]),
    ("mm_estimate_bytes", C.c_int64, [_I64, _I32, _I32, _I32, _I32, _I32, _I32, C.c_int]),
    ("mm_apply_precond_2l_noalloc", C.c_int, [_VP, _VP, _VP, _I32]),
    ("mm_solve_launch", C.c_int, [_VP, _I32]),
    ("mm_build_coarse_from_solve", C.c_int, [_VP, _I32, _D, C.POINTER(_I32)]),
    ("mm_solve_poll", C.c_int, [_VP, C.POINTER(_I32), C.POINTER(_I32)]),
    ("mm_set_templates", C.c_int, [_VP, _I32, _I32, _VP, _VP, _I32, _I32, C.c_int]),
    ("mm_export_coarse", C.c_int, [_VP, _VP, C.POINTER(_I64)]),
    ("mm_import_coarse", C.c_int, [_VP, _VP, _I64]),
    ("mm_fma_peak", C.c_int, [C.c_int, C.c_int, _D, C.POINTER(_D)]),
    ("mm_set_reduction", C.c_int, [_VP, _VP, _VP, C.c_int]),
]

# mm_reduce_fn: int fn(void* buf, int64_t count, int32_t elem_bytes, void* user)
REDUCE_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_int64, C.c_int32, C.c_void_p)

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libmapmaker.so and bind every entry point (raises if absent)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1801_08937_gb300.build.build() "
                           "(nvcc, sm_103a); there is no fallback implementation")
    lib = C.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class MapMakerError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _arg(x, np_dtype, writable=False):
    """(pointer, mem, keepalive) for a numpy array or a torch tensor."""
    if x is None:
        return None, MM_HOST, None
    if _is_torch(x):
        import torch
        want = {np.float64: torch.float64, np.float32: torch.float32, np.int32: torch.int32,
                np.int64: torch.int64}[np_dtype]
        if x.dtype != want:
            raise TypeError(f"tensor dtype {x.dtype}, expected {want}")
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(x.data_ptr()), (MM_DEVICE if x.is_cuda else MM_HOST), x
    a = np.asarray(x)
    if a.dtype != np_dtype or not a.flags.c_contiguous:
        if writable:
            raise TypeError(f"output array must be a C-contiguous {np.dtype(np_dtype)} array")
        a = np.ascontiguousarray(a, dtype=np_dtype)
    return C.c_void_p(a.ctypes.data), MM_HOST, a


def _numel(x) -> int:
    return int(x.numel()) if _is_torch(x) else int(np.asarray(x).size)


def _device_of(x):
    """CUDA device index of a torch tensor on the GPU, else None (host memory)."""
    return x.device.index if (_is_torch(x) and x.is_cuda) else None


def _mem(*mems):
    ms = {m for m in mems if m is not None}
    if len(ms) > 1:
        raise ValueError("mix of host and device arrays in one call")
    return ms.pop() if ms else MM_HOST


class Context:
    """One map-making problem on one GPU (a ``mm_ctx``)."""

    def __init__(self, device: int = 0, stream=None, precision: int = MM_FP64):
        self.lib = load_library()
        h = C.c_void_p()
        st = self.lib.mm_create(C.byref(h), int(device), C.c_void_p(stream or 0), int(precision))
        if st != MM_OK:
            raise MapMakerError(st, "mm_create failed")
        self.h = h
        self.device = int(device)
        self.precision = precision
        self.n_pix = 0
        self.n_samples = 0

    def close(self):
        if getattr(self, "h", None):
            self.lib.mm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, ok=(MM_OK,)):
        if st not in ok:
            raise MapMakerError(st, self.lib.mm_last_error(self.h).decode())
        return st

    def _count(self, x, per: int, what: str) -> int:
        """Number of right-hand sides (or vectors) in x, which must hold a whole number of them."""
        if per <= 0:
            return 1   # no pointing yet: the library answers MM_ERR_STATE before reading x
        n = _numel(x)
        if n == 0 or n % per:
            raise ValueError(f"{what} holds {n} elements, not a positive multiple of {per}")
        d = _device_of(x)
        if d is not None and d != self.device:
            raise ValueError(f"{what} is on cuda:{d}, the context on cuda:{self.device}")
        return n // per

    def _check_out(self, out, like, need: int, what: str):
        """A caller's output array must hold `need` elements and live where the input lives."""
        if _numel(out) < need:
            raise ValueError(f"{what} holds {_numel(out)} elements, the call writes {need}")
        if _device_of(out) != _device_of(like):
            raise ValueError(f"{what} and the input must both be host memory or both on cuda:{self.device}")

    @property
    def tod_dtype(self):
        return np.float32 if self.precision == MM_FP32_MIXED else np.float64

    # --- entry points, same names as the C ABI ---
    def setup_pointing(self, pix, psi, block_off, block_band, band, n_pix, n_det=1):
        band = np.ascontiguousarray(band, dtype=np.float64)
        if band.ndim == 1:
            band = band[None, :]
        p_pix, m1, k1 = _arg(pix, np.int32)
        p_psi, m2, k2 = _arg(psi, np.float32)
        bo = np.ascontiguousarray(block_off, dtype=np.int64)
        bb = np.ascontiguousarray(block_band, dtype=np.int32)
        n = int(bo[-1])
        if _numel(pix) != n or _numel(psi) != n:
            raise ValueError(f"pix and psi hold {_numel(pix)} and {_numel(psi)} samples, block_off ends at {n}")
        if bb.size != bo.size - 1:
            raise ValueError(f"block_band holds {bb.size} entries for {bo.size - 1} blocks")
        self._check(self.lib.mm_setup_pointing(
            self.h, n, int(n_det), int(n_pix), p_pix, p_psi, int(bo.shape[0] - 1),
            C.c_void_p(bo.ctypes.data), C.c_void_p(bb.ctypes.data), int(band.shape[0]),
            int(band.shape[1] - 1), C.c_void_p(band.ctypes.data), _mem(m1, m2)))
        self.n_pix = int(n_pix)
        self.n_samples = n

    def setup_scan(self, scan):
        """Pointing and weight of a synthetic scan object (pix, psi, blocks, bands)."""
        self.setup_pointing(scan.pix, scan.psi, scan.block_off, scan.block_band, scan.band,
                            scan.n_pix, n_det=scan.n_det)

    def set_templates(self, poly_order=-1, subscan_off=None, az_bin=None, n_az_bins=0, stokes=0):
        """Template filters F = F_B W^-1 F_G W^-1 F_B (mm_set_templates); subscan_off is host memory.
        stokes: 0 I, Q, U; 1 (or True) Q, U from d^-; 2 I from d^+."""
        so = None if subscan_off is None else np.ascontiguousarray(subscan_off, dtype=np.int64)
        pa, m1, k1 = _arg(az_bin, np.int32)
        self._check(self.lib.mm_set_templates(
            self.h, int(poly_order), 0 if so is None else int(so.shape[0] - 1),
            None if so is None else C.c_void_p(so.ctypes.data), pa, int(n_az_bins), int(stokes), _mem(m1)))

    def build_bd(self, rcond_min: float = 1e-3) -> int:
        n = C.c_int32(0)
        self._check(self.lib.mm_build_bd(self.h, float(rcond_min), C.byref(n)))
        return n.value

    def _map_out(self, like, nrhs):
        if like is not None and _is_torch(like) and like.is_cuda:
            import torch
            return torch.empty((nrhs, self.n_pix, 3), dtype=torch.float64, device=like.device)
        return np.empty((nrhs, self.n_pix, 3), dtype=np.float64)

    def rhs(self, tod, out=None):
        nrhs = self._count(tod, self.n_samples, "tod")
        if out is None:
            out = self._map_out(tod, nrhs)
        else:
            self._check_out(out, tod, nrhs * 3 * self.n_pix, "out")
        pt, m1, k1 = _arg(tod, self.tod_dtype)
        po, m2, k2 = _arg(out, np.float64, writable=True)
        self._check(self.lib.mm_rhs(self.h, pt, po, nrhs, _mem(m1, m2)))
        return out

    def apply_A(self, x, out=None):
        nrhs = self._count(x, 3 * self.n_pix, "x")
        if out is None:
            out = self._map_out(x, nrhs)
        else:
            self._check_out(out, x, nrhs * 3 * self.n_pix, "out")
        px, m1, k1 = _arg(x, np.float64)
        po, m2, k2 = _arg(out, np.float64, writable=True)
        self._check(self.lib.mm_apply_A(self.h, px, po, nrhs, _mem(m1, m2)))
        return out

    def apply_precond(self, which, x, out=None):
        nrhs = self._count(x, 3 * self.n_pix, "x")
        if out is None:
            out = self._map_out(x, nrhs)
        else:
            self._check_out(out, x, nrhs * 3 * self.n_pix, "out")
        px, m1, k1 = _arg(x, np.float64)
        po, m2, k2 = _arg(out, np.float64, writable=True)
        self._check(self.lib.mm_apply_precond(self.h, int(which), px, po, nrhs, _mem(m1, m2)))
        return out

    def apply_precond_2l_noalloc(self, x, out):
        """y = M_2l x into a caller-owned device array; the call allocates no device memory."""
        nrhs = self._count(x, 3 * self.n_pix, "x")
        if _device_of(x) is None or _device_of(out) is None:
            raise ValueError("apply_precond_2l_noalloc takes device arrays only")
        self._check_out(out, x, nrhs * 3 * self.n_pix, "out")
        px, m1, k1 = _arg(x, np.float64)
        po, m2, k2 = _arg(out, np.float64, writable=True)
        self._check(self.lib.mm_apply_precond_2l_noalloc(self.h, px, po, nrhs))
        return out

    def build_coarse(self, b=None, m_max=200, eps_arn=1e-8, k=32, eps_lambda=0.2) -> int:
        kout = C.c_int32(0)
        pb, m1, kb = _arg(b, np.float64)
        self._check(self.lib.mm_build_coarse(self.h, pb, int(m_max), float(eps_arn), int(k),
                                             float(eps_lambda), C.byref(kout), m1))
        return kout.value

    def build_coarse_from_solve(self, k=32, eps_lambda=0.2) -> int:
        kout = C.c_int32(0)
        self._check(self.lib.mm_build_coarse_from_solve(self.h, int(k), float(eps_lambda), C.byref(kout)))
        return kout.value

    def set_coarse(self, Z):
        k = self._count(Z, 3 * self.n_pix, "Z")
        pz, m1, kz = _arg(Z, np.float64)
        self._check(self.lib.mm_set_coarse(self.h, k, pz, m1))

    def get_coarse(self):
        k = C.c_int32(0)
        self._check(self.lib.mm_get_coarse(self.h, None, None, C.byref(k)))
        Z = np.empty((k.value, self.n_pix, 3))
        ritz = np.empty(k.value)
        self._check(self.lib.mm_get_coarse(self.h, C.c_void_p(Z.ctypes.data), C.c_void_p(ritz.ctypes.data),
                                           C.byref(k)))
        return Z, ritz

    def set_reduction(self, fn, on_device=False):
        """Sum of partial products over ranks that each hold part of the timeline (mm_set_reduction).

        fn(arr) receives a numpy view (float32 or float64) of a host staging buffer and must replace it
        in place by its element-wise sum over all ranks (e.g. torch.distributed.all_reduce on
        torch.from_numpy(arr) with gloo); with on_device=True, fn(ptr, count, elem_bytes) receives the
        device pointer instead.  fn=None switches the reduction off."""
        if fn is None:
            self._check(self.lib.mm_set_reduction(self.h, None, None, 0))
            self._reduce_cb = None
            return

        def cb(ptr, count, elem, user):
            try:
                if on_device:
                    return int(fn(ptr, count, elem) or 0)
                ct = C.c_float if elem == 4 else C.c_double
                fn(np.ctypeslib.as_array((ct * count).from_address(ptr)))
                return 0
            except Exception:   # reported as MM_ERR_REDUCE by the library
                return 1

        self._reduce_cb = REDUCE_FN(cb)
        self._check(self.lib.mm_set_reduction(self.h, C.cast(self._reduce_cb, C.c_void_p), None,
                                              int(bool(on_device))))

    def export_coarse(self) -> bytes:
        """Checkpoint of the coarse space (Z, A Z, E^-1, Ritz values, operator fingerprint)."""
        n = C.c_int64(0)
        self._check(self.lib.mm_export_coarse(self.h, None, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        self._check(self.lib.mm_export_coarse(self.h, C.cast(buf, C.c_void_p), C.byref(n)))
        return buf.raw[:n.value]

    def import_coarse(self, data: bytes):
        """Install a checkpoint written by export_coarse for the same operator (MM_ERR_ARG otherwise)."""
        buf = C.create_string_buffer(bytes(data), len(data))
        self._check(self.lib.mm_import_coarse(self.h, C.cast(buf, C.c_void_p), len(data)))

    def solve(self, tod, precond=MM_PRECOND_BD, tol=1e-8, max_iter=500, rhs_len=None, out=None):
        nrhs = self._count(tod, self.n_samples, "tod")
        if out is None:
            out = self._map_out(tod, nrhs)
        else:
            self._check_out(out, tod, nrhs * 3 * self.n_pix, "out")
        if rhs_len is not None and np.asarray(rhs_len).size != nrhs:
            raise ValueError(f"rhs_len holds {np.asarray(rhs_len).size} lengths for {nrhs} right-hand sides")
        info = (mm_solve_info * nrhs)()
        pt, m1, k1 = _arg(tod, self.tod_dtype)
        po, m2, k2 = _arg(out, np.float64, writable=True)
        lens = None if rhs_len is None else np.ascontiguousarray(rhs_len, dtype=np.int64)
        st = self.lib.mm_solve(self.h, pt, po, nrhs, None if lens is None else C.c_void_p(lens.ctypes.data),
                               int(precond), float(tol), int(max_iter), info, _mem(m1, m2))
        self._check(st, ok=(MM_OK, MM_ERR_NOT_CONVERGED))
        return out, [_info_dict(i) for i in info]

    def solve_begin(self, tod, precond=MM_PRECOND_BD, tol=1e-8, max_iter=500, rhs_len=None):
        nrhs = self._count(tod, self.n_samples, "tod")
        if rhs_len is not None and np.asarray(rhs_len).size != nrhs:
            raise ValueError(f"rhs_len holds {np.asarray(rhs_len).size} lengths for {nrhs} right-hand sides")
        pt, m1, k1 = _arg(tod, self.tod_dtype)
        lens = None if rhs_len is None else np.ascontiguousarray(rhs_len, dtype=np.int64)
        self._keep = (k1, lens)
        self._nrhs = nrhs
        self._check(self.lib.mm_solve_begin(self.h, pt, nrhs, None if lens is None else C.c_void_p(lens.ctypes.data),
                                            int(precond), float(tol), int(max_iter), m1))

    def solve_step(self, n_iter: int) -> bool:
        done = C.c_int32(0)
        self._check(self.lib.mm_solve_step(self.h, int(n_iter), C.byref(done)))
        return bool(done.value)

    def solve_launch(self, n_iter: int):
        self._check(self.lib.mm_solve_launch(self.h, int(n_iter)))

    def solve_poll(self):
        """(ready, done): ready once the last launch's state read-back has landed."""
        r, d = C.c_int32(0), C.c_int32(0)
        self._check(self.lib.mm_solve_poll(self.h, C.byref(r), C.byref(d)))
        return bool(r.value), bool(d.value)

    def solve_end(self, out=None, like=None):
        if out is None:
            out = self._map_out(like, self._nrhs)
        elif _numel(out) < self._nrhs * 3 * self.n_pix:
            raise ValueError(f"out holds {_numel(out)} elements, the call writes {self._nrhs * 3 * self.n_pix}")
        info = (mm_solve_info * self._nrhs)()
        po, m, ko = _arg(out, np.float64, writable=True)
        st = self.lib.mm_solve_end(self.h, po, info, m)
        self._check(st, ok=(MM_OK, MM_ERR_NOT_CONVERGED))
        return out, [_info_dict(i) for i in info]

    def set_option(self, name: str, value: float):
        self._check(self.lib.mm_set_option(self.h, name.encode(), float(value)))

    def get_option(self, name: str) -> float:
        v = C.c_double(0)
        self._check(self.lib.mm_get_option(self.h, name.encode(), C.byref(v)))
        return v.value


def _info_dict(i):
    return dict(iters=i.iters, status=STATUS_NAMES.get(i.status, i.status), rel_res=i.rel_res,
                true_rel_res=i.true_rel_res, t_solve_ms=i.t_solve_ms, refinements=i.refinements,
                precond_used="M_2l" if i.precond_used == MM_PRECOND_2L else "M_BD")


def fma_peak(device=0, fp64=False, seconds=1.0) -> float:
    """Measured CUDA-core FMA rate of the device in flop/s (float32, or float64 with fp64=True)."""
    v = C.c_double(0)
    st = load_library().mm_fma_peak(int(device), int(bool(fp64)), float(seconds), C.byref(v))
    if st != MM_OK:
        raise MapMakerError(st, "mm_fma_peak failed")
    return v.value


def estimate_bytes(n_samples, n_pix, n_bands, half_bw, nrhs, m_max, k, precision=MM_FP64) -> int:
    return int(load_library().mm_estimate_bytes(int(n_samples), int(n_pix), int(n_bands), int(half_bw),
                                                int(nrhs), int(m_max), int(k), int(precision)))
