"""The C ABI library loads and exports every entry point of include/mapmaker.h (CPU only)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mapmaker.h")


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mm_[A-Za-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1801_08937_gb300 import build as B
    from paper_1801_08937_gb300 import mapmaker as M
    if not os.path.exists(M.LIB_PATH):
        B.build()
    return M.load_library()


def test_header_declares_the_boundary():
    names = declared()
    for required in ("mm_setup_pointing", "mm_build_bd", "mm_build_coarse", "mm_apply_A", "mm_solve"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1801_08937_gb300 import mapmaker as M
    out = subprocess.run(["nm", "-D", "--defined-only", M.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (mm_[A-Za-z_0-9]+)\b", out))
    for name in declared():
        assert name in exported, name
        assert hasattr(lib, name)


def test_binding_covers_every_symbol():
    from paper_1801_08937_gb300 import mapmaker as M
    bound = {s[0] for s in M.SIGNATURES}
    assert set(declared()) <= bound


def test_estimate_bytes_is_host_arithmetic(lib):
    from paper_1801_08937_gb300 import mapmaker as M
    small = M.estimate_bytes(1 << 20, 1024, 8, 512, 1, 100, 16)
    big = M.estimate_bytes(1 << 27, 65536, 128, 2048, 1, 200, 32)
    assert 0 < small < big
    # one more right-hand side needs at least its timeline
    assert M.estimate_bytes(1 << 20, 1024, 8, 512, 2, 100, 16) - small >= (1 << 20) * 8


def test_no_oracle_in_product_path():
    pkg = os.path.join(ROOT, "paper_1801_08937_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f


def test_create_without_a_device_fails_cleanly(lib):
    """No usable GPU: mm_create returns an error status and no context; the NULL-context calls are safe."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import ctypes as C
    from paper_1801_08937_gb300 import mapmaker as M
    h = C.c_void_p()
    assert lib.mm_create(C.byref(h), 0, None, M.MM_FP64) == M.MM_ERR_CUDA
    assert h.value is None
    assert lib.mm_destroy(None) == M.MM_OK
    assert lib.mm_last_error(None) == b"null context"


def test_estimate_bytes_is_host_arithmetic_and_grows_with_the_problem(lib):
    from paper_1801_08937_gb300 import mapmaker as M
    base = dict(n_samples=1 << 20, n_pix=4096, n_bands=8, half_bw=512, nrhs=1, m_max=100, k=32)

    def est(prec=M.MM_FP64, **over):
        a = dict(base)
        a.update(over)
        return M.estimate_bytes(a["n_samples"], a["n_pix"], a["n_bands"], a["half_bw"], a["nrhs"], a["m_max"],
                                a["k"], prec)

    b0 = est()
    assert b0 > (1 << 20) * 8                              # at least the pointing
    for key, val in (("n_samples", 1 << 21), ("n_pix", 8192), ("nrhs", 4), ("m_max", 200), ("k", 64)):
        assert est(**{key: val}) > b0, key
    # float32 timelines, plus double-float weights for the refinement residuals
    assert est(M.MM_FP32_MIXED) == b0 - (1 << 20) * 4 + (1 << 20) * 16


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    """No libmapmaker.so: loading raises instead of falling back to anything else."""
    from paper_1801_08937_gb300 import mapmaker as M
    monkeypatch.setattr(M, "_lib", None)
    with pytest.raises(RuntimeError, match="no fallback"):
        M.load_library(str(tmp_path / "libmapmaker.so"))


def test_binding_marshals_arrays_without_copying_what_it_can_pass():
    import numpy as np
    from paper_1801_08937_gb300 import mapmaker as M
    a = np.arange(6, dtype=np.float64)
    p, mem, keep = M._arg(a, np.float64)
    assert p.value == a.ctypes.data and mem == M.MM_HOST and keep is a
    p, mem, keep = M._arg(a.astype(np.float32), np.float64)          # converted copy for an input
    assert keep.dtype == np.float64 and np.array_equal(keep, a)
    with pytest.raises(TypeError):
        M._arg(a.astype(np.float32), np.float64, writable=True)      # an output is never silently copied
    with pytest.raises(TypeError):
        M._arg(a[::2], np.float64, writable=True)
    torch = pytest.importorskip("torch")
    t = torch.zeros(4, dtype=torch.float64)
    p, mem, keep = M._arg(t, np.float64)
    assert p.value == t.data_ptr() and mem == M.MM_HOST
    with pytest.raises(TypeError):
        M._arg(t.float(), np.float64)
    with pytest.raises(ValueError):
        M._arg(torch.zeros((4, 4), dtype=torch.float64).t(), np.float64)
    assert M._mem(M.MM_HOST, None) == M.MM_HOST
    with pytest.raises(ValueError):
        M._mem(M.MM_HOST, M.MM_DEVICE)


def test_binding_signatures_match_the_header():
    """Every entry point of the binding passes as many arguments as include/mapmaker.h declares."""
    from paper_1801_08937_gb300 import mapmaker as M
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    decls = {}
    for m in re.finditer(r"\b(mm_[A-Za-z_0-9]+)\s*\(([^;{]*?)\)\s*;", src, flags=re.S):
        params = m.group(2).strip()
        n = 0 if params in ("", "void") else params.count(",") + 1
        decls[m.group(1)] = n
    bound = {name: len(args) for name, _res, args in M.SIGNATURES}
    missing = sorted(set(decls) - set(bound))
    assert not missing, missing
    for name, n in decls.items():
        assert bound[name] == n, (name, bound[name], n)


def test_binding_argument_types_match_the_header():
    """Argument kinds agree position by position: pointers, 64-bit and 32-bit integers (enums are
    ints), doubles, so ctypes never passes a value of the wrong width."""
    import ctypes as C
    from paper_1801_08937_gb300 import mapmaker as M
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)

    def kind_c(param):
        param = " ".join(param.split())
        if "*" in param or param.startswith("mm_reduce_fn"):
            return "ptr"
        if param.startswith("int64_t"):
            return "i64"
        if param.startswith(("int32_t", "int ", "mm_precision", "mm_precond")):
            return "i32"
        if param.startswith("double"):
            return "f64"
        raise AssertionError(param)

    def kind_py(t):
        if t in (C.c_void_p, C.c_char_p) or hasattr(t, "_type_") and isinstance(t._type_, type):
            return "ptr"
        if t is C.c_int64 or t is C.c_longlong:
            return "i64"
        if t in (C.c_int32, C.c_int):
            return "i32"
        if t is C.c_double:
            return "f64"
        raise AssertionError(t)

    sig = {name: args for name, _res, args in M.SIGNATURES}
    for m in re.finditer(r"\b(mm_[A-Za-z_0-9]+)\s*\(([^;{]*?)\)\s*;", src, flags=re.S):
        params = [q for q in m.group(2).split(",") if q.strip() not in ("", "void")]
        want = [kind_c(q.strip()) for q in params]
        got = [kind_py(t) for t in sig[m.group(1)]]
        assert want == got, (m.group(1), want, got)


class _RecordingLib:
    """Stands in for libmapmaker.so: records every entry point called (returns MM_OK)."""

    def __init__(self):
        self.calls = []

    def __getattr__(self, name):
        def fn(*args):
            self.calls.append(name)
            return 0
        return fn


def _fake_context(n_pix=4, n_samples=64):
    from paper_1801_08937_gb300 import mapmaker as M
    c = object.__new__(M.Context)
    c.lib = _RecordingLib()
    c.h = None
    c.device = 0
    c.precision = M.MM_FP64
    c.n_pix = n_pix
    c.n_samples = n_samples
    return c


def test_binding_refuses_arrays_of_the_wrong_size_before_any_call():
    """x must hold a whole number of [n_pix][3] maps and a caller's output at least as many values
    as the call writes: otherwise ValueError, and no entry point is called (an undersized output
    would be written past its end)."""
    import numpy as np
    c = _fake_context()
    n = 3 * c.n_pix
    for call in (lambda x, o: c.apply_A(x, out=o), lambda x, o: c.apply_precond(0, x, out=o)):
        with pytest.raises(ValueError):
            call(np.zeros(n + 1), None)                         # not a whole number of maps
        with pytest.raises(ValueError):
            call(np.zeros(2 * n), np.zeros(2 * n - 1))          # output one value short
        with pytest.raises(ValueError):
            call(np.zeros(0), None)
    with pytest.raises(ValueError):
        c.rhs(np.zeros(c.n_samples), out=np.zeros(n - 3))
    with pytest.raises(ValueError):
        c.rhs(np.zeros(c.n_samples + 5))
    with pytest.raises(ValueError):
        c.solve(np.zeros(2 * c.n_samples), out=np.zeros(n))     # two maps written, room for one
    with pytest.raises(ValueError):
        c.solve(np.zeros(2 * c.n_samples), rhs_len=[10])        # one length for two right-hand sides
    with pytest.raises(ValueError):
        c.set_coarse(np.zeros(n + 2))
    with pytest.raises(ValueError):
        c.setup_pointing(np.zeros(10, np.int32), np.zeros(9, np.float32), [0, 10], [0], np.ones(3), c.n_pix)
    assert c.lib.calls == []
    # well-formed calls go through
    c.apply_A(np.zeros(2 * n), out=np.zeros(2 * n))
    c.rhs(np.zeros(c.n_samples))
    assert c.lib.calls == ["mm_apply_A", "mm_rhs"]


def test_binding_refuses_host_outputs_for_device_inputs_and_the_noalloc_host_arrays():
    import numpy as np
    torch = pytest.importorskip("torch")
    c = _fake_context()
    n = 3 * c.n_pix
    x = torch.zeros(n, dtype=torch.float64)
    with pytest.raises(ValueError):
        c.apply_precond_2l_noalloc(x, torch.zeros(n, dtype=torch.float64))   # host tensors
    with pytest.raises(ValueError):
        c.apply_precond_2l_noalloc(np.zeros(n), np.zeros(n))
    assert c.lib.calls == []
