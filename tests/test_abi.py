"""The C-ABI library builds, loads and exports every entry point include/lcs_bound.h declares.

No GPU: only calls that need no device (status strings, defaults, argument
validation that happens before any CUDA call).
"""
import ctypes
import os
import re

import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "lcs_bound.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[\w]+\s*\*?\s*(lcs_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def L():
    from paper_2407_10925_gb300 import binding

    return binding.lib()


def test_header_declares_the_documented_api():
    names = declared_functions()
    for required in ["lcs_bound_create", "lcs_bound_iterate", "lcs_bound_read", "lcs_bound_destroy",
                     "lcs_bound_set_start", "lcs_bound_export", "lcs_bound_errstr", "lcs_sweep_fx"]:
        assert required in names


def test_every_declared_symbol_is_exported(L):
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert missing == []


def test_status_strings(L):
    from paper_2407_10925_gb300 import binding

    for st in range(9):
        assert binding.lcs_bound_errstr(st) != "unknown status"
    assert binding.lcs_bound_errstr(0) == "ok"


def test_default_opts(L):
    from paper_2407_10925_gb300 import binding

    o = binding.lcs_bound_default_opts()
    assert (o.check_every, o.r_mode, o.f_mode, o.frac_bits, o.symmetry) == (0, 0, 0, 44, 1)


@pytest.mark.parametrize("shape", [(1, 2, 3), (2, 1, 3), (2, 2, 0), (2, 17, 1), (2, 2, 20)])
def test_bad_shapes_rejected_before_any_device_call(L, shape):
    from paper_2407_10925_gb300 import binding

    with pytest.raises(binding.LcsError) as e:
        binding.lcs_bound_create(*shape)
    assert e.value.status == binding.LCS_EINVAL


def test_bad_options_rejected(L):
    from paper_2407_10925_gb300 import binding

    o = binding.lcs_bound_default_opts()
    o.frac_bits = 70
    with pytest.raises(binding.LcsError) as e:
        binding.lcs_bound_create(2, 2, 3, o)
    assert e.value.status == binding.LCS_EINVAL
    o = binding.lcs_bound_default_opts()
    o.f_mode = 1  # every non-empty advance set: compiled for sigma = 2 (d = 2, 3) and (3, 2) only
    with pytest.raises(binding.LcsError) as e:
        binding.lcs_bound_create(4, 2, 3, o)
    assert e.value.status == binding.LCS_EUNSUPPORTED
    o.f_mode = 2
    with pytest.raises(binding.LcsError) as e:
        binding.lcs_bound_create(2, 2, 3, o)
    assert e.value.status == binding.LCS_EINVAL


def test_null_handle_calls_fail_cleanly(L):
    from paper_2407_10925_gb300 import binding

    assert L.lcs_bound_iterate(None, 1) == binding.LCS_EINVAL
    assert L.lcs_bound_save(None, b"/nonexistent/x") == binding.LCS_EINVAL
    assert L.lcs_bound_restore(None, b"/nonexistent/x") == binding.LCS_EINVAL
    assert L.lcs_bound_export_stored_fx(None, 0, None, 0) == binding.LCS_EINVAL
    assert L.lcs_bound_orbit_size(None, None) == binding.LCS_EINVAL
    assert L.lcs_bound_set_start_orbit_fx(None, None, 0) == binding.LCS_EINVAL
    assert L.lcs_bound_export_orbit_fx(None, 0, None, 0) == binding.LCS_EINVAL
    assert L.lcs_bound_read(None, None, None, None, None, None) == binding.LCS_EINVAL
    L.lcs_bound_destroy(None)
    assert L.lcs_host_free(None) == binding.LCS_OK
    assert L.lcs_host_free(12345) == binding.LCS_EINVAL  # not a buffer of lcs_host_alloc
    assert L.lcs_host_alloc(0, None) == binding.LCS_EINVAL


def test_missing_library_fails_loudly(monkeypatch):
    """Without the CUDA library (not built and nvcc absent) every entry point
    raises: the binding has no CPU path to fall back to."""
    from paper_2407_10925_gb300 import binding

    def no_nvcc():
        raise RuntimeError("nvcc not found: the CUDA library cannot be built")

    monkeypatch.setattr(binding, "_lib", None)
    monkeypatch.setattr(binding._build, "up_to_date", lambda: False)
    monkeypatch.setattr(binding._build, "_nvcc", no_nvcc)
    with pytest.raises(RuntimeError, match="nvcc not found"):
        binding.lib()
    with pytest.raises(RuntimeError, match="nvcc not found"):
        binding.LcsBound(2, 2, 8)
    with pytest.raises(RuntimeError, match="nvcc not found"):
        binding.lcs_bound_default_opts()


def _split_params(params):
    if params in ("", "void"):
        return []
    out, depth, cur = [], 0, ""
    for ch in params:
        depth += ch in "(["
        depth -= ch in ")]"
        if ch == "," and depth == 0:
            out.append(cur.strip())
            cur = ""
        else:
            cur += ch
    return out + [cur.strip()]


def _declarations():
    """(return type, name, parameter count, parameters) of every function the header declares"""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    out = []
    for m in re.finditer(r"^\s*((?:const\s+)?[\w]+\s*\*?)\s*(lcs_\w+)\s*\(([^;]*?)\)\s*;", text, flags=re.M | re.S):
        ret, name, params = m.group(1).replace(" ", ""), m.group(2), _split_params(m.group(3).strip())
        out.append((ret, name, len(params), params))
    return out


def test_binding_signatures_match_the_header(L):
    """Every declared function has ctypes argtypes of the header's arity and
    the restype of its C return type, so a changed declaration cannot be
    called with stale marshalling."""
    import ctypes

    want_res = {"lcs_status": ctypes.c_int, "void": None, "constchar*": ctypes.c_char_p, "int64_t": ctypes.c_int64}
    decls = _declarations()
    assert len(decls) == len(declared_functions())
    scalars = {"int": ctypes.c_int, "int64_t": ctypes.c_int64, "uint64_t": ctypes.c_uint64, "double": ctypes.c_double,
               "float": ctypes.c_float, "lcs_status": ctypes.c_int, "size_t": ctypes.c_size_t}
    for ret, name, n, params in decls:
        fn = getattr(L, name)
        assert fn.argtypes is not None and len(fn.argtypes) == n, (name, n, fn.argtypes)
        assert ret in want_res, (name, ret)
        assert fn.restype == want_res[ret], (name, ret, fn.restype)
        for param, ct in zip(params, fn.argtypes):
            if re.search(r"\(\s*\*\s*\w+\s*\)\s*\(", param):  # a function pointer: a ctypes callback type
                assert issubclass(ct, ctypes._CFuncPtr), (name, param, ct)
            elif "*" in param:  # any other pointer: void*, char*, or a pointer to a struct or scalar
                assert ct in (ctypes.c_void_p, ctypes.c_char_p) or issubclass(ct, ctypes._Pointer), (name, param, ct)
            else:
                ctype = param.replace("const ", "").split()[0]
                assert ct == scalars[ctype], (name, param, ct)


def test_product_never_reaches_the_oracle():
    """The oracle is test infrastructure.  The package (Python, CUDA and the C
    header) never names it.  bench.py imports it only in its CPU-sample
    functions (the cpu_baseline leg and the reference arm), and the entry
    module only in build() and smoke()."""
    import ast

    pkg = os.path.join(ROOT, "paper_2407_10925_gb300")
    for base, _, files in os.walk(pkg):
        if "_build" in base:
            continue
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".c", ".cpp")):
                text = open(os.path.join(base, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", text, flags=re.M), f
                assert "lcs_oracle" not in text and "orc_" not in text, f
    assert "oracle" not in open(HEADER).read().lower()

    allowed = {"bench.py": {"window_arguments", "_oracle_window", "oracle_sample"},
               "__graft_entry__.py": {"build", "smoke"}}
    for name, funcs in allowed.items():
        tree = ast.parse(open(os.path.join(ROOT, name)).read())
        found = set()
        for fn in ast.walk(tree):
            if isinstance(fn, ast.FunctionDef):
                for node in ast.walk(fn):
                    if isinstance(node, ast.Import) and any(a.name.split(".")[0] == "oracle" for a in node.names):
                        found.add(fn.name)
                    if isinstance(node, ast.ImportFrom) and (node.module or "").split(".")[0] == "oracle":
                        found.add(fn.name)
        top = [n for n in tree.body if isinstance(n, (ast.Import, ast.ImportFrom))]
        assert not any("oracle" in ast.dump(n) for n in top), name  # no module-level import
        assert found <= funcs, (name, found)


def test_overlapping_buffers_rejected_before_any_device_call(L):
    """The stateless entry points refuse an output that shares a byte with an
    input (or, for the one that allocates nothing, results inside a vector or
    each other) before touching the device.  The addresses are never read."""
    import ctypes

    from paper_2407_10925_gb300 import binding

    n = 2 ** 8  # (2, 2, 2): 256 states, 2048 bytes per vector
    base = 1 << 40
    v0, v1 = base, base + 4 * 8 * n

    def noalloc(prev, out, R, arg):
        arr = (ctypes.c_void_p * 2)(*prev)
        return L.lcs_sweep_incr_fx_noalloc(2, 2, 4, 44, 0, arr, out, R, arg, None)

    def sweep(prev, out):
        arr = (ctypes.c_void_p * 2)(*prev)
        return L.lcs_sweep_fx(2, 2, 4, 0, 44, arr, out, None)

    ok_out, R, arg = base + 8 * 8 * n, base + 16 * 8 * n, base + 16 * 8 * n + 64
    # an output vector that starts inside an input, or ends inside one (offset views)
    for out in (v0 + 8, v1 - 8 * n + 8, v1 + 8 * (n - 1)):
        assert noalloc([v0, v1], out, R, arg) == binding.LCS_EINVAL
        assert sweep([v0, v1], out) == binding.LCS_EINVAL
    # the 8-byte results inside a vector, or on top of each other
    assert noalloc([v0, v1], ok_out, v0 + 8 * (n - 1), arg) == binding.LCS_EINVAL
    assert noalloc([v0, v1], ok_out, R, ok_out + 8) == binding.LCS_EINVAL
    assert noalloc([v0, v1], ok_out, R, R + 4) == binding.LCS_EINVAL
    assert "overlap" in binding.lcs_bound_last_error() or "inside" in binding.lcs_bound_last_error()


def test_binding_checks_vector_sizes_before_the_call(L):
    """The C side receives bare pointers and cannot see a short buffer: the
    binding checks the count and the length of every vector first."""
    import numpy as np

    from paper_2407_10925_gb300 import binding

    n = 2 ** 8
    good = [np.zeros(n, dtype=np.int64) for _ in range(2)]
    short = np.zeros(n - 1, dtype=np.int64)
    one = np.zeros(1, dtype=np.int64)
    empty = np.zeros(0, dtype=np.int64)
    cases = [
        lambda: binding.lcs_sweep_incr_fx_noalloc(2, 2, 4, [good[0], short], good[1], one, one),
        lambda: binding.lcs_sweep_incr_fx_noalloc(2, 2, 4, good[:1], good[1], one, one),
        lambda: binding.lcs_sweep_incr_fx_noalloc(2, 2, 4, good, short, one, one),
        lambda: binding.lcs_sweep_incr_fx_noalloc(2, 2, 4, good, good[1], empty, one),
        lambda: binding.lcs_sweep_incr_fx_noalloc(2, 2, 4, good, good[1], one, empty),
        lambda: binding.lcs_sweep_fx(2, 2, 4, [short, good[1]], good[0]),
        lambda: binding.lcs_sweep_fx(2, 2, 4, good, short),
        lambda: binding.lcs_sweep_fx(2, 2, 4, good + [good[0]], good[0]),
    ]
    for call in cases:
        with pytest.raises(ValueError):
            call()


def test_build_compiles_every_cuda_source():
    """build.py's list of translation units holds every .cu file of csrc/ once
    (a source left out would leave its kernels unlinked; the general kernels
    are spread over several units)."""
    import os

    from paper_2407_10925_gb300 import build

    csrc = os.path.join(os.path.dirname(os.path.abspath(build.__file__)), "csrc")
    on_disk = sorted(f for f in os.listdir(csrc) if f.endswith(".cu"))
    assert sorted(build.SOURCES) == on_disk
    assert len(set(build.SOURCES)) == len(build.SOURCES)
