"""CPU oracle for the feasible-triplet sweep of arXiv 2407.10925 (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
legs may import this package.  The CUDA library never calls it.  The oracle
itself is the plain C file ``lcs_oracle.c`` next to this module; this module
compiles it with gcc and wraps it with ctypes (argument marshalling only).

Functions follow the paper's section 2.1: ``F`` is Eq. ineq3 built from
Algorithm 1's F_z, ``run`` is Algorithm 2 (FeasibleTriplet), ``check`` is the
W/E step of Algorithm 2 (Lemma 1's feasibility condition).  Two arithmetics:
``"f64"`` (IEEE double, round-to-nearest iterates, directed-rounding check)
and ``"fx"`` (int64 multiples of 2^-K, exact sums, floor means).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lcs_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liblcs_oracle.so")
_lock = threading.Lock()
_lib = None

DEFAULT_FRAC_BITS = 44
RN, RD, RU = 0, 1, 2


class OracleError(RuntimeError):
    pass


def build(force: bool = False, mutant: int = 0) -> str:
    """Compile the oracle into ``oracle/_build/liblcs_oracle.so`` (gcc, no FP contraction).

    ``mutant`` > 0 builds a deliberately wrong variant (``ORC_MUTANT``) for the
    mutation test of the pins.
    """
    os.makedirs(_BUILD, exist_ok=True)
    so = _SO if mutant == 0 else os.path.join(_BUILD, f"liblcs_oracle_mutant{mutant}.so")
    if force or not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(_SRC):
        tmp = so + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-Wall", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               f"-DORC_MUTANT={int(mutant)}", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, so)
    return so


class Result(ctypes.Structure):
    _fields_ = [
        ("iters_done", ctypes.c_int64),
        ("newest_row", ctypes.c_int64),
        ("have_check", ctypes.c_int64),
        ("kept_iter", ctypes.c_int64),
        ("argmin", ctypes.c_uint64),
        ("R_f64", ctypes.c_double), ("E_f64", ctypes.c_double),
        ("R_fx", ctypes.c_int64), ("E_fx", ctypes.c_int64),
        ("r_f64", ctypes.c_double), ("eps_f64", ctypes.c_double),
        ("r_fx", ctypes.c_int64), ("eps_fx", ctypes.c_int64),
        ("bound_rd", ctypes.c_double),
    ]


def _load(path):
    L = ctypes.CDLL(path)
    i64, u64, dbl, i32 = ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_int
    vp = ctypes.c_void_p
    L.orc_F_f64.argtypes = [i32, i32, i32, i32, i32, vp, u64, u64, vp]
    L.orc_F_fx.argtypes = [i32, i32, i32, i32, i32, vp, u64, u64, vp]
    L.orc_encode.argtypes = [i32, i32, i32, vp]
    L.orc_encode.restype = u64
    L.orc_decode.argtypes = [i32, i32, i32, u64, vp]
    L.orc_check_f64.argtypes = [i32, i32, i32, i32, vp, dbl, vp, vp, vp]
    L.orc_check_fx.argtypes = [i32, i32, i32, i32, i32, vp, i64, vp, vp, vp]
    L.orc_run_f64.argtypes = [i32, i32, i32, i64, i32, i32, i32, vp, vp, vp, ctypes.POINTER(Result)]
    L.orc_run_fx.argtypes = [i32, i32, i32, i64, i32, i32, i32, i32, vp, vp, vp, ctypes.POINTER(Result)]
    for name in ("orc_add_dir", "orc_mul_dir", "orc_div_dir"):
        getattr(L, name).argtypes = [dbl, dbl, i32]
        getattr(L, name).restype = dbl
    L.orc_F_fx_generated.argtypes = [i32, i32, i32, i32, vp, vp, u64, i32, vp, u64, vp]
    L.orc_splitmix64_at.argtypes = [u64, u64]
    L.orc_splitmix64_at.restype = u64
    L.orc_fx_to_double_rd.argtypes = [i64, i32]
    L.orc_fx_to_double_rd.restype = dbl
    if L.orc_result_size() != ctypes.sizeof(Result):
        raise OracleError("orc_result layout mismatch")
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _load(build())
    return _lib


class use_mutant:
    """Context manager: route every call of this module to a mutant build (tests only)."""

    def __init__(self, mutant: int):
        self.path = build(mutant=mutant)

    def __enter__(self):
        global _lib
        lib()
        self.saved = _lib
        _lib = _load(self.path)
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved


def _check(st: int, what: str):
    if st != 0:
        raise OracleError(f"{what} failed with status {st}")


def n_states(sigma: int, d: int, h: int) -> int:
    return sigma ** (d * h)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _ptr_array(vs):
    arr = (ctypes.c_void_p * len(vs))(*[v.ctypes.data for v in vs])
    return arr


def encode(sigma: int, d: int, h: int, digits) -> int:
    """Paper index of the state whose string j has digit digits[p][j] at position p (0 = head)."""
    X = np.ascontiguousarray(np.asarray(digits, dtype=np.int32).reshape(h, d))
    return int(lib().orc_encode(sigma, d, h, _ptr(X)))


def decode(sigma: int, d: int, h: int, x: int) -> np.ndarray:
    X = np.zeros((h, d), dtype=np.int32)
    _check(lib().orc_decode(sigma, d, h, x, _ptr(X)), "decode")
    return X


def strings_of(sigma: int, d: int, h: int, x: int):
    """The d strings of state x as tuples of letters (head first)."""
    X = decode(sigma, d, h, x)
    return [tuple(int(X[p, j]) for p in range(h)) for j in range(d)]


def F(sigma: int, d: int, h: int, vs, arith: str = "fx", f_mode: int = 0, mode: int = RN,
      frac_bits: int = DEFAULT_FRAC_BITS, x0: int = 0, x1: int | None = None) -> np.ndarray:
    """F(v_1, .., v_d) over states [x0, x1); vs[k-1] is the k-th argument v_k (Eq. ineq3)."""
    n = n_states(sigma, d, h)
    x1 = n if x1 is None else x1
    if len(vs) != d:
        raise ValueError("F takes d argument vectors")
    if arith == "f64":
        vs = [np.ascontiguousarray(v, dtype=np.float64) for v in vs]
        out = np.empty(x1 - x0, dtype=np.float64)
        _check(lib().orc_F_f64(sigma, d, h, f_mode, mode, _ptr_array(vs), x0, x1, _ptr(out)), "F_f64")
    elif arith == "fx":
        vs = [np.ascontiguousarray(v, dtype=np.int64) for v in vs]
        out = np.empty(x1 - x0, dtype=np.int64)
        _check(lib().orc_F_fx(sigma, d, h, f_mode, frac_bits, _ptr_array(vs), x0, x1, _ptr(out)), "F_fx")
    else:
        raise ValueError(arith)
    return out


def check(sigma: int, d: int, h: int, u, R, arith: str = "fx", f_mode: int = 0,
          frac_bits: int = DEFAULT_FRAC_BITS, want_W: bool = False):
    """(E, W): W = u + dR - F(u + (d-1)R, .., u), E = max(0, max W)  (Algorithm 2; Lemma 1)."""
    n = n_states(sigma, d, h)
    if arith == "f64":
        u = np.ascontiguousarray(u, dtype=np.float64)
        work = np.empty((d + 1) * n, dtype=np.float64)
        W = np.empty(n, dtype=np.float64) if want_W else None
        E = ctypes.c_double()
        _check(lib().orc_check_f64(sigma, d, h, f_mode, _ptr(u), float(R), _ptr(work),
                                   _ptr(W) if want_W else None, ctypes.byref(E)), "check_f64")
        return float(E.value), W
    u = np.ascontiguousarray(u, dtype=np.int64)
    work = np.empty((d + 1) * n, dtype=np.int64)
    W = np.empty(n, dtype=np.int64) if want_W else None
    E = ctypes.c_int64()
    _check(lib().orc_check_fx(sigma, d, h, f_mode, frac_bits, _ptr(u), int(R), _ptr(work),
                              _ptr(W) if want_W else None, ctypes.byref(E)), "check_fx")
    return int(E.value), W


def run(sigma: int, d: int, h: int, n_iters: int, arith: str = "fx", check_every: int = 0, r_mode: int = 0,
        f_mode: int = 0, frac_bits: int = DEFAULT_FRAC_BITS, start=None, want_u: bool = False) -> dict:
    """Algorithm 2 for n_iters iterations from ``start`` (d vectors v_0..v_{d-1}; default zeros).

    Returns a dict with the kept triplet, the last iteration's R/argmin/E, the
    rounded-down bound and ``iterates`` = [newest, 1 older, .., d-1 older].
    """
    n = n_states(sigma, d, h)
    dt = np.float64 if arith == "f64" else np.int64
    hist = np.zeros((d + 1, n), dtype=dt)
    if start is not None:
        for k in range(d):
            hist[k] = np.asarray(start[k], dtype=dt)
    work = np.empty((d + 1) * n, dtype=dt)
    u = np.empty(n, dtype=dt) if want_u else None
    res = Result()
    if arith == "f64":
        st = lib().orc_run_f64(sigma, d, h, n_iters, check_every, r_mode, f_mode, _ptr(hist), _ptr(work),
                               _ptr(u) if want_u else None, ctypes.byref(res))
    elif arith == "fx":
        st = lib().orc_run_fx(sigma, d, h, n_iters, check_every, r_mode, f_mode, frac_bits, _ptr(hist), _ptr(work),
                              _ptr(u) if want_u else None, ctypes.byref(res))
    else:
        raise ValueError(arith)
    _check(st, "run")
    rows = d + 1
    newest = int(res.newest_row)
    iterates = [hist[(newest - k) % rows].copy() for k in range(d)]
    out = {f: getattr(res, f) for f, _ in Result._fields_}
    out["iterates"] = iterates
    out["u"] = u
    out["arith"] = arith
    out["frac_bits"] = frac_bits
    if arith == "fx":
        out["R"], out["E"], out["r"], out["eps"] = res.R_fx, res.E_fx, res.r_fx, res.eps_fx
    else:
        out["R"], out["E"], out["r"], out["eps"] = res.R_f64, res.E_f64, res.r_f64, res.eps_f64
    return out


def add_dir(a, b, mode):
    return lib().orc_add_dir(a, b, mode)


def mul_dir(a, b, mode):
    return lib().orc_mul_dir(a, b, mode)


def div_dir(a, m, mode):
    return lib().orc_div_dir(a, m, mode)


def fx_to_double_rd(a: int, frac_bits: int = DEFAULT_FRAC_BITS) -> float:
    return lib().orc_fx_to_double_rd(int(a), frac_bits)


def splitmix64_at(seed: int, i: int) -> int:
    return int(lib().orc_splitmix64_at(seed, i))


def F_generated(sigma: int, d: int, h: int, seeds, bases, spread: int, xs,
                frac_bits: int = DEFAULT_FRAC_BITS, symmetric: int = 0) -> np.ndarray:
    """F (fx) at the states xs, argument k being bases[k-1] + (SplitMix64(seeds[k-1], c(y)) mod spread).

    c(y) = y (symmetric = 0), min(y, N-1-y) (1), the smallest index of y's
    orbit under complement and string swap (2; sigma = d = 2), or under
    complement and the orders of the three strings (3; sigma = 2, d = 3).
    """
    seeds = np.ascontiguousarray(seeds, dtype=np.uint64)
    bases = np.ascontiguousarray(bases, dtype=np.int64)
    xs = np.ascontiguousarray(xs, dtype=np.uint64)
    out = np.empty(xs.size, dtype=np.int64)
    _check(lib().orc_F_fx_generated(sigma, d, h, frac_bits, _ptr(seeds), _ptr(bases), int(spread),
                                    int(symmetric), _ptr(xs), xs.size, _ptr(out)), "F_fx_generated")
    return out
