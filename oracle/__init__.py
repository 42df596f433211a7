"""CPU oracle for the Hawkes log-likelihood, gradient and location resample.

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package.  It shares no code with
the CUDA library and never imports it.

Functions follow the paper's Sec. 2.1 (eqs. 2-4, the closed-form integral
term), Sec. 2.3.1 (the 1e-40 clip) and Sec. 2.2 (uniform-in-county location
draws of the cut posterior); the C source states each formula.
"""
import ctypes
import os

import numpy as np

from . import build_oracle

_lib = None

_P = ctypes.POINTER
_D = _P(ctypes.c_double)
_I32 = _P(ctypes.c_int32)
_U64 = _P(ctypes.c_uint64)


def lib(path=None):
    """Load (building first if needed) the oracle shared library."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    if _lib is None:
        _lib = _bind(ctypes.CDLL(build_oracle.build()))
    return _lib


def _bind(L):
    for suf in ("f64", "ld"):
        f = getattr(L, "oracle_loglik_grad_" + suf)
        f.argtypes = [ctypes.c_int64, _D, _D, _D, _D, _D, ctypes.c_int64, ctypes.c_int64,
                      _D, _D, ctypes.c_int, ctypes.c_int]
        f.restype = ctypes.c_int
    L.oracle_max_threads_f64.restype = ctypes.c_int
    L.oracle_philox4x64_10.argtypes = [_U64, _U64, _U64]
    L.oracle_philox4x64_10.restype = None
    L.oracle_resample.argtypes = [ctypes.c_int64, _I32, ctypes.c_int32, ctypes.c_int32, _I32, _D,
                                  ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, _D, _D]
    L.oracle_resample.restype = ctypes.c_int
    return L


def _dp(a):
    return a.ctypes.data_as(_D) if a is not None else None


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def loglik_grad(t, x, y, params, s=None, row_begin=0, row_end=None, rows=False,
                threads=0, precision="f64", L=None, bg_time_only=False):
    """Eq. 4 log-likelihood and its gradient, as a plain double loop.

    ``params`` = (mu, tau_x, tau_t, theta, omega, h); ``s`` = per-event source
    bandwidth scale (None: s_j = 1).  Returns ``out7`` = [ell, d/dmu, d/dtau_x,
    d/dtau_t, d/dtheta, d/domega, d/dh]; with ``rows=True`` also the per-row
    array [m, 9] = (ell_i, six partials, log lambda_i, Lambda_i).
    ``precision`` "ld" uses the long-double build.  ``bg_time_only``: the
    time-only background of eq. 2, mu phi1(dt; tau_t) / tau_x^2.
    """
    L = L or lib()
    t, x, y, s = _f64(t), _f64(x), _f64(y), _f64(s)
    n = t.shape[0]
    row_end = n if row_end is None else row_end
    p = np.ascontiguousarray(params, dtype=np.float64)
    out = np.zeros(7)
    r9 = np.zeros((max(row_end - row_begin, 0), 9)) if rows else None
    f = getattr(L, "oracle_loglik_grad_" + precision)
    rc = f(n, _dp(t), _dp(x), _dp(y), _dp(s), _dp(p), row_begin, row_end, _dp(out), _dp(r9),
           int(threads), 1 if bg_time_only else 0)
    if rc != 0:
        raise ValueError("oracle_loglik_grad: bad arguments")
    return (out, r9) if rows else out


def max_threads():
    return int(lib().oracle_max_threads_f64())


def philox4x64_10(ctr, key, L=None):
    """One Philox4x64-10 block: counter (4 x u64), key (2 x u64) -> 4 x u64."""
    L = L or lib()
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    o = np.zeros(4, dtype=np.uint64)
    L.oracle_philox4x64_10(c.ctypes.data_as(_U64), k.ctypes.data_as(_U64), o.ctypes.data_as(_U64))
    return o


def resample(county, n_counties, tri_county, tri_xy, seed, stream, iteration, L=None):
    """Uniform-in-county location draw; returns (x, y) float64 arrays."""
    L = L or lib()
    county = np.ascontiguousarray(county, dtype=np.int32)
    tri_county = np.ascontiguousarray(tri_county, dtype=np.int32)
    tri_xy = np.ascontiguousarray(tri_xy, dtype=np.float64).reshape(-1)
    n = county.shape[0]
    xo, yo = np.zeros(n), np.zeros(n)
    rc = L.oracle_resample(n, county.ctypes.data_as(_I32), int(n_counties), tri_county.shape[0],
                           tri_county.ctypes.data_as(_I32), _dp(tri_xy), int(seed), int(stream),
                           int(iteration), _dp(xo), _dp(yo))
    if rc != 0:
        raise ValueError("oracle_resample: bad arguments")
    return xo, yo
