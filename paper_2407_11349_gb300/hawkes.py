"""Python binding of libhawkes (include/hawkes.h): argument marshalling only.

Every computation runs in the CUDA library; there is no CPU fallback.  If the
shared library is missing, importing the binding raises: build it first with
``python -c "import __graft_entry__ as g; g.build()"`` (or
``paper_2407_11349_gb300.build.build()``).

The module-level functions carry the C names (``hawkes_create``,
``hawkes_loglik_grad``, ...) and take the same arguments as host arrays or
device pointers; the ``Hawkes`` class wraps one context for convenience.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# HAWKES_DEBUG=1 in the environment selects the debug build (device index
# checks; built by build.build(debug=True)).
LIB_PATH = os.path.join(_HERE, "lib", "libhawkes_debug.so" if os.environ.get("HAWKES_DEBUG") == "1"
                        else "libhawkes.so")

HAWKES_OK = 0
HAWKES_F32 = 0
HAWKES_F64 = 1
HAWKES_MODEL2 = 0
HAWKES_MODEL1 = 2
HAWKES_SKIP_UNDERFLOW = 4
HAWKES_BG_TIME = 8
HAWKES_SKIP_SPATIAL = 16
HAWKES_LOGLIK_ONLY = 32
KERNEL_CLASSES = ("prep", "sweep", "rows64", "final", "reduce", "resample", "other")


class HawkesError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {strerror(status)} ({status})")


class hawkes_params(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("mu", "tau_x", "tau_t", "theta", "omega", "h")]


class hawkes_profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64 * 8), ("ms", ctypes.c_double * 8)]


_D = ctypes.POINTER(ctypes.c_double)
_I32 = ctypes.POINTER(ctypes.c_int32)
_VP = ctypes.c_void_p
_lib = None

# name -> (restype, argtypes), mirroring include/hawkes.h
_SIGS = {
    "hawkes_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "hawkes_create": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.c_int, _VP]),
    "hawkes_destroy": (None, [_VP]),
    "hawkes_set_events": (ctypes.c_int, [_VP, ctypes.c_int64, _D, _D, _D, _I32, ctypes.c_int32, _D]),
    "hawkes_set_counties": (ctypes.c_int, [_VP, ctypes.c_int32, _I32, _D]),
    "hawkes_resample_locations": (ctypes.c_int, [_VP, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]),
    "hawkes_get_locations": (ctypes.c_int, [_VP, _D, _D]),
    "hawkes_loglik_grad": (ctypes.c_int, [_VP, ctypes.POINTER(hawkes_params), ctypes.c_uint32,
                                          ctypes.c_int64, ctypes.c_int64, _D, _D]),
    "hawkes_loglik_grad_async": (ctypes.c_int, [_VP, _VP, ctypes.c_uint32, _VP]),
    "hawkes_loglik_rows": (ctypes.c_int, [_VP, ctypes.POINTER(hawkes_params), ctypes.c_uint32, _D, _D]),
    "hawkes_profile_enable": (ctypes.c_int, [_VP, ctypes.c_int]),
    "hawkes_profile_read": (ctypes.c_int, [_VP, ctypes.POINTER(hawkes_profile)]),
    "hawkes_num_events": (ctypes.c_int64, [_VP]),
    "hawkes_sweep_variants": (ctypes.c_int, []),
    "hawkes_check_bounded_wait": (ctypes.c_int, [_VP, _D]),
    "hawkes_set_spatial_window": (ctypes.c_int, [_VP, ctypes.c_int64]),
    "hawkes_debug_build": (ctypes.c_int, []),
    "hawkes_debug_set_item": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "hawkes_set_sweep_variant": (ctypes.c_int, [_VP, ctypes.c_int]),
    "hawkes_get_sweep_variant": (ctypes.c_int, [_VP]),
    "hawkes_tune": (ctypes.c_int, [_VP, ctypes.POINTER(hawkes_params), ctypes.c_uint32, ctypes.c_int,
                                   ctypes.POINTER(ctypes.c_int), _D]),
    "hawkes_tune_cached": (ctypes.c_int, [_VP, ctypes.POINTER(hawkes_params), ctypes.c_uint32, ctypes.c_int,
                                          ctypes.c_char_p, ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(ctypes.c_int)]),
    "hawkes_tune_cache_get": (ctypes.c_int, [ctypes.c_char_p, ctypes.c_char_p, ctypes.POINTER(ctypes.c_int),
                                             ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), _D]),
    "hawkes_tune_cache_put": (ctypes.c_int, [ctypes.c_char_p, ctypes.c_char_p, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_int, ctypes.c_double]),
    "hawkes_shard_bounds": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                           ctypes.POINTER(ctypes.c_int64)]),
    "hawkes_shard_tile_rows": (ctypes.c_int64, [_VP]),
    "hawkes_shard_moments": (ctypes.c_int, [_VP, _VP, ctypes.c_uint32, ctypes.c_int, ctypes.c_int, _VP]),
    "hawkes_finalize_moments": (ctypes.c_int, [_VP, _VP, ctypes.c_uint32, _VP, _VP]),
    "hawkes_loglik_grad_noalloc": (ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_int64, _VP,
                                                  ctypes.c_uint32, _VP, _VP]),
    "hawkes_batch_create": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.POINTER(_VP), ctypes.c_int32,
                                           ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                                           ctypes.c_uint32, _VP]),
    "hawkes_batch_destroy": (None, [_VP]),
    "hawkes_batch_run": (ctypes.c_int, [_VP, _VP, ctypes.c_uint64, _VP]),
    "hawkes_batch_capture": (ctypes.c_int, [_VP, _VP, _VP]),
    "hawkes_batch_wait": (ctypes.c_int, [_VP]),
    "hawkes_batch_tune": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), _D]),
    "hawkes_batch_set_config": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "hawkes_batch_set_chains_per_cta": (ctypes.c_int, [_VP, ctypes.c_int]),
    "hawkes_batch_get_config": (ctypes.c_int, [_VP] + [ctypes.POINTER(ctypes.c_int)] * 5),
    "hawkes_batch_tune_cached": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, ctypes.c_char_p,
                                                ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                                ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "hawkes_mlp_create": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.c_int, _VP, ctypes.c_uint64]),
    "hawkes_mlp_destroy": (None, [_VP]),
    "hawkes_mlp_get_params": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_float)]),
    "hawkes_mlp_set_params": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_float)]),
    "hawkes_mlp_set_data": (ctypes.c_int, [_VP, ctypes.c_int64, _D, _D, _D]),
    "hawkes_mlp_train": (ctypes.c_int, [_VP, ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_uint64, _D]),
    "hawkes_mlp_loss_grad": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_float),
                                            ctypes.POINTER(ctypes.c_float), _D, ctypes.POINTER(ctypes.c_float),
                                            ctypes.POINTER(ctypes.c_float)]),
    "hawkes_mlp_predict": (ctypes.c_int, [_VP, ctypes.c_int64, _VP, _VP, _VP]),
    "hawkes_mlp_stats": (ctypes.c_int, [_VP, _D]),
    "hawkes_mlp_wait": (ctypes.c_int, [_VP]),
}


def lib():
    """The loaded libhawkes (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{os.path.basename(LIB_PATH)} not built ({LIB_PATH}); run the package build first")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def strerror(status):
    return lib().hawkes_strerror(int(status)).decode()


def _check(rc, where):
    if rc != HAWKES_OK:
        raise HawkesError(rc, where)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _dp(a):
    return None if a is None else a.ctypes.data_as(_D)


def as_params(p):
    if isinstance(p, hawkes_params):
        return p
    p = [float(v) for v in p]
    return hawkes_params(*p)


# --- C-named thin wrappers -------------------------------------------------

def hawkes_create(device=0, stream=0):
    h = _VP()
    _check(lib().hawkes_create(ctypes.byref(h), int(device), _VP(int(stream) or None)), "hawkes_create")
    return h


def hawkes_destroy(ctx):
    lib().hawkes_destroy(ctx)


def hawkes_set_events(ctx, t, x, y, county, county_scale):
    t, x, y, cs = _f64(t), _f64(x), _f64(y), _f64(county_scale)
    county = np.ascontiguousarray(county, dtype=np.int32)
    _check(lib().hawkes_set_events(ctx, t.shape[0], _dp(t), _dp(x), _dp(y), county.ctypes.data_as(_I32),
                                   cs.shape[0], _dp(cs)), "hawkes_set_events")


def hawkes_set_counties(ctx, tri_county, tri_xy):
    tc = np.ascontiguousarray(tri_county, dtype=np.int32)
    txy = np.ascontiguousarray(tri_xy, dtype=np.float64).reshape(-1)
    _check(lib().hawkes_set_counties(ctx, tc.shape[0], tc.ctypes.data_as(_I32), _dp(txy)),
           "hawkes_set_counties")


def hawkes_resample_locations(ctx, seed, stream, iteration):
    _check(lib().hawkes_resample_locations(ctx, int(seed), int(stream), int(iteration)),
           "hawkes_resample_locations")


def hawkes_get_locations(ctx):
    n = lib().hawkes_num_events(ctx)
    x, y = np.empty(n), np.empty(n)
    _check(lib().hawkes_get_locations(ctx, _dp(x), _dp(y)), "hawkes_get_locations")
    return x, y


def hawkes_loglik_grad(ctx, params, flags=HAWKES_F32, row_begin=0, row_end=None):
    n = lib().hawkes_num_events(ctx)
    row_end = n if row_end is None else row_end
    ll = ctypes.c_double()
    g = np.zeros(6)
    p = as_params(params)
    _check(lib().hawkes_loglik_grad(ctx, ctypes.byref(p), int(flags), int(row_begin), int(row_end),
                                    ctypes.byref(ll), _dp(g)), "hawkes_loglik_grad")
    return ll.value, g


def hawkes_loglik_grad_async(ctx, d_params, flags, d_out):
    """d_params, d_out: device addresses (e.g. torch ``tensor.data_ptr()``)."""
    _check(lib().hawkes_loglik_grad_async(ctx, _VP(int(d_params)), int(flags), _VP(int(d_out))),
           "hawkes_loglik_grad_async")


def hawkes_loglik_rows(ctx, params, flags=HAWKES_F32):
    n = lib().hawkes_num_events(ctx)
    out = np.zeros(7)
    rows = np.zeros((n, 9))
    p = as_params(params)
    _check(lib().hawkes_loglik_rows(ctx, ctypes.byref(p), int(flags), _dp(out), _dp(rows)),
           "hawkes_loglik_rows")
    return out, rows


def hawkes_profile_enable(ctx, on):
    _check(lib().hawkes_profile_enable(ctx, 1 if on else 0), "hawkes_profile_enable")


def hawkes_profile_read(ctx):
    pr = hawkes_profile()
    _check(lib().hawkes_profile_read(ctx, ctypes.byref(pr)), "hawkes_profile_read")
    return {k: (int(pr.launches[i]), float(pr.ms[i])) for i, k in enumerate(KERNEL_CLASSES)}


def hawkes_num_events(ctx):
    return int(lib().hawkes_num_events(ctx))


def hawkes_sweep_variants():
    return int(lib().hawkes_sweep_variants())


def hawkes_set_sweep_variant(ctx, variant):
    _check(lib().hawkes_set_sweep_variant(ctx, int(variant)), "hawkes_set_sweep_variant")


def hawkes_get_sweep_variant(ctx):
    return int(lib().hawkes_get_sweep_variant(ctx))


def hawkes_tune(ctx, params, flags=HAWKES_F32, reps=2):
    """Time every sweep variant on the current events; keep the fastest.
    Returns (chosen index, mean sweep ms per variant)."""
    nv = hawkes_sweep_variants()
    ms = np.zeros(nv)
    ch = ctypes.c_int(-1)
    p = as_params(params)
    _check(lib().hawkes_tune(ctx, ctypes.byref(p), int(flags), int(reps), ctypes.byref(ch), _dp(ms)),
           "hawkes_tune")
    return ch.value, ms


def hawkes_tune_cached(ctx, params, cache_path, flags=HAWKES_F32, reps=2):
    """Autotune through the JSON cache at ``cache_path`` (see include/hawkes.h).
    Returns (chosen variant, True if it came from the cache)."""
    ch, hit = ctypes.c_int(-1), ctypes.c_int(0)
    p = as_params(params)
    _check(lib().hawkes_tune_cached(ctx, ctypes.byref(p), int(flags), int(reps), os.fsencode(cache_path),
                                    ctypes.byref(ch), ctypes.byref(hit)), "hawkes_tune_cached")
    return ch.value, bool(hit.value)


def hawkes_tune_cache_get(cache_path, key):
    """(variant, chunk, order, ms) stored under ``key``, or None (host only)."""
    v, c, o, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    rc = lib().hawkes_tune_cache_get(os.fsencode(cache_path), key.encode(), ctypes.byref(v), ctypes.byref(c),
                                     ctypes.byref(o), ctypes.byref(ms))
    if rc < 0:
        _check(rc, "hawkes_tune_cache_get")
    return (v.value, c.value, o.value, ms.value) if rc == 1 else None


def hawkes_tune_cache_put(cache_path, key, variant, chunk, order, ms):
    """Insert or replace ``key`` in the cache file (host only)."""
    _check(lib().hawkes_tune_cache_put(os.fsencode(cache_path), key.encode(), int(variant), int(chunk),
                                       int(order), float(ms)), "hawkes_tune_cache_put")


def hawkes_debug_build():
    """1 if the loaded library is the HAWKES_DEBUG build."""
    return int(lib().hawkes_debug_build())


def hawkes_debug_set_item(ctx, k, row_tile, col_begin, col_end):
    """Debug build only: overwrite work item k (a test hook for the checks)."""
    _check(lib().hawkes_debug_set_item(ctx, int(k), int(row_tile), int(col_begin), int(col_end)),
           "hawkes_debug_set_item")


def hawkes_shard_bounds(n, tile_rows, nshards):
    """Row boundaries [nshards + 1] of the symmetric sweep's split into shards
    of about equal pair counts (host only; no device needed)."""
    b = (ctypes.c_int64 * (int(nshards) + 1))()
    _check(lib().hawkes_shard_bounds(int(n), int(tile_rows), int(nshards), b), "hawkes_shard_bounds")
    return np.array(list(b), dtype=np.int64)


def hawkes_shard_tile_rows(ctx):
    r = int(lib().hawkes_shard_tile_rows(ctx))
    _check(min(r, 0), "hawkes_shard_tile_rows")
    return r


def hawkes_shard_moments(ctx, d_params, flags, shard, nshards, d_moments):
    _check(lib().hawkes_shard_moments(ctx, _VP(int(d_params)), int(flags), int(shard), int(nshards),
                                      _VP(int(d_moments))), "hawkes_shard_moments")


def hawkes_finalize_moments(ctx, d_params, flags, d_moments, d_out):
    _check(lib().hawkes_finalize_moments(ctx, _VP(int(d_params)), int(flags), _VP(int(d_moments)),
                                         _VP(int(d_out))), "hawkes_finalize_moments")


HAWKES_NOALLOC_MAX_N = 65536


def hawkes_loglik_grad_noalloc(d_t, d_x, d_y, d_s, n, d_params, flags, d_out, stream=0):
    """Allocation-free evaluation for callers that cannot allocate device memory
    (see include/hawkes.h).  All pointers are device addresses of the caller's
    buffers (``d_s`` may be 0 for s_j = 1); queued on ``stream``, no wait."""
    _check(lib().hawkes_loglik_grad_noalloc(_VP(int(d_t)), _VP(int(d_x)), _VP(int(d_y)),
                                            _VP(int(d_s) or None), int(n), _VP(int(d_params)),
                                            int(flags), _VP(int(d_out)), _VP(int(stream) or None)),
           "hawkes_loglik_grad_noalloc")


def hawkes_batch_create(ctxs, seeds=None, streams=None, flags=HAWKES_F32, stream=0):
    P = len(ctxs)
    arr = (_VP * P)(*[c.value if isinstance(c, _VP) else c for c in ctxs])
    sd = st = None
    if seeds is not None:
        sd = (ctypes.c_uint64 * P)(*[int(v) for v in seeds])
        st = (ctypes.c_uint64 * P)(*[int(v) for v in streams])
    h = _VP()
    _check(lib().hawkes_batch_create(ctypes.byref(h), arr, P, sd, st, int(flags), _VP(int(stream) or None)),
           "hawkes_batch_create")
    return h


def hawkes_batch_destroy(b):
    lib().hawkes_batch_destroy(b)


def hawkes_batch_run(b, d_params, iteration, d_out):
    _check(lib().hawkes_batch_run(b, _VP(int(d_params)), int(iteration), _VP(int(d_out))), "hawkes_batch_run")


def hawkes_batch_capture(b, d_params, d_out):
    _check(lib().hawkes_batch_capture(b, _VP(int(d_params)), _VP(int(d_out))), "hawkes_batch_capture")


def hawkes_batch_wait(b):
    _check(lib().hawkes_batch_wait(b), "hawkes_batch_wait")


def hawkes_batch_tune(b, d_params, d_out, reps=1):
    """Returns (variant, chunk tiles, item order, mean sweep ms) of the fastest configuration."""
    v, c, o, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    _check(lib().hawkes_batch_tune(b, _VP(int(d_params)), _VP(int(d_out)), int(reps), ctypes.byref(v),
                                   ctypes.byref(c), ctypes.byref(o), ctypes.byref(ms)), "hawkes_batch_tune")
    return v.value, c.value, o.value, ms.value


def hawkes_batch_tune_cached(b, d_params, d_out, cache_path, reps=1):
    """Batch autotune through the JSON cache.  Returns (variant, chunk tiles,
    item order, True if it came from the cache)."""
    v, c, o, hit = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().hawkes_batch_tune_cached(b, _VP(int(d_params)), _VP(int(d_out)), int(reps),
                                          os.fsencode(cache_path), ctypes.byref(v), ctypes.byref(c),
                                          ctypes.byref(o), ctypes.byref(hit)), "hawkes_batch_tune_cached")
    return v.value, c.value, o.value, bool(hit.value)


def hawkes_batch_set_config(b, variant, chunk, order=1):
    _check(lib().hawkes_batch_set_config(b, int(variant), int(chunk), int(order)), "hawkes_batch_set_config")


def hawkes_batch_set_chains_per_cta(b, chains_per_cta):
    _check(lib().hawkes_batch_set_chains_per_cta(b, int(chains_per_cta)), "hawkes_batch_set_chains_per_cta")


def hawkes_batch_get_config(b):
    """(variant, chunk, order, chains_per_cta, n_groups) of the batch."""
    v = [ctypes.c_int() for _ in range(5)]
    _check(lib().hawkes_batch_get_config(b, *[ctypes.byref(x) for x in v]), "hawkes_batch_get_config")
    return tuple(x.value for x in v)


class Batch:
    """Many contexts evaluated in one persistent sweep launch (optionally a CUDA graph)."""

    def __init__(self, hawkes_list, seeds=None, streams=None, flags=HAWKES_F32, stream=0):
        self.members = list(hawkes_list)  # keep the contexts alive
        self.b = hawkes_batch_create([h.ctx for h in self.members], seeds, streams, flags, stream)

    def close(self):
        if self.b:
            hawkes_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, d_params, iteration, d_out):
        hawkes_batch_run(self.b, d_params, iteration, d_out)

    def capture(self, d_params, d_out):
        hawkes_batch_capture(self.b, d_params, d_out)

    def wait(self):
        hawkes_batch_wait(self.b)

    def tune(self, d_params, d_out, reps=1):
        return hawkes_batch_tune(self.b, d_params, d_out, reps)

    def set_config(self, variant, chunk, order=1):
        hawkes_batch_set_config(self.b, variant, chunk, order)

    def set_chains_per_cta(self, k):
        hawkes_batch_set_chains_per_cta(self.b, k)

    def config(self):
        """(variant, chunk, order, chains_per_cta, n_groups)."""
        return hawkes_batch_get_config(self.b)

    def tune_cached(self, d_params, d_out, cache_path, reps=1):
        return hawkes_batch_tune_cached(self.b, d_params, d_out, cache_path, reps)


HAWKES_MLP_NPARAMS = 69639
_F = ctypes.POINTER(ctypes.c_float)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


class MLP:
    """The surrogate network (include/hawkes.h, hawkes_mlp_*)."""

    def __init__(self, device=0, stream=0, seed=0):
        h = _VP()
        _check(lib().hawkes_mlp_create(ctypes.byref(h), int(device), _VP(int(stream) or None), int(seed)),
               "hawkes_mlp_create")
        self.m = h

    def close(self):
        if self.m:
            lib().hawkes_mlp_destroy(self.m)
            self.m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self):
        p = np.zeros(HAWKES_MLP_NPARAMS, dtype=np.float32)
        _check(lib().hawkes_mlp_get_params(self.m, p.ctypes.data_as(_F)), "hawkes_mlp_get_params")
        return p

    def set_params(self, p):
        p = _f32(p)
        _check(lib().hawkes_mlp_set_params(self.m, p.ctypes.data_as(_F)), "hawkes_mlp_set_params")

    def set_data(self, X, Y, F=None):
        """Training set: X[n x 6] log-parameters, Y[n x 7] targets, F[n] the
        optional seventh-input feature (None: the constant 1)."""
        X = _f64(X).reshape(-1, 6)
        Y = _f64(Y).reshape(-1, 7)
        F = None if F is None else _f64(F).reshape(-1)
        _check(lib().hawkes_mlp_set_data(self.m, X.shape[0], _dp(X), _dp(F), _dp(Y)), "hawkes_mlp_set_data")

    def train(self, steps, batch=512, lr=1e-3, seed=0):
        loss = ctypes.c_double()
        _check(lib().hawkes_mlp_train(self.m, int(steps), int(batch), float(lr), int(seed), ctypes.byref(loss)),
               "hawkes_mlp_train")
        return loss.value

    def loss_grad(self, Xs, Ts):
        Xs, Ts = _f32(Xs).reshape(-1, 7), _f32(Ts).reshape(-1, 7)
        B = Xs.shape[0]
        g = np.zeros(HAWKES_MLP_NPARAMS, dtype=np.float32)
        Y = np.zeros((B, 7), dtype=np.float32)
        loss = ctypes.c_double()
        _check(lib().hawkes_mlp_loss_grad(self.m, B, Xs.ctypes.data_as(_F), Ts.ctypes.data_as(_F),
                                          ctypes.byref(loss), g.ctypes.data_as(_F), Y.ctypes.data_as(_F)),
               "hawkes_mlp_loss_grad")
        return loss.value, g, Y

    def predict(self, d_logp, count, d_out, d_feature=0):
        """Device pointers: d_logp[count x 6] (and d_feature[count] when the
        network was trained with a feature) -> d_out[count x 7] (queued)."""
        _check(lib().hawkes_mlp_predict(self.m, int(count), _VP(int(d_logp)), _VP(int(d_feature) or None),
                                        _VP(int(d_out))), "hawkes_mlp_predict")

    def stats(self):
        s = np.zeros(28)
        _check(lib().hawkes_mlp_stats(self.m, _dp(s)), "hawkes_mlp_stats")
        return s

    def wait(self):
        _check(lib().hawkes_mlp_wait(self.m), "hawkes_mlp_wait")


# --- convenience wrapper ---------------------------------------------------

class Hawkes:
    """One libhawkes context on one GPU."""

    def __init__(self, device=0, stream=0):
        self.ctx = hawkes_create(device, stream)

    def close(self):
        if self.ctx:
            hawkes_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_events(self, t, county, county_scale, x=None, y=None):
        hawkes_set_events(self.ctx, t, x, y, county, county_scale)

    def set_counties(self, tri_county, tri_xy):
        hawkes_set_counties(self.ctx, tri_county, tri_xy)

    def load(self, ds, counties=True):
        """Events and county triangles of a ``synth.Dataset``."""
        self.set_events(ds.t, ds.county, ds.county_scale, ds.x, ds.y)
        if counties:
            self.set_counties(ds.counties.tri_county, ds.counties.tri_xy)
        return self

    def resample(self, seed, stream, iteration):
        hawkes_resample_locations(self.ctx, seed, stream, iteration)

    def locations(self):
        return hawkes_get_locations(self.ctx)

    def loglik_grad(self, params, flags=HAWKES_F32, row_begin=0, row_end=None):
        return hawkes_loglik_grad(self.ctx, params, flags, row_begin, row_end)

    def loglik_grad_async(self, d_params, d_out, flags=HAWKES_F32):
        hawkes_loglik_grad_async(self.ctx, d_params, flags, d_out)

    def loglik_rows(self, params, flags=HAWKES_F32):
        return hawkes_loglik_rows(self.ctx, params, flags)

    def profile(self, on=None):
        if on is not None:
            hawkes_profile_enable(self.ctx, on)
        return hawkes_profile_read(self.ctx)

    def check_bounded_wait(self):
        """Seconds the device-side bounded wait took to give up (raises if it did not)."""
        sec = ctypes.c_double()
        _check(lib().hawkes_check_bounded_wait(self.ctx, ctypes.byref(sec)), "hawkes_check_bounded_wait")
        return sec.value

    def tune(self, params, flags=HAWKES_F32, reps=2):
        return hawkes_tune(self.ctx, params, flags, reps)

    def tune_cached(self, params, cache_path, flags=HAWKES_F32, reps=2):
        return hawkes_tune_cached(self.ctx, params, cache_path, flags, reps)

    def set_spatial_window(self, events):
        """Events per time window of the HAWKES_SKIP_SPATIAL order."""
        _check(lib().hawkes_set_spatial_window(self.ctx, int(events)), "hawkes_set_spatial_window")

    def set_variant(self, v):
        hawkes_set_sweep_variant(self.ctx, v)

    def tile_rows(self):
        """Rows per row tile of the current sweep variant (the shard granularity)."""
        return hawkes_shard_tile_rows(self.ctx)

    def shard_moments(self, d_params, shard, nshards, d_moments, flags=HAWKES_F32):
        """Queue shard `shard` of `nshards` of the symmetric sweep; its six
        moment vectors (6 x n doubles) go to device memory d_moments."""
        hawkes_shard_moments(self.ctx, d_params, flags, shard, nshards, d_moments)

    def finalize_moments(self, d_params, d_moments, d_out, flags=HAWKES_F32):
        """Queue the finalisation of moment vectors summed over all shards:
        ell and the six partials to device memory d_out[7]."""
        hawkes_finalize_moments(self.ctx, d_params, flags, d_moments, d_out)

    @property
    def variant(self):
        return hawkes_get_sweep_variant(self.ctx)

    @property
    def n(self):
        return hawkes_num_events(self.ctx)
