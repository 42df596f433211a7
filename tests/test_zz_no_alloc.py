"""The allocation-free entry point (hawkes_loglik_grad_noalloc) against the
regular one.

It exists for callers that cannot allocate device memory (code inside a
device allocator or memory-pool callback, applications that pre-reserve all
device memory): it takes the caller's device buffers and works in a fixed
scratch array built into the library.  Here the test plays such a caller: it
owns the input and output buffers, calls the entry point twice in a row
through the C ABI (different sizes and models, so the second call sees the
first call's leftovers in the shared scratch), and compares each result with
hawkes_loglik_grad on the same events, within the FP32-path tolerances of
the parity tests: 1e-6 relative on the log-likelihood, 1e-5 on each gradient
component relative to max(|g_k|, 1e-3 sum_i |d ell_i / d p_k|).

The file name sorts last so that a run stopping at the first failure has run
every other test before this one.
"""
import numpy as np
import pytest

from paper_2407_11349_gb300 import synth
from paper_2407_11349_gb300.hawkes import (HAWKES_BG_TIME, HAWKES_F32, HAWKES_MODEL1,
                                           HAWKES_NOALLOC_MAX_N, Hawkes, HawkesError,
                                           hawkes_loglik_grad_noalloc)

pytestmark = pytest.mark.gpu

P0 = synth.DEFAULT_PARAMS
TOL_LL32 = 1e-6
TOL_G32 = 1e-5


def _close(got, ref, rows):
    scale = np.abs(rows[:, 1:7]).sum(axis=0)
    e_ll = abs(got[0] - ref[0]) / abs(ref[0])
    denom = np.maximum(np.abs(ref[1:]), 1e-3 * scale)
    e_g = np.abs(got[1:] - ref[1:]) / np.where(denom > 0, denom, 1.0)
    assert e_ll <= TOL_LL32, f"loglik rel err {e_ll:.3g}"
    assert np.all(e_g <= TOL_G32), f"grad rel errs {e_g}"


def test_noalloc_matches_regular_entry_point_on_two_calls():
    torch = pytest.importorskip("torch")
    cases = [
        (synth.grid_dataset(40_000, 400.0, 40, 40, seed=21), HAWKES_F32),
        (synth.grid_dataset(5_000, 100.0, 20, 20, seed=22), HAWKES_F32 | HAWKES_MODEL1),
        (synth.grid_dataset(3_000, 100.0, 20, 20, seed=23), HAWKES_F32 | HAWKES_BG_TIME),
    ]
    hk = Hawkes(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev).cuda_stream
    try:
        for ds, flags in cases:
            model1 = bool(flags & HAWKES_MODEL1)
            t = torch.tensor(ds.t, dtype=torch.float64, device=dev)
            x = torch.tensor(ds.x, dtype=torch.float64, device=dev)
            y = torch.tensor(ds.y, dtype=torch.float64, device=dev)
            s = None if model1 else torch.tensor(ds.s, dtype=torch.float64, device=dev)
            p = torch.tensor(P0, dtype=torch.float64, device=dev)
            out = torch.full((7,), float("nan"), dtype=torch.float64, device=dev)
            torch.cuda.synchronize(dev)
            hawkes_loglik_grad_noalloc(t.data_ptr(), x.data_ptr(), y.data_ptr(),
                                       0 if s is None else s.data_ptr(), ds.n, p.data_ptr(),
                                       flags, out.data_ptr(), stream)
            torch.cuda.synchronize(dev)
            got = out.cpu().numpy()
            assert np.all(np.isfinite(got))

            hk.set_events(ds.t, ds.county, ds.county_scale, ds.x, ds.y)
            ref, rows = hk.loglik_rows(P0, flags)
            _close(got, ref, rows)
    finally:
        hk.close()


def test_noalloc_rejects_sizes_above_its_limit():
    torch = pytest.importorskip("torch")
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(HawkesError) as e:
        hawkes_loglik_grad_noalloc(buf.data_ptr(), buf.data_ptr(), buf.data_ptr(), 0,
                                   HAWKES_NOALLOC_MAX_N + 1, buf.data_ptr(), HAWKES_F32,
                                   buf.data_ptr(), 0)
    assert e.value.status == -8
