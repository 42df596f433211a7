"""The allocation-free entry point (hawkes_loglik_grad_noalloc) against the
regular one.

It exists for callers that cannot allocate device memory (code inside a
device allocator or memory-pool callback, applications that pre-reserve all
device memory): it takes the caller's device buffers and works in a fixed
scratch array built into the library.  Here the test plays such a caller: it
owns the input and output buffers, calls the entry point several times in a
row through the C ABI (different sizes and models, so each call sees the
previous call's leftovers in the shared scratch, up to the largest size the
scratch holds), and compares each result with hawkes_loglik_grad on the
same events and, at the largest size, with the FP64 CPU oracle, within the
FP32-path tolerances of the parity tests: 1e-6 relative on the
log-likelihood, 1e-5 on each gradient component relative to
max(|g_k|, 1e-3 sum_i |d ell_i / d p_k|).  It also checks what the entry
point is for: a repeated call changes neither PyTorch's allocated bytes nor
the device's free memory; and that bad input made on the host (unsorted
times, a negative bandwidth) comes back as seven NaN outputs.

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
        (synth.grid_dataset(HAWKES_NOALLOC_MAX_N, 600.0, 40, 40, seed=24), HAWKES_F32),
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
            if ds.n == HAWKES_NOALLOC_MAX_N:  # the largest size: also against the oracle
                import oracle
                oref, orows = oracle.loglik_grad(ds.t, ds.x, ds.y, P0, s=ds.s, rows=True)
                _close(got, oref, orows)
    finally:
        hk.close()


def test_noalloc_repeated_call_allocates_nothing():
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    ds = synth.grid_dataset(8_000, 100.0, 20, 20, seed=25)
    t, x, y, s = (torch.tensor(a, dtype=torch.float64, device=dev) for a in (ds.t, ds.x, ds.y, ds.s))
    p = torch.tensor(P0, dtype=torch.float64, device=dev)
    out = torch.empty(7, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream

    def call():
        hawkes_loglik_grad_noalloc(t.data_ptr(), x.data_ptr(), y.data_ptr(), s.data_ptr(), ds.n,
                                   p.data_ptr(), HAWKES_F32, out.data_ptr(), stream)
        torch.cuda.synchronize(dev)
        return out.cpu().numpy().copy()

    first = call()  # may set the device up and load the kernels
    alloc0, free0 = torch.cuda.memory_allocated(dev), torch.cuda.mem_get_info(dev)[0]
    second = call()
    alloc1, free1 = torch.cuda.memory_allocated(dev), torch.cuda.mem_get_info(dev)[0]
    assert alloc1 == alloc0 and free1 == free0, (alloc0, alloc1, free0, free1)
    # the same result up to the order of the FP32 atomics
    assert np.all(np.isfinite(second)) and np.allclose(first, second, rtol=1e-6, atol=0)


@pytest.mark.parametrize("bad", ["unsorted", "tau_x"])
def test_noalloc_bad_input_gives_nan(bad):
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    ds = synth.grid_dataset(2_000, 100.0, 20, 20, seed=26)
    tt = ds.t.copy()
    pp = np.array(P0, dtype=np.float64)
    if bad == "unsorted":
        tt[[10, 11]] = tt[[11, 10]] + np.array([0.0, 1e-3])  # t[10] > t[11]
        assert tt[10] > tt[11]
    else:
        pp[1] = -1.0
    t, x, y, s = (torch.tensor(a, dtype=torch.float64, device=dev) for a in (tt, ds.x, ds.y, ds.s))
    p = torch.tensor(pp, dtype=torch.float64, device=dev)
    out = torch.zeros(7, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    hawkes_loglik_grad_noalloc(t.data_ptr(), x.data_ptr(), y.data_ptr(), s.data_ptr(), ds.n,
                               p.data_ptr(), HAWKES_F32, out.data_ptr(), stream)
    torch.cuda.synchronize(dev)
    assert np.all(np.isnan(out.cpu().numpy()))
    # the next good call is clean: every call clears the error flag
    p.copy_(torch.tensor(P0, dtype=torch.float64))
    t.copy_(torch.tensor(ds.t, dtype=torch.float64))
    hawkes_loglik_grad_noalloc(t.data_ptr(), x.data_ptr(), y.data_ptr(), s.data_ptr(), ds.n,
                               p.data_ptr(), HAWKES_F32, out.data_ptr(), stream)
    torch.cuda.synchronize(dev)
    assert np.all(np.isfinite(out.cpu().numpy()))


def test_noalloc_rejects_sizes_above_its_limit():
    torch = pytest.importorskip("torch")
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(HawkesError) as e:
        hawkes_loglik_grad_noalloc(buf.data_ptr(), buf.data_ptr(), buf.data_ptr(), 0,
                                   HAWKES_NOALLOC_MAX_N + 1, buf.data_ptr(), HAWKES_F32,
                                   buf.data_ptr(), 0)
    assert e.value.status == -8
