"""The log-likelihood-only sweep (HAWKES_LOGLIK_ONLY) and the symmetric row
shards (hawkes_shard_moments / hawkes_finalize_moments) through the C ABI,
against the FP64 CPU oracle.

Tolerances as in the parity tests: the log-likelihood within 1e-6 relative,
each gradient component within 1e-5 relative to max(|g_k|, 1e-3 S_k), where
S_k = sum_i |d ell_i / d p_k|; FP64 path 1e-10.
"""
import numpy as np
import pytest

import oracle
from paper_2407_11349_gb300 import synth
from paper_2407_11349_gb300.hawkes import (HAWKES_BG_TIME, HAWKES_F32, HAWKES_F64, HAWKES_LOGLIK_ONLY,
                                           HAWKES_MODEL1, HAWKES_SKIP_SPATIAL, HAWKES_SKIP_UNDERFLOW,
                                           Batch, Hawkes, HawkesError)

pytestmark = pytest.mark.gpu

P0 = synth.DEFAULT_PARAMS
TOL_LL32 = 1e-6
TOL_G32 = 1e-5
TOL_F64 = 1e-10
LL = HAWKES_LOGLIK_ONLY


@pytest.fixture(scope="module")
def hk():
    h = Hawkes(0)
    yield h
    h.close()


def assert_close(got, ref, rows, tol_ll, tol_g, what=""):
    scale = np.abs(rows[:, 1:7]).sum(axis=0)
    e_ll = abs(got[0] - ref[0]) / abs(ref[0])
    denom = np.maximum(np.abs(ref[1:]), 1e-3 * scale)
    e_g = np.abs(got[1:] - ref[1:]) / np.where(denom > 0, denom, 1.0)
    assert e_ll <= tol_ll, f"{what}: loglik rel err {e_ll:.3g}"
    assert np.all(e_g <= tol_g), f"{what}: grad rel errs {e_g}"


# ---------------------------------------------------------------------------
# Log-likelihood only
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n,ties,model1,bgt", [(1, False, False, False), (257, False, False, False),
                                               (2049, False, True, False), (3000, True, False, False),
                                               (5000, False, False, False), (3000, False, False, True)])
def test_loglik_only_matches_oracle(hk, n, ties, model1, bgt):
    ds = synth.grid_dataset(n, 100.0, 20, 20, seed=90 + n)
    if ties:
        ds = synth.integer_day_times(ds)
    hk.set_events(ds.t, ds.county, ds.county_scale, ds.x, ds.y)
    ref = oracle.loglik_grad(ds.t, ds.x, ds.y, P0, s=None if model1 else ds.s, bg_time_only=bgt)
    fl = LL | (HAWKES_MODEL1 if model1 else 0) | (HAWKES_BG_TIME if bgt else 0)
    for prec, tol in ((HAWKES_F32, TOL_LL32), (HAWKES_F64, TOL_F64)):
        ll, g = hk.loglik_grad(P0, prec | fl)
        assert abs(ll - ref[0]) <= tol * abs(ref[0]), (prec, ll, ref[0])
        assert np.all(np.isnan(g)), "the gradient is not evaluated"


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4])
def test_loglik_only_variants_windows_and_skips(hk, variant):
    ds = synth.grid_dataset(6000, 1200.0, 20, 20, seed=95)
    hk.set_events(ds.t, ds.county, ds.county_scale, ds.x, ds.y)
    ref = oracle.loglik_grad(ds.t, ds.x, ds.y, P0, s=ds.s)
    wref = oracle.loglik_grad(ds.t, ds.x, ds.y, P0, s=ds.s, row_begin=1000, row_end=4500)
    hk.set_variant(variant)
    try:
        for fl in (LL, LL | HAWKES_SKIP_UNDERFLOW, LL | HAWKES_SKIP_SPATIAL):
            ll, _ = hk.loglik_grad(P0, fl)
            assert abs(ll - ref[0]) <= TOL_LL32 * abs(ref[0]), (variant, fl)
        ll, _ = hk.loglik_grad(P0, LL, 1000, 4500)
        assert abs(ll - wref[0]) <= TOL_LL32 * abs(wref[0])
    finally:
        hk.set_variant(0)


def test_loglik_only_equals_full_path_at_c2(hk):
    """N = 100,000 after a resample: the two-moment sweep gives the full
    sweep's log-likelihood up to FP32 summation order."""
    ds = synth.config_dataset("c2")
    hk.load(ds)
    hk.resample(1, 0, 4)
    ll_full, _ = hk.loglik_grad(P0, HAWKES_F32)
    ll, g = hk.loglik_grad(P0, LL)
    assert abs(ll - ll_full) <= 1e-7 * abs(ll_full) and np.all(np.isnan(g))


def test_loglik_only_batch(hk):
    torch = pytest.importorskip("torch")
    base = synth.voronoi_dataset(12_000, n_cells=300, seed=97)
    dss = [base] * 3 + synth.regional_subsets(base, [2_000, 5_000], seed=98)
    params = synth.chain_params(len(dss), seed=99)
    hks = [Hawkes(0).load(d) for d in dss]
    try:
        dp = torch.tensor(params, dtype=torch.float64, device="cuda")
        dout = torch.zeros((len(dss), 7), dtype=torch.float64, device="cuda")
        b = Batch(hks, [5] * len(dss), list(range(len(dss))), LL)
        try:
            torch.cuda.synchronize()
            b.run(dp.data_ptr(), 2, dout.data_ptr())
            b.wait()
            got = dout.cpu().numpy()
        finally:
            b.close()
        for p, (h, d) in enumerate(zip(hks, dss)):
            x, y = h.locations()
            ref = oracle.loglik_grad(d.t, x, y, params[p], s=d.s)
            assert abs(got[p, 0] - ref[0]) <= TOL_LL32 * abs(ref[0]), p
            assert np.all(np.isnan(got[p, 1:]))
    finally:
        for h in hks:
            h.close()


# ---------------------------------------------------------------------------
# Symmetric row shards
# ---------------------------------------------------------------------------

def _sharded(h, torch, p, G, flags=HAWKES_F32, order=None):
    """Run G shards one after another on this GPU, add their moment vectors,
    finalise from the sum."""
    n = h.n
    dp = torch.tensor(p, dtype=torch.float64, device="cuda")
    tot = torch.zeros(6 * n, dtype=torch.float64, device="cuda")
    m = torch.empty(6 * n, dtype=torch.float64, device="cuda")
    for g in (order or range(G)):
        h.shard_moments(dp.data_ptr(), g, G, m.data_ptr(), flags)
        torch.cuda.synchronize()
        tot += m
    out = torch.empty(7, dtype=torch.float64, device="cuda")
    h.finalize_moments(dp.data_ptr(), tot.data_ptr(), out.data_ptr(), flags)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("G", [1, 2, 4, 7])
def test_symmetric_shards_match_oracle(hk, G):
    torch = pytest.importorskip("torch")
    ds = synth.grid_dataset(20_000, 300.0, 30, 30, seed=101)
    hk.set_events(ds.t, ds.county, ds.county_scale, ds.x, ds.y)
    ref, rows = oracle.loglik_grad(ds.t, ds.x, ds.y, P0, s=ds.s, rows=True)
    got = _sharded(hk, torch, P0, G, order=list(reversed(range(G))))
    assert_close(got, ref, rows, TOL_LL32, TOL_G32, f"G={G}")


@pytest.mark.parametrize("flags", [HAWKES_MODEL1, HAWKES_BG_TIME, HAWKES_SKIP_UNDERFLOW, LL])
def test_symmetric_shards_with_flags(hk, flags):
    torch = pytest.importorskip("torch")
    ds = synth.integer_day_times(synth.grid_dataset(9_000, 400.0, 20, 20, seed=102))
    hk.set_events(ds.t, ds.county, ds.county_scale, ds.x, ds.y)
    ref, rows = oracle.loglik_grad(ds.t, ds.x, ds.y, P0, s=None if flags & HAWKES_MODEL1 else ds.s, rows=True,
                                   bg_time_only=bool(flags & HAWKES_BG_TIME))
    got = _sharded(hk, torch, P0, 3, flags)
    if flags & LL:
        assert abs(got[0] - ref[0]) <= TOL_LL32 * abs(ref[0]) and np.all(np.isnan(got[1:]))
    else:
        assert_close(got, ref, rows, TOL_LL32, TOL_G32, f"flags={flags}")


def test_symmetric_shards_equal_whole_sweep_at_c2(hk):
    """N = 100,000 after a resample: 4 shards summed equal the one-launch
    sweep up to the order of the FP64 additions; the bounds split the pairs
    evenly."""
    torch = pytest.importorskip("torch")
    from paper_2407_11349_gb300 import shard
    ds = synth.config_dataset("c2")
    hk.load(ds)
    hk.resample(1, 0, 2)
    whole = np.concatenate(hk.loglik_grad(P0, HAWKES_F32), axis=None)
    got = _sharded(hk, torch, P0, 4)
    assert np.all(np.abs(got - whole) <= 1e-9 * np.abs(whole)), (got, whole)
    tr = hk.tile_rows()
    b = shard.symmetric_row_bounds(ds.n, tr, 4)
    pairs = np.array([(e - a) * (a + e - 1) / 2 for a, e in zip(b[:-1], b[1:])])
    # whole row tiles: each shard within one (largest) tile of an equal share
    assert np.all(np.abs(pairs - ds.n * (ds.n - 1) / 8) <= tr * ds.n), pairs


def test_shard_arguments_are_checked(hk):
    torch = pytest.importorskip("torch")
    ds = synth.grid_dataset(3000, 100.0, 20, 20, seed=103)
    hk.set_events(ds.t, ds.county, ds.county_scale, ds.x, ds.y)
    dp = torch.tensor(P0, dtype=torch.float64, device="cuda")
    m = torch.empty(6 * ds.n, dtype=torch.float64, device="cuda")
    for shard_, G, fl in ((2, 2, 0), (-1, 2, 0), (0, 0, 0), (0, 2, HAWKES_F64), (0, 2, HAWKES_SKIP_SPATIAL)):
        with pytest.raises(HawkesError) as e:
            hk.shard_moments(dp.data_ptr(), shard_, G, m.data_ptr(), fl)
        assert e.value.status == -1
    ll, g = hk.loglik_grad(P0, HAWKES_F32)  # still usable
    assert np.isfinite(ll)
