"""libhawkes (CUDA, called through the C ABI) against the FP64 CPU oracle.

Tolerances (stated once, used everywhere below):
  FP64 GPU path: every output within 1e-10 relative of the oracle.
  FP32 GPU path: the log-likelihood within 1e-6 relative; each gradient
    component within 1e-5 relative, measured against max(|g_k|, 1e-3 S_k)
    where S_k = sum_i |d ell_i / d p_k| (the scale of the component's terms,
    so that a component that happens to cancel to near zero is judged on the
    size of what cancelled).
  Per-row values (FP32): log lambda_i within 2e-6 absolute (a relative rate
    error); Lambda_i within 1e-12 relative (computed in FP64 on both sides).
  Resample: bit-identical coordinates.
"""
import numpy as np
import pytest

import oracle
from paper_2407_11349_gb300 import synth
from paper_2407_11349_gb300.hawkes import (HAWKES_BG_TIME, HAWKES_F32, HAWKES_F64, HAWKES_MODEL1,
                                           HAWKES_SKIP_UNDERFLOW, Hawkes, HawkesError)

pytestmark = pytest.mark.gpu

P0 = synth.DEFAULT_PARAMS
TOL_F64 = 1e-10
TOL_LL32 = 1e-6
TOL_G32 = 1e-5


@pytest.fixture(scope="module")
def hk():
    h = Hawkes(0)
    yield h
    h.close()


def small_grid(n, seed=0, T=100.0):
    return synth.grid_dataset(n, T, 20, 20, seed=seed)


def oracle_rows(ds, p=P0, model1=False, bg_time=False, row_begin=0, row_end=None):
    s = None if model1 else ds.s
    return oracle.loglik_grad(ds.t, ds.x, ds.y, p, s=s, rows=True, bg_time_only=bg_time,
                              row_begin=row_begin, row_end=row_end)


def assert_close(got_ll, got_g, ref, ref_rows, tol_ll, tol_g, what=""):
    scale = np.abs(ref_rows[:, 1:7]).sum(axis=0)
    e_ll = abs(got_ll - ref[0]) / max(abs(ref[0]), 1e-300)
    denom = np.maximum(np.abs(ref[1:]), 1e-3 * scale)
    denom = np.where(denom > 0, denom, 1.0)
    e_g = np.abs(got_g - ref[1:]) / denom
    assert e_ll <= tol_ll, f"{what} loglik rel err {e_ll:.3g} > {tol_ll}"
    assert np.all(e_g <= tol_g), f"{what} grad rel errs {e_g} > {tol_g}"
    return e_ll, e_g


def check_both(hk, ds, p=P0, model1=False, what=""):
    hk.set_events(ds.t, ds.county, ds.county_scale, ds.x, ds.y)
    ref, rows = oracle_rows(ds, p, model1)
    fl = HAWKES_MODEL1 if model1 else 0
    ll64, g64 = hk.loglik_grad(p, HAWKES_F64 | fl)
    assert_close(ll64, g64, ref, rows, TOL_F64, TOL_F64, what + " f64")
    ll32, g32 = hk.loglik_grad(p, HAWKES_F32 | fl)
    return assert_close(ll32, g32, ref, rows, TOL_LL32, TOL_G32, what + " f32")


@pytest.mark.parametrize("n", [1, 2, 3, 31, 255, 256, 257, 1023, 1024, 1025, 2049, 5000])
def test_sizes_and_ragged_tails(hk, n):
    check_both(hk, small_grid(n, seed=n), what=f"n={n}")


def test_workload_c1(hk):
    """N=2,000, 20x20 grid, seed 0: the small configuration, both paths."""
    ds = synth.config_dataset("c1")
    check_both(hk, ds, what="c1")
    out, rows = hk.loglik_rows(P0, HAWKES_F32)
    ref, rrows = oracle_rows(ds)
    assert np.max(np.abs(rows[:, 7] - rrows[:, 7])) < 2e-6
    assert np.max(np.abs(rows[:, 8] - rrows[:, 8]) / np.abs(rrows[:, 8])) < 1e-12


def test_ties_integer_days(hk):
    ds = synth.integer_day_times(small_grid(3000, seed=5))
    assert np.sum(np.diff(ds.t) == 0) > 2500
    check_both(hk, ds, what="ties")


def test_model1_flag(hk):
    check_both(hk, small_grid(1500, seed=6), model1=True, what="model1")


@pytest.mark.parametrize("p", [(0.5, 20.0, 7.0, 0.0, 0.2, 2.0), (0.0, 20.0, 7.0, 0.3, 0.2, 2.0),
                               (2.0, 5.0, 2.0, 0.9, 1.5, 0.7)])
def test_degenerate_and_other_parameters(hk, p):
    check_both(hk, small_grid(1800, seed=7), p=p, what=f"p={p}")


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4])
def test_sweep_variants_agree(hk, variant):
    ds = small_grid(6000, seed=12)
    hk.set_events(ds.t, ds.county, ds.county_scale, ds.x, ds.y)
    ref, rows = oracle_rows(ds)
    hk.set_variant(variant)
    try:
        ll, g = hk.loglik_grad(P0, HAWKES_F32)
        assert_close(ll, g, ref, rows, TOL_LL32, TOL_G32, f"variant {variant}")
        ll, g = hk.loglik_grad(P0, HAWKES_F32, 1000, 4500)
        wref = oracle.loglik_grad(ds.t, ds.x, ds.y, P0, s=ds.s, row_begin=1000, row_end=4500)
        assert_close(ll, g, wref, rows[1000:4500], TOL_LL32, TOL_G32, f"variant {variant} window")
    finally:
        hk.set_variant(0)


def test_tune_picks_a_variant(hk):
    ds = small_grid(20000, seed=13)
    hk.set_events(ds.t, ds.county, ds.county_scale, ds.x, ds.y)
    chosen, ms = hk.tune(P0, reps=1)
    assert 0 <= chosen < len(ms) and np.all(ms > 0) and ms[chosen] == ms.min()
    hk.set_variant(0)


def test_row_windows_sum_to_whole(hk):
    ds = small_grid(4100, seed=8)
    hk.set_events(ds.t, ds.county, ds.county_scale, ds.x, ds.y)
    ref, rows = oracle_rows(ds)
    cuts = [0, 700, 2500, 3072, ds.n]
    for flags, tl, tg in ((HAWKES_F64, TOL_F64, TOL_F64), (HAWKES_F32, TOL_LL32, TOL_G32)):
        tot_ll, tot_g = 0.0, np.zeros(6)
        for a, b in zip(cuts[:-1], cuts[1:]):
            ll, g = hk.loglik_grad(P0, flags, a, b)
            wref = oracle.loglik_grad(ds.t, ds.x, ds.y, P0, s=ds.s, row_begin=a, row_end=b)
            assert_close(ll, g, wref, rows[a:b], tl, tg, f"window [{a},{b})")
            tot_ll += ll
            tot_g += g
        assert_close(tot_ll, tot_g, ref, rows, tl, tg, "sum of windows")


def test_async_matches_sync(hk):
    torch = pytest.importorskip("torch")
    ds = small_grid(3000, seed=9)
    hk.set_events(ds.t, ds.county, ds.county_scale, ds.x, ds.y)
    ll, g = hk.loglik_grad(P0, HAWKES_F32)
    dp = torch.tensor(P0, dtype=torch.float64, device="cuda")
    dout = torch.zeros(7, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    hk.loglik_grad_async(dp.data_ptr(), dout.data_ptr(), HAWKES_F32)
    hk.profile()  # waits for the context stream
    o = dout.cpu().numpy()
    # FP32 partial sums are combined with atomics whose order varies from run
    # to run, so repeated evaluations agree to the FP32 path's tolerance only
    ref, rows = oracle_rows(ds)
    assert_close(o[0], o[1:], np.concatenate([[ll], g]), rows, TOL_LL32, TOL_G32, "async vs sync")


def test_resample_bit_exact(hk):
    for ds in (synth.config_dataset("c1"),
               synth.voronoi_dataset(20_000, n_cells=300, seed=10)):
        hk.load(ds)
        for it in (0, 1, 17):
            hk.resample(1234, 5, it)
            gx, gy = hk.locations()
            ox, oy = oracle.resample(ds.county, ds.counties.n, ds.counties.tri_county,
                                     ds.counties.tri_xy, 1234, 5, it)
            assert np.array_equal(gx, ox) and np.array_equal(gy, oy), f"iteration {it}"
        # the likelihood then uses the resampled locations
        ll, g = hk.loglik_grad(P0, HAWKES_F32)
        if ds.n <= 2000:
            ref, rows = oracle.loglik_grad(ds.t, ox, oy, P0, s=ds.s, rows=True)
            assert_close(ll, g, ref, rows, TOL_LL32, TOL_G32, "after resample")


def test_invalid_input_is_reported(hk):
    ds = small_grid(100, seed=11)
    with pytest.raises(HawkesError) as e:
        hk.set_events(ds.t[::-1].copy(), ds.county, ds.county_scale, ds.x, ds.y)
    assert e.value.status == -2
    with pytest.raises(HawkesError) as e:
        bad = ds.county.copy()
        bad[3] = 10_000
        hk.set_events(ds.t, bad, ds.county_scale, ds.x, ds.y)
    assert e.value.status == -1
    hk.set_events(ds.t, ds.county, ds.county_scale, ds.x, ds.y)
    with pytest.raises(HawkesError):
        hk.loglik_grad((0.5, -1.0, 7.0, 0.3, 0.2, 2.0))
    with pytest.raises(HawkesError):
        hk.loglik_grad(P0, HAWKES_F32, 50, 10)
    ll, g = hk.loglik_grad(P0)  # the context stays usable
    assert np.isfinite(ll)


@pytest.mark.parametrize("ties", [False, True])
def test_underflow_skip_matches_oracle(hk, ties):
    """Skipping tiles whose terms are exact FP32 zeros changes nothing: a
    6,000-event workload over 1,200 days (most pairs far apart in time)."""
    ds = synth.grid_dataset(6000, 1200.0, 20, 20, seed=15)
    if ties:
        ds = synth.integer_day_times(ds)
    hk.set_events(ds.t, ds.county, ds.county_scale, ds.x, ds.y)
    ref, rows = oracle_rows(ds)
    for p in (P0, (0.5, 20.0, 7.0, 0.3, 2.0, 2.0)):
        ref, rows = oracle_rows(ds, p)
        ll, g = hk.loglik_grad(p, HAWKES_F32 | HAWKES_SKIP_UNDERFLOW)
        assert_close(ll, g, ref, rows, TOL_LL32, TOL_G32, "skip")
        ll2, g2 = hk.loglik_grad(p, HAWKES_F32 | HAWKES_SKIP_UNDERFLOW, 1000, 5000)
        w = oracle.loglik_grad(ds.t, ds.x, ds.y, p, s=ds.s, row_begin=1000, row_end=5000)
        assert_close(ll2, g2, w, rows[1000:5000], TOL_LL32, TOL_G32, "skip window")


def test_underflow_skip_c2_matches_full(hk):
    ds = synth.config_dataset("c2")
    hk.set_events(ds.t, ds.county, ds.county_scale, ds.x, ds.y)
    full, rows = hk.loglik_rows(P0, HAWKES_F32)
    ll, g = hk.loglik_grad(P0, HAWKES_F32 | HAWKES_SKIP_UNDERFLOW)
    assert_close(ll, g, full, rows, 1e-9, 1e-8, "skip vs full")


def test_bounded_wait_gives_up_and_context_survives(hk):
    """A device-side wait on a barrier that nothing completes must give up
    within its bound (about 2 s), report HAWKES_ERR_TIMEOUT, and leave the
    context usable."""
    sec = hk.check_bounded_wait()
    assert 0.2 < sec < 20.0
    ds = small_grid(500, seed=14)
    hk.set_events(ds.t, ds.county, ds.county_scale, ds.x, ds.y)
    ref = oracle.loglik_grad(ds.t, ds.x, ds.y, P0, s=ds.s)
    ll, g = hk.loglik_grad(P0)
    assert abs(ll - ref[0]) <= TOL_LL32 * abs(ref[0])


def test_c2_sampled_rows_and_paths(hk):
    """N=100,000 (60x60 grid, 1,200 d) after one resample: FP32 rows against the
    oracle one by one on sampled rows; FP32 totals against the FP64 GPU path."""
    ds = synth.config_dataset("c2")
    hk.load(ds)
    hk.resample(1, 0, 0)
    x, y = hk.locations()
    out32, rows32 = hk.loglik_rows(P0, HAWKES_F32)
    ll64, g64 = hk.loglik_grad(P0, HAWKES_F64)
    rng = np.random.default_rng(0)
    idx = np.concatenate([[0, 1, ds.n - 1], rng.choice(ds.n, 61, replace=False)])
    ref = np.stack([oracle.loglik_grad(ds.t, x, y, P0, s=ds.s, row_begin=i, row_end=i + 1,
                                       rows=True)[1][0] for i in idx])
    got = rows32[idx]
    assert np.max(np.abs(got[:, 7] - ref[:, 7])) < 2e-6
    assert np.max(np.abs(got[:, 8] - ref[:, 8]) / np.abs(ref[:, 8])) < 1e-12
    gscale = np.abs(ref[:, 1:7]).max(axis=0)
    assert np.all(np.abs(got[:, 1:7] - ref[:, 1:7]) <= TOL_G32 * np.maximum(np.abs(ref[:, 1:7]), 1e-3 * gscale))
    # totals: FP32 against the FP64 GPU path (itself pinned to the oracle above)
    ref7 = np.concatenate([[ll64], g64])
    assert_close(out32[0], out32[1:], ref7, rows32, TOL_LL32, TOL_G32, "c2 f32 vs f64")


def test_c3_full_size_sampled(hk):
    """N=1,000,000 Voronoi workload in the benchmark's launch configuration:
    sampled rows against the oracle, and row shards summing to the whole."""
    ds = synth.config_dataset("c3")
    hk.load(ds)
    hk.resample(2, 0, 0)
    x, y = hk.locations()
    out32, rows32 = hk.loglik_rows(P0, HAWKES_F32)
    assert np.all(np.isfinite(out32))
    rng = np.random.default_rng(1)
    idx = np.concatenate([[0, ds.n // 2, ds.n - 1], rng.choice(ds.n, 21, replace=False)])
    ref = np.stack([oracle.loglik_grad(ds.t, x, y, P0, s=ds.s, row_begin=i, row_end=i + 1,
                                       rows=True)[1][0] for i in idx])
    got = rows32[idx]
    assert np.max(np.abs(got[:, 7] - ref[:, 7])) < 2e-6
    assert np.max(np.abs(got[:, 8] - ref[:, 8]) / np.abs(ref[:, 8])) < 1e-12
    gscale = np.abs(ref[:, 1:7]).max(axis=0)
    assert np.all(np.abs(got[:, 1:7] - ref[:, 1:7]) <= TOL_G32 * np.maximum(np.abs(ref[:, 1:7]), 1e-3 * gscale))
    # the sum over rows of the per-row values is the total
    assert abs(rows32[:, 0].sum() - out32[0]) <= 1e-9 * abs(out32[0])
    # shards (window kernel, no symmetric shortcut) sum to the symmetric whole
    cuts = [0, 400_000, 700_000, ds.n]
    tot = np.zeros(7)
    for a, b in zip(cuts[:-1], cuts[1:]):
        ll, g = hk.loglik_grad(P0, HAWKES_F32, a, b)
        tot += np.concatenate([[ll], g])
    assert_close(tot[0], tot[1:], out32, rows32, TOL_LL32, TOL_G32, "c3 shards")


# ---------------------------------------------------------------------------
# Eq. 2's time-only background (HAWKES_BG_TIME)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n,ties,model1", [(1, False, False), (257, False, False),
                                           (2049, False, True), (3000, True, False),
                                           (5000, False, False)])
def test_bg_time_matches_oracle(hk, n, ties, model1):
    ds = small_grid(n, seed=40 + n)
    if ties:
        ds = synth.integer_day_times(ds)
    hk.set_events(ds.t, ds.county, ds.county_scale, ds.x, ds.y)
    ref, rows = oracle_rows(ds, model1=model1, bg_time=True)
    fl = HAWKES_BG_TIME | (HAWKES_MODEL1 if model1 else 0)
    ll, g = hk.loglik_grad(P0, HAWKES_F64 | fl)
    assert_close(ll, g, ref, rows, TOL_F64, TOL_F64, f"bg_time n={n} f64")
    ll, g = hk.loglik_grad(P0, HAWKES_F32 | fl)
    assert_close(ll, g, ref, rows, TOL_LL32, TOL_G32, f"bg_time n={n} f32")
    if n > 1:  # the background really changed
        other = oracle_rows(ds, model1=model1)[0]
        assert abs(other[0] - ref[0]) > 1e-3 * abs(ref[0])


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4])
def test_bg_time_variants_and_windows(hk, variant):
    ds = small_grid(6000, seed=41)
    hk.set_events(ds.t, ds.county, ds.county_scale, ds.x, ds.y)
    ref, rows = oracle_rows(ds, bg_time=True)
    hk.set_variant(variant)
    try:
        ll, g = hk.loglik_grad(P0, HAWKES_F32 | HAWKES_BG_TIME)
        assert_close(ll, g, ref, rows, TOL_LL32, TOL_G32, f"bg_time variant {variant}")
        wref, _ = oracle_rows(ds, bg_time=True, row_begin=1000, row_end=4500)
        ll, g = hk.loglik_grad(P0, HAWKES_F32 | HAWKES_BG_TIME, 1000, 4500)
        assert_close(ll, g, wref, rows[1000:4500], TOL_LL32, TOL_G32, f"bg_time variant {variant} window")
    finally:
        hk.set_variant(0)


def test_bg_time_with_underflow_skip(hk):
    ds = synth.integer_day_times(synth.grid_dataset(6000, 1200.0, 20, 20, seed=42))
    hk.set_events(ds.t, ds.county, ds.county_scale, ds.x, ds.y)
    ref, rows = oracle_rows(ds, bg_time=True)
    ll, g = hk.loglik_grad(P0, HAWKES_F32 | HAWKES_BG_TIME | HAWKES_SKIP_UNDERFLOW)
    assert_close(ll, g, ref, rows, TOL_LL32, TOL_G32, "bg_time + skip")


@pytest.mark.parametrize("bg_time", [False, True])
def test_integer_days_100k_against_fp64_path(hk, bg_time):
    """N = 100,000 on integer days (runs of equal time gaps, the regime where
    long FP32 summation chains drift), FP32 path against the FP64 path (which
    the tests above hold to 1e-10 of the oracle), at the FP32 tolerances."""
    ds = synth.integer_day_times(synth.grid_dataset(100_000, 300.0, 20, 20, seed=5))
    hk.set_events(ds.t, ds.county, ds.county_scale, ds.x, ds.y)
    fl = HAWKES_BG_TIME if bg_time else 0
    ref, rows = hk.loglik_rows(P0, HAWKES_F64 | fl)
    ll, g = hk.loglik_grad(P0, HAWKES_F32 | fl)
    assert_close(ll, g, ref, rows, TOL_LL32, TOL_G32, f"integer days 100k bg_time={bg_time}")


def test_tune_cache_on_the_device(hk, tmp_path):
    """The first cached tune searches and stores, the second reads the file:
    same variant, selected on the context, under the documented key."""
    import json
    from paper_2407_11349_gb300.hawkes import hawkes_get_sweep_variant, hawkes_sweep_variants
    ds = small_grid(20000, seed=13)
    hk.set_events(ds.t, ds.county, ds.county_scale, ds.x, ds.y)
    path = str(tmp_path / "tune.json")
    v1, hit1 = hk.tune_cached(P0, path, reps=1)
    assert not hit1 and 0 <= v1 < hawkes_sweep_variants()
    hk.set_variant((v1 + 1) % hawkes_sweep_variants())
    v2, hit2 = hk.tune_cached(P0, path, reps=1)
    assert hit2 and v2 == v1 and hawkes_get_sweep_variant(hk.ctx) == v1
    doc = json.load(open(path))
    (key,) = doc
    assert key.endswith("|single|n<=2^15|flags=0") and "|sm_10" in key
    v3, hit3 = hk.tune_cached(P0, path, flags=HAWKES_BG_TIME, reps=1)  # another key: a miss
    assert not hit3 and len(json.load(open(path))) == 2
    hk.set_variant(0)


def _synthetic(n, seed, t=None, same_xy=False):
    ds = small_grid(n, seed=seed)
    if t is not None:
        ds.t = np.full(n, float(t))
    if same_xy:
        ds.x = np.full(n, ds.x[0])
        ds.y = np.full(n, ds.y[0])
    return ds


def _check_flags(hk, ds, p, fl=0, what=""):
    hk.set_events(ds.t, ds.county, ds.county_scale, ds.x, ds.y)
    ref, rows = oracle.loglik_grad(ds.t, ds.x, ds.y, p, s=ds.s, rows=True, bg_time_only=bool(fl & HAWKES_BG_TIME))
    for prec, tl, tg in ((HAWKES_F64, TOL_F64, TOL_F64), (HAWKES_F32, TOL_LL32, TOL_G32)):
        ll, g = hk.loglik_grad(p, prec | fl)
        assert_close(ll, g, ref, rows, tl, tg, f"{what} prec={prec}")
    return ref, rows


def test_all_events_at_one_instant(hk):
    """Every pair is a tie: no background, no excitation, every rate clipped;
    ell = N log(1e-40) - sum Lambda_i, and only the Lambda terms have a gradient."""
    ds = _synthetic(3000, 50, t=37.5)
    ref, rows = _check_flags(hk, ds, P0, what="one instant")
    assert np.all(rows[:, 7] == np.log(1e-40))


def test_all_events_at_one_location(hk):
    """r = 0 for every pair: the spatial factors are at their maxima."""
    ds = _synthetic(2500, 51, same_xy=True)
    _check_flags(hk, ds, P0, what="one location")
    _check_flags(hk, ds, P0, HAWKES_BG_TIME, what="one location, time-only background")


@pytest.mark.parametrize("p", [(0.5, 0.05, 0.01, 0.3, 50.0, 0.01),     # tiny bandwidths: most terms underflow
                               (0.5, 5e3, 1e3, 0.3, 1e-3, 5e2)])      # huge bandwidths: every pair counts
def test_extreme_bandwidths(hk, p):
    ds = small_grid(3000, seed=52)
    _check_flags(hk, ds, p, what=f"p={p}")


# ---------------------------------------------------------------------------
# Exact spatial skip (HAWKES_SKIP_SPATIAL)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n,window,ties,model1", [(300, 256, False, False), (6000, 1024, False, False),
                                                  (6000, 1024, True, False), (5000, 256, False, True),
                                                  (7000, 32768, True, False)])
def test_spatial_skip_matches_oracle(hk, n, window, ties, model1):
    """Events over 1,200 days on a 20 x 20 grid of 50 km counties: most pairs
    are exact FP32 zeros by time or distance and are skipped; the sum of the
    rest equals the oracle's at the FP32-path tolerances."""
    from paper_2407_11349_gb300.hawkes import HAWKES_SKIP_SPATIAL
    ds = synth.grid_dataset(n, 1200.0, 20, 20, seed=60 + n + window)
    if ties:
        ds = synth.integer_day_times(ds)
    hk.set_events(ds.t, ds.county, ds.county_scale, ds.x, ds.y)
    hk.set_spatial_window(window)
    s = None if model1 else ds.s
    ref, rows = oracle.loglik_grad(ds.t, ds.x, ds.y, P0, s=s, rows=True)
    fl = HAWKES_F32 | HAWKES_SKIP_SPATIAL | (HAWKES_MODEL1 if model1 else 0)
    ll, g = hk.loglik_grad(P0, fl)
    assert_close(ll, g, ref, rows, TOL_LL32, TOL_G32, f"spatial n={n} window={window}")
    # other bandwidths, same order: on these sparse events (1,200 days) every
    # excitation term but a few is below FP32's 2^-126, so d/dh and d/domega
    # rest on terms FP32 flushes; the flush-bound fix-up recomputes the rows
    # that carry them in FP64
    p2 = (2.0, 5.0, 2.0, 0.9, 1.5, 0.7)
    ll2, g2 = hk.loglik_grad(p2, fl)
    ref2, rows2 = oracle.loglik_grad(ds.t, ds.x, ds.y, p2, s=s, rows=True)
    assert_close(ll2, g2, ref2, rows2, TOL_LL32, TOL_G32, f"spatial n={n} other parameters")


def test_spatial_skip_after_resample_and_at_100k(hk):
    """The order is built from the locations of its first use; after a
    resample the tiles' boxes follow the events.  N = 100,000 over 1,200 days
    against the regular FP32 path."""
    from paper_2407_11349_gb300.hawkes import HAWKES_SKIP_SPATIAL
    ds = synth.config_dataset("c2")
    hk.load(ds)
    hk.set_spatial_window(32768)
    ll_a, g_a = hk.loglik_grad(P0, HAWKES_F32 | HAWKES_SKIP_SPATIAL)
    ll_b, g_b = hk.loglik_grad(P0, HAWKES_F32)
    scale = np.abs(g_b) + 1e-3 * np.max(np.abs(g_b))
    assert abs(ll_a - ll_b) <= 1e-6 * abs(ll_b) and np.all(np.abs(g_a - g_b) <= 1e-5 * scale)
    hk.resample(3, 0, 1)
    ll_a, g_a = hk.loglik_grad(P0, HAWKES_F32 | HAWKES_SKIP_SPATIAL)
    ll_b, g_b = hk.loglik_grad(P0, HAWKES_F32)
    scale = np.abs(g_b) + 1e-3 * np.max(np.abs(g_b))
    assert abs(ll_a - ll_b) <= 1e-6 * abs(ll_b) and np.all(np.abs(g_a - g_b) <= 1e-5 * scale)


def test_spatial_skip_rejects_what_it_does_not_cover(hk):
    from paper_2407_11349_gb300.hawkes import HAWKES_SKIP_SPATIAL
    ds = small_grid(2000, seed=61)
    hk.set_events(ds.t, ds.county, ds.county_scale, ds.x, ds.y)
    for fl, rows in ((HAWKES_F64 | HAWKES_SKIP_SPATIAL, None), (HAWKES_BG_TIME | HAWKES_SKIP_SPATIAL, None),
                     (HAWKES_SKIP_SPATIAL, (100, 900))):
        with pytest.raises(HawkesError) as e:
            if rows:
                hk.loglik_grad(P0, fl, *rows)
            else:
                hk.loglik_grad(P0, fl)
        assert e.value.status == -1
    with pytest.raises(HawkesError):
        hk.set_spatial_window(100)
    ll, g = hk.loglik_grad(P0, HAWKES_F32)  # still usable
    assert np.isfinite(ll)


# ---------------------------------------------------------------------------
# Terms below FP32's range: the flush-bound fix-up of the FP32 path
# ---------------------------------------------------------------------------

def raw_rel(got, ref):
    """Relative error of each output against its own magnitude (no floor)."""
    return np.abs(np.asarray(got) - ref) / np.maximum(np.abs(ref), 1e-300)


@pytest.mark.parametrize("n,p", [(300, (2.0, 5.0, 2.0, 0.9, 1.5, 0.7)), (6000, (2.0, 5.0, 2.0, 0.9, 1.5, 0.7)),
                                 (3000, (0.5, 0.05, 0.01, 0.3, 50.0, 0.01))])
@pytest.mark.parametrize("extra", [0, HAWKES_SKIP_UNDERFLOW])
def test_flushed_terms_fp32_path_matches_oracle_unfloored(hk, n, p, extra):
    """Sparse events (1,200 days, 20 x 20 grid of 50 km counties) at
    bandwidths where nearly every excitation term, or every term, is below
    2^-126: the outputs that rest on those terms are tiny but nonzero in the
    oracle.  The FP32 path must still give every output within 1e-6 (ell)
    and 1e-5 (each partial) of the oracle relative to the output itself."""
    ds = synth.grid_dataset(n, 1200.0, 20, 20, seed=70 + n)
    hk.set_events(ds.t, ds.county, ds.county_scale, ds.x, ds.y)
    ref, rows = oracle.loglik_grad(ds.t, ds.x, ds.y, p, s=ds.s, rows=True)
    ll, g = hk.loglik_grad(p, HAWKES_F32 | extra)
    e = raw_rel(np.concatenate([[ll], g]), ref)
    assert e[0] <= TOL_LL32 and np.all(e[1:] <= TOL_G32), f"raw rel errs {e} (ref {ref})"
    out, rws = hk.loglik_rows(p, HAWKES_F32 | extra)  # per-row values follow the fix-up
    assert np.allclose(out, np.concatenate([[ll], g]), rtol=1e-12, atol=0)
    assert abs(rws[:, 0].sum() - out[0]) <= 1e-9 * abs(out[0])
    assert np.all(raw_rel(rws[:, 1:7].sum(axis=0), out[1:]) <= 1e-9)


def test_flush_fixup_is_idle_at_normal_bandwidths(hk):
    """At the workload's parameters no row is recomputed for the flush bound:
    the outputs equal those of the sweep alone, so the FP32 path costs what
    it did before the fix-up existed (checked through the per-kernel
    timing: the fix-up kernel returns at once)."""
    ds = synth.config_dataset("c2")
    hk.load(ds)
    hk.profile(True)
    hk.loglik_grad(P0, HAWKES_F32)
    prof = hk.profile(False)
    launches, ms = prof["rows64"]
    assert launches == 2 and ms < 0.2, prof  # the floor-rate rows and the idle fix-up


# ---------------------------------------------------------------------------
# Full-size totals at N = 1,000,000 (c3)
# ---------------------------------------------------------------------------

def _golden_c3():
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_c3.json")
    return json.load(open(path)) if os.path.exists(path) else None


def test_c3_totals_against_fp64_path_and_stored_oracle(hk):
    """The whole N = 1,000,000 sum after resample(2, 0, 0): the FP32 path's
    seven totals against the FP64 GPU path at full size, and both against the
    oracle's values stored in tests/golden/oracle_c3.json (written by
    tests/golden/make_golden_c3.py from the oracle alone) once the inputs are
    checked to be the same.  Errors are relative to each output itself, with
    no floor: 1e-6 (ell) and 1e-5 (each partial) for FP32, 1e-10 for FP64."""
    ds = synth.config_dataset("c3")
    hk.load(ds)
    hk.resample(2, 0, 0)
    x, y = hk.locations()
    f32 = np.concatenate(hk.loglik_grad(P0, HAWKES_F32), axis=None)
    f64 = np.concatenate(hk.loglik_grad(P0, HAWKES_F64), axis=None)
    e = raw_rel(f32, f64)
    print("c3 FP32 vs FP64 GPU, raw relative errors:", e)
    assert e[0] <= TOL_LL32 and np.all(e[1:] <= TOL_G32), e
    doc = _golden_c3()
    assert doc is not None, "tests/golden/oracle_c3.json missing"
    fp = synth.fingerprint({"t": ds.t, "x": x, "y": y, "s": ds.s})
    assert synth.same_inputs(fp["stats"], doc["inputs"]["stats"]), "c3 inputs differ from the stored ones"
    ref = np.array(doc["loglik_grad"])
    e32, e64 = raw_rel(f32, ref), raw_rel(f64, ref)
    print("c3 against the stored oracle: FP32", e32, "FP64", e64)
    assert np.all(e64 <= TOL_F64), e64
    assert e32[0] <= TOL_LL32 and np.all(e32[1:] <= TOL_G32), e32
