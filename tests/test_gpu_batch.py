"""Batched evaluation (one persistent sweep launch over many problems, and its
CUDA-graph replay) against the FP64 CPU oracle on each problem's own location
draw, and against one call per problem through the regular entry point, at
the FP32-path tolerances of the parity tests."""
import numpy as np
import pytest

from paper_2407_11349_gb300 import synth
from paper_2407_11349_gb300.hawkes import Batch, Hawkes, HAWKES_BG_TIME, HAWKES_F32, HawkesError

pytestmark = pytest.mark.gpu

TOL_LL32 = 1e-6
TOL_G32 = 1e-5


def _close(got, ref, rows, what):
    scale = np.abs(rows[:, 1:7]).sum(axis=0)
    e_ll = abs(got[0] - ref[0]) / abs(ref[0])
    denom = np.maximum(np.abs(ref[1:]), 1e-3 * scale)
    e_g = np.abs(got[1:] - ref[1:]) / np.where(denom > 0, denom, 1.0)
    assert e_ll <= TOL_LL32, f"{what}: loglik rel err {e_ll:.3g}"
    assert np.all(e_g <= TOL_G32), f"{what}: grad rel errs {e_g}"


@pytest.fixture(scope="module")
def problems():
    torch = pytest.importorskip("torch")
    base = synth.voronoi_dataset(20_000, n_cells=400, seed=31)
    chains = [base] * 4
    regions = synth.regional_subsets(base, [3_000, 7_100, 12_345], seed=32)
    dss = chains + regions
    params = synth.chain_params(len(dss), seed=33)
    hks = [Hawkes(0).load(ds) for ds in dss]
    seeds = [77] * len(dss)
    streams = list(range(len(dss)))
    yield torch, dss, params, hks, seeds, streams
    for h in hks:
        h.close()


def _sequential(hks, params, seeds, streams, it, flags=HAWKES_F32):
    out = []
    for h, p, sd, st in zip(hks, params, seeds, streams):
        h.resample(sd, st, it)
        ref, rows = h.loglik_rows(p, flags)
        out.append((ref, rows))
    return out


def test_batch_eager_and_graph_match_sequential(problems):
    torch, dss, params, hks, seeds, streams = problems
    P = len(dss)
    dp = torch.tensor(params, dtype=torch.float64, device="cuda")
    dout = torch.zeros((P, 7), dtype=torch.float64, device="cuda")
    b = Batch(hks, seeds, streams, HAWKES_F32)
    try:
        torch.cuda.synchronize()
        b.run(dp.data_ptr(), 3, dout.data_ptr())
        b.wait()
        got = dout.cpu().numpy()
        ref = _sequential(hks, params, seeds, streams, 3)
        for p in range(P):
            _close(got[p], *ref[p], f"eager problem {p}")
        b.capture(dp.data_ptr(), dout.data_ptr())
        for it in (5, 6):
            dout.zero_()
            torch.cuda.synchronize()
            b.run(dp.data_ptr(), it, dout.data_ptr())
            b.wait()
            got = dout.cpu().numpy()
            ref = _sequential(hks, params, seeds, streams, it)
            for p in range(P):
                _close(got[p], *ref[p], f"graph iteration {it} problem {p}")
    finally:
        b.close()


@pytest.mark.parametrize("graph", [False, True])
def test_batch_matches_oracle(problems, graph):
    """Every problem's seven outputs against the oracle evaluated on the
    locations the batch drew for it (read back from its context): 4 chains
    of a 20,000-event Voronoi workload with their own parameters and
    resample streams, and 3 regional subsets of uneven size."""
    import oracle
    torch, dss, params, hks, seeds, streams = problems
    P = len(dss)
    dp = torch.tensor(params, dtype=torch.float64, device="cuda")
    dout = torch.zeros((P, 7), dtype=torch.float64, device="cuda")
    b = Batch(hks, seeds, streams, HAWKES_F32)
    try:
        if graph:
            b.capture(dp.data_ptr(), dout.data_ptr())
        torch.cuda.synchronize()
        b.run(dp.data_ptr(), 21, dout.data_ptr())
        b.wait()
        got = dout.cpu().numpy()
    finally:
        b.close()
    for p in range(P):
        x, y = hks[p].locations()
        ref, rows = oracle.loglik_grad(dss[p].t, x, y, params[p], s=dss[p].s, rows=True)
        _close(got[p], ref, rows, f"{'graph' if graph else 'eager'} problem {p} vs oracle")
    # the chains share events but drew their own locations
    x0, _ = hks[0].locations()
    x1, _ = hks[1].locations()
    assert not np.array_equal(x0, x1)


def test_batch_tune_then_still_correct(problems):
    torch, dss, params, hks, seeds, streams = problems
    P = len(dss)
    dp = torch.tensor(params, dtype=torch.float64, device="cuda")
    dout = torch.zeros((P, 7), dtype=torch.float64, device="cuda")
    b = Batch(hks, seeds, streams, HAWKES_F32)
    try:
        torch.cuda.synchronize()
        v, ch, order, ms = b.tune(dp.data_ptr(), dout.data_ptr(), reps=1)
        assert 0 <= v < 5 and ch in (16, 32, 64) and order in (0, 1) and ms > 0
        b.run(dp.data_ptr(), 9, dout.data_ptr())
        b.wait()
        got = dout.cpu().numpy()
        ref = _sequential(hks, params, seeds, streams, 9)
        for p in range(P):
            _close(got[p], *ref[p], f"tuned problem {p}")
    finally:
        b.close()


def test_batch_reports_invalid_problem(problems):
    torch, dss, params, hks, seeds, streams = problems
    P = len(dss)
    bad = params.copy()
    bad[2, 1] = -1.0  # tau_x < 0 for problem 2
    dp = torch.tensor(bad, dtype=torch.float64, device="cuda")
    dout = torch.zeros((P, 7), dtype=torch.float64, device="cuda")
    b = Batch(hks, None, None, HAWKES_F32)
    try:
        torch.cuda.synchronize()
        b.run(dp.data_ptr(), 0, dout.data_ptr())
        with pytest.raises(HawkesError):
            b.wait()
        got = dout.cpu().numpy()
        assert np.all(np.isnan(got[2])) and np.all(np.isfinite(np.delete(got, 2, axis=0)))
    finally:
        b.close()


def test_batch_time_only_background(problems):
    """The batch with eq. 2's time-only background against sequential calls
    with the same flag."""
    torch, dss, params, hks, seeds, streams = problems
    P = len(dss)
    fl = HAWKES_F32 | HAWKES_BG_TIME
    dp = torch.tensor(params, dtype=torch.float64, device="cuda")
    dout = torch.zeros((P, 7), dtype=torch.float64, device="cuda")
    b = Batch(hks, seeds, streams, fl)
    try:
        b.capture(dp.data_ptr(), dout.data_ptr())
        torch.cuda.synchronize()
        b.run(dp.data_ptr(), 9, dout.data_ptr())
        b.wait()
        got = dout.cpu().numpy()
        ref = _sequential(hks, params, seeds, streams, 9, fl)
        for p in range(P):
            _close(got[p], *ref[p], f"time-only background problem {p}")
    finally:
        b.close()


def test_batch_tune_cached(problems, tmp_path):
    torch, dss, params, hks, seeds, streams = problems
    P = len(dss)
    dp = torch.tensor(params, dtype=torch.float64, device="cuda")
    dout = torch.zeros((P, 7), dtype=torch.float64, device="cuda")
    path = str(tmp_path / "tune.json")
    b = Batch(hks, seeds, streams, HAWKES_F32)
    try:
        first = b.tune_cached(dp.data_ptr(), dout.data_ptr(), path)
        assert first[3] is False
        b.set_config(0, 16, 1)
        second = b.tune_cached(dp.data_ptr(), dout.data_ptr(), path)
        assert second[3] is True and second[:3] == first[:3]
        torch.cuda.synchronize()
        b.run(dp.data_ptr(), 4, dout.data_ptr())
        b.wait()
        got = dout.cpu().numpy()
        ref = _sequential(hks, params, seeds, streams, 4)
        for p in range(P):
            _close(got[p], *ref[p], f"cached configuration problem {p}")
    finally:
        b.close()


def test_batch_with_underflow_skip(problems):
    """The batch with the exact underflow skip (which reads each problem's
    times from its descriptor) against sequential calls without it."""
    from paper_2407_11349_gb300.hawkes import HAWKES_SKIP_UNDERFLOW
    torch, dss, params, hks, seeds, streams = problems
    assert max(ds.t[-1] - ds.t[0] for ds in dss) > 500.0  # long enough for skips
    P = len(dss)
    dp = torch.tensor(params, dtype=torch.float64, device="cuda")
    dout = torch.zeros((P, 7), dtype=torch.float64, device="cuda")
    b = Batch(hks, seeds, streams, HAWKES_F32 | HAWKES_SKIP_UNDERFLOW)
    try:
        torch.cuda.synchronize()
        b.run(dp.data_ptr(), 11, dout.data_ptr())
        b.wait()
        got = dout.cpu().numpy()
        ref = _sequential(hks, params, seeds, streams, 11)
        for p in range(P):
            _close(got[p], *ref[p], f"skip problem {p}")
        b.capture(dp.data_ptr(), dout.data_ptr())
        torch.cuda.synchronize()
        b.run(dp.data_ptr(), 12, dout.data_ptr())
        b.wait()
        got = dout.cpu().numpy()
        ref = _sequential(hks, params, seeds, streams, 12)
        for p in range(P):
            _close(got[p], *ref[p], f"skip graph problem {p}")
    finally:
        b.close()


# ---------------------------------------------------------------------------
# Several chains per CTA (problems with identical event times swept together)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("kc,graph", [(2, False), (2, True), (4, False), (4, True)])
def test_chains_per_cta_matches_oracle(problems, kc, graph):
    """The four chains share their event times, so k = 2 makes two groups and
    k = 4 one; the regional subsets are swept one per item.  Every problem's
    outputs against the oracle on its own location draw, and against the
    batch with one chain per CTA on the same draws."""
    import oracle
    torch, dss, params, hks, seeds, streams = problems
    P = len(dss)
    dp = torch.tensor(params, dtype=torch.float64, device="cuda")
    dout = torch.zeros((P, 7), dtype=torch.float64, device="cuda")
    b = Batch(hks, seeds, streams, HAWKES_F32)
    try:
        b.set_chains_per_cta(kc)
        assert b.config()[3:] == (kc, 4 // kc)
        if graph:
            b.capture(dp.data_ptr(), dout.data_ptr())
        torch.cuda.synchronize()
        b.run(dp.data_ptr(), 23, dout.data_ptr())
        b.wait()
        got = dout.cpu().numpy()
        b.set_chains_per_cta(1)
        assert b.config()[3:] == (1, 0)
        b.run(dp.data_ptr(), 23, dout.data_ptr())
        b.wait()
        one = dout.cpu().numpy()
    finally:
        b.close()
    for p in range(P):
        x, y = hks[p].locations()
        ref, rows = oracle.loglik_grad(dss[p].t, x, y, params[p], s=dss[p].s, rows=True)
        _close(got[p], ref, rows, f"k={kc} {'graph' if graph else 'eager'} problem {p} vs oracle")
        _close(got[p], one[p], rows, f"k={kc} vs k=1 problem {p}")


def test_chains_per_cta_remainder_model1_and_invalid_member():
    """Three chains of one data set and one other problem at k = 2 (Model 1):
    one group of two, the third chain and the other problem one per item.
    Then a group member with invalid parameters: its outputs are NaN and the
    error is reported, its group partner is unaffected."""
    import oracle
    from paper_2407_11349_gb300.hawkes import HAWKES_MODEL1
    torch = pytest.importorskip("torch")
    base = synth.voronoi_dataset(9_000, n_cells=200, seed=41)
    other = synth.voronoi_dataset(4_321, n_cells=100, seed=42)
    dss = [base, base, base, other]
    params = synth.chain_params(4, seed=43)
    hks = [Hawkes(0).load(ds) for ds in dss]
    fl = HAWKES_F32 | HAWKES_MODEL1
    dp = torch.tensor(params, dtype=torch.float64, device="cuda")
    dout = torch.zeros((4, 7), dtype=torch.float64, device="cuda")
    b = Batch(hks, [5] * 4, [0, 1, 2, 3], fl)
    try:
        b.set_chains_per_cta(2)
        assert b.config()[3:] == (2, 1)
        torch.cuda.synchronize()
        b.run(dp.data_ptr(), 3, dout.data_ptr())
        b.wait()
        got = dout.cpu().numpy()
        refs = []
        for p in range(4):
            x, y = hks[p].locations()
            refs.append(oracle.loglik_grad(dss[p].t, x, y, params[p], s=None, rows=True))
            _close(got[p], *refs[p], f"remainder problem {p}")
        bad = params.copy()
        bad[1, 2] = -1.0  # tau_t < 0 for the second member of the group
        dp.copy_(torch.from_numpy(bad))
        b.run(dp.data_ptr(), 3, dout.data_ptr())
        with pytest.raises(HawkesError):
            b.wait()
        got2 = dout.cpu().numpy()
        assert np.all(np.isnan(got2[1]))
        for p in (0, 2, 3):
            _close(got2[p], *refs[p], f"valid problem {p} beside an invalid group member")
    finally:
        b.close()
        for h in hks:
            h.close()


def test_chains_per_cta_arguments(problems):
    """k must be 1, 2 or 4, and k > 1 needs the full space-time gradient."""
    from paper_2407_11349_gb300.hawkes import HAWKES_LOGLIK_ONLY, HAWKES_SKIP_UNDERFLOW
    torch, dss, params, hks, seeds, streams = problems
    b = Batch(hks, seeds, streams, HAWKES_F32)
    try:
        for k in (0, 3, 5, 8):
            with pytest.raises(HawkesError):
                b.set_chains_per_cta(k)
    finally:
        b.close()
    for fl in (HAWKES_BG_TIME, HAWKES_LOGLIK_ONLY, HAWKES_SKIP_UNDERFLOW):
        b = Batch(hks, seeds, streams, HAWKES_F32 | fl)
        try:
            with pytest.raises(HawkesError):
                b.set_chains_per_cta(2)
            b.set_chains_per_cta(1)
        finally:
            b.close()
