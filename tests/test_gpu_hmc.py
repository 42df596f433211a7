"""Surrogate HMC on the GPU: exact-kernel evaluations from warmup train the
network on the GPU; then exact HMC and surrogate HMC sample the same target
(locations held fixed, so both target p(Theta | X, t) exactly).  The test
checks (i) the two posteriors agree within Monte Carlo error, and (ii) what
the network gains: exact-kernel evaluations per effective sample."""
import numpy as np
import pytest

from paper_2407_11349_gb300 import diagnostics as dg
from paper_2407_11349_gb300 import hmc, synth
from paper_2407_11349_gb300.hawkes import MLP

pytestmark = pytest.mark.gpu


def test_surrogate_hmc_matches_exact_and_saves_exact_evaluations():
    pytest.importorskip("torch")
    ds = synth.clustered_dataset(5000, seed=41)
    C, L = 4, 10
    eta0 = np.log(synth.DEFAULT_PARAMS)
    tgt = hmc.HawkesTarget(ds, C, seed=5)
    try:
        init = np.tile(eta0, (C, 1)) + np.random.default_rng(0).normal(0, 0.01, (C, 6))
        ex = hmc.Sampler(tgt, hmc.Prior(eta0), init, n_leapfrog=L, seed=1, cut=False)
        ex.record = []
        last = ex.warmup(400)
        assert len(ex.record) == 1 + 400 * (L + 1)  # initial scale evaluation + warmup
        # train on the evaluations from the last slow adaptation window on
        X, Y = hmc.training_set(ex.record[1 + last * (L + 1):])
        ex.record = None
        assert X.shape[0] > 0.9 * C * (400 - last) * (L + 1)

        net = MLP(0, seed=2)
        net.set_data(X, Y)
        loss = net.train(4000, batch=256, lr=1e-3, seed=3)
        assert loss < 0.01
        field = hmc.SurrogateField(net, C)

        n0 = tgt.n_exact
        d_ex, acc_ex, _ = ex.sample(600)
        exact_evals_ex = tgt.n_exact - n0

        su = hmc.Sampler(tgt, hmc.Prior(eta0), ex.q.copy(), n_leapfrog=L, seed=4, cut=False)
        su.eps = ex.eps.copy()
        su.set_cov(ex.cov)
        n0 = tgt.n_exact
        d_su, acc_su, _ = su.sample(600, field)
        exact_evals_su = tgt.n_exact - n0

        s_ex = dg.summary(d_ex, hmc.NAMES)
        s_su = dg.summary(d_su, hmc.NAMES)
        for nm in hmc.NAMES:
            diff = abs(s_ex[nm]["mean"] - s_su[nm]["mean"])
            se = np.hypot(s_ex[nm]["mcse"], s_su[nm]["mcse"])
            assert diff < 4.5 * se, (nm, s_ex[nm], s_su[nm])
        assert acc_su.mean() > 0.6
        ess_ex = min(s_ex[nm]["bulk_ess"] for nm in hmc.NAMES)
        ess_su = min(s_su[nm]["bulk_ess"] for nm in hmc.NAMES)
        # exact-kernel evaluations per effective sample: the network's gain
        assert exact_evals_su / ess_su < 0.5 * exact_evals_ex / ess_ex

        # the anchored field (shifted by the exact minus the network's gradient
        # at a fixed point) targets the same posterior
        sa = hmc.Sampler(tgt, hmc.Prior(eta0), ex.q.copy(), n_leapfrog=L, seed=6, cut=False)
        sa.eps = ex.eps.copy()
        sa.set_cov(ex.cov)
        n0 = tgt.n_exact
        d_sa, acc_sa, _ = sa.sample(600, field, anchor=np.median(X, axis=0))
        assert tgt.n_exact - n0 == 600 * 3 * C
        s_sa = dg.summary(d_sa, hmc.NAMES)
        for nm in hmc.NAMES:
            diff = abs(s_ex[nm]["mean"] - s_sa[nm]["mean"])
            se = np.hypot(s_ex[nm]["mcse"], s_sa[nm]["mcse"])
            assert diff < 4.5 * se, (nm, s_ex[nm], s_sa[nm])
        assert acc_sa.mean() > 0.6
        net.close()
    finally:
        tgt.close()


def test_cut_scheme_feature_surrogate_and_loglik_only_target():
    """Under the cut scheme: the warmup records each location draw's feature
    (the exact log-likelihood at a fixed anchor under that draw); a network
    trained with it as its seventh input drives surrogate HMC with the
    feature of each new draw, costing three exact evaluations per iteration
    (anchor, start, end).  The target's log-likelihood-only evaluations give
    the full ones' values (the univariate MH sampler uses them)."""
    pytest.importorskip("torch")
    ds = synth.clustered_dataset(4000, seed=43)
    C, L = 4, 8
    eta0 = np.log(synth.DEFAULT_PARAMS)
    tgt = hmc.HawkesTarget(ds, C, seed=6)
    try:
        init = np.tile(eta0, (C, 1)) + np.random.default_rng(1).normal(0, 0.01, (C, 6))
        ex = hmc.Sampler(tgt, hmc.Prior(eta0), init, n_leapfrog=L, seed=2, cut=True)
        ex.record = []
        last = ex.warmup(200, feature_anchor=eta0)
        X, Y, F = hmc.training_set(ex.record[1 + last * (L + 1):], with_feature=True)
        assert X.shape[0] == F.shape[0] > 0.8 * C * (200 - last) * (L + 1) and np.all(np.isfinite(F))
        net = MLP(0, seed=4)
        try:
            net.set_data(X, Y, F)
            net.train(2000, batch=256, lr=1e-3, seed=5)
            field = hmc.SurrogateField(net, C, feature=True)
            smp = hmc.Sampler(tgt, hmc.Prior(eta0), ex.q, n_leapfrog=L, seed=7, cut=True)
            smp.eps, smp.iteration = ex.eps.copy(), ex.iteration
            smp.set_cov(ex.cov)
            n0 = tgt.n_exact
            d, acc, _ = smp.sample(50, field=field, feature_anchor=eta0)
            assert tgt.n_exact - n0 == 50 * C * 3
            assert np.all(np.isfinite(d)) and acc.mean() > 0.05
        finally:
            net.close()
        q = ex.q.copy()
        ll_full, _ = tgt.eval(q)
        ll_only, g = tgt.eval_loglik(q)
        assert np.all(np.abs(ll_only - ll_full) <= 1e-7 * np.abs(ll_full)) and np.all(np.isnan(g))
    finally:
        tgt.close()
