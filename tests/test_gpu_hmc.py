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
