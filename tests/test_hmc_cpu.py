"""HMC drivers and diagnostics on the host, against closed forms (no GPU).

Targets here are Gaussians whose posterior (likelihood x Normal(eta0, 2^2)
prior x Jacobian e^{sum eta}) is Gaussian in closed form, so the samplers'
means and variances can be judged within Monte Carlo error; the surrogate is
deliberately biased, and the exact accept step must still remove the bias.
"""
import numpy as np
import pytest

from paper_2407_11349_gb300 import diagnostics as dg
from paper_2407_11349_gb300 import hmc


def ar1(rho, chains, n, seed):
    rng = np.random.default_rng(seed)
    x = np.zeros((chains, n))
    e = rng.standard_normal((chains, n)) * np.sqrt(1 - rho ** 2)
    x[:, 0] = rng.standard_normal(chains)
    for t in range(1, n):
        x[:, t] = rho * x[:, t - 1] + e[:, t]
    return x


@pytest.mark.parametrize("rho", [0.0, 0.5, 0.9])
def test_ess_matches_ar1_closed_form(rho):
    x = ar1(rho, 4, 20000, seed=int(10 * rho))
    expect = x.size * (1 - rho) / (1 + rho)
    got = dg.ess(x)
    assert abs(got / expect - 1) < 0.1, (got, expect)
    assert abs(dg.bulk_ess(x) / expect - 1) < 0.12


def test_rhat_detects_shifted_chains():
    x = ar1(0.3, 4, 4000, seed=3)
    assert dg.rhat(x) < 1.01
    y = x.copy()
    y[0] += 1.0
    assert dg.rhat(y) > 1.05
    assert dg.tail_ess(x) > 1000


class GaussTarget:
    """log-likelihood -1/2 sum ((eta - m)/s)^2, no dependence on locations."""

    def __init__(self, m, s, C):
        self.m, self.s, self.C = np.asarray(m), np.asarray(s), C
        self.n_exact = 0

    def eval(self, eta):
        self.n_exact += eta.shape[0]
        d = (eta - self.m) / self.s
        return -0.5 * np.sum(d * d, axis=1), -d / self.s

    def resample_eval(self, iteration, eta):
        return self.eval(eta)


def posterior(m, s, eta0, sd=hmc.PRIOR_SD):
    prec = 1 / s ** 2 + 1 / sd ** 2
    return (m / s ** 2 + eta0 / sd ** 2 + 1.0) / prec, 1 / prec


M = np.array([0.3, -1.0, 2.0, 0.0, 1.5, -0.5])
S = np.array([0.1, 0.3, 0.05, 0.2, 0.5, 0.15])
ETA0 = np.zeros(6)


def _run(field, seed, n=1500):
    """Warmup with exact gradients (as the pipeline does), then sample with
    ``field`` driving the trajectories."""
    C = 4
    tgt = GaussTarget(M, S, C)
    smp = hmc.Sampler(tgt, hmc.Prior(ETA0), np.tile(M, (C, 1)) + 0.01, n_leapfrog=8, seed=seed)
    smp.warmup(300)
    draws, acc, _ = smp.sample(n, field)
    return draws, acc, tgt


def _check_posterior(draws, rhat_max=1.05):
    mean, var = posterior(M, S, ETA0)
    summ = dg.summary(draws, hmc.NAMES)
    for k, nm in enumerate(hmc.NAMES):
        x = draws[:, :, k]
        assert abs(x.mean() - mean[k]) < 4.5 * summ[nm]["mcse"], (nm, x.mean(), mean[k])
        assert abs(x.var() / var[k] - 1) < 0.25, (nm, x.var(), var[k])
        assert summ[nm]["rhat"] < rhat_max


def test_exact_hmc_recovers_gaussian_posterior():
    draws, acc, tgt = _run(None, seed=1)
    assert acc.mean() > 0.6
    _check_posterior(draws)


def test_surrogate_hmc_with_biased_field_is_still_exact():
    # the surrogate's gradient points at the wrong mean with the wrong scale
    def field(eta):
        d = (eta - (M + 0.3 * S)) / (1.3 * S)
        return None, -d / (1.3 * S)

    draws, acc, tgt = _run(field, seed=2, n=3000)
    assert 0.05 < acc.mean() < 0.99
    # exactness: means within Monte Carlo error and variances right, although
    # the trajectories follow the wrong field (mixing is slower: looser R-hat)
    _check_posterior(draws, rhat_max=1.1)


def test_checkpoint_resume_is_bit_identical(tmp_path):
    C = 2
    t1 = GaussTarget(M, S, C)
    a = hmc.Sampler(t1, hmc.Prior(ETA0), np.tile(M, (C, 1)), n_leapfrog=5, seed=9)
    a.warmup(40)
    for _ in range(10):
        a.transition()
    path = tmp_path / "ck.npz"
    hmc.save(path, a)
    ref = [a.transition().copy() for _ in range(15)]
    ref_q = a.q.copy()
    t2 = GaussTarget(M, S, C)
    b = hmc.Sampler(t2, hmc.Prior(ETA0), np.zeros((C, 6)), n_leapfrog=1, seed=0)
    hmc.load(path, b)
    got = [b.transition().copy() for _ in range(15)]
    assert np.array_equal(np.stack(ref), np.stack(got))
    assert np.array_equal(ref_q, b.q)


def test_univariate_mh_recovers_gaussian_posterior():
    C = 4
    tgt = GaussTarget(M, S, C)
    mh = hmc.MHSampler(tgt, hmc.Prior(ETA0), np.tile(M, (C, 1)), seed=3)
    mh.warmup(500)
    draws, acc, _ = mh.sample(4000)
    assert 0.25 < acc.mean() < 0.6
    mean, var = posterior(M, S, ETA0)
    summ = dg.summary(draws, hmc.NAMES)
    for k, nm in enumerate(hmc.NAMES):
        x = draws[:, :, k]
        assert abs(x.mean() - mean[k]) < 4.5 * summ[nm]["mcse"], (nm, x.mean(), mean[k])
        assert abs(x.var() / var[k] - 1) < 0.3


def test_anchored_surrogate_removes_a_slope_error_and_stays_exact():
    """A surrogate whose gradient is off by a constant (what a change of the
    locations does to the slope) is made exact by the anchor shift:
    acceptance returns to the exact-HMC level and the posterior is right."""
    bias = 3.0 / S

    def field(eta):
        return None, -(eta - M) / S ** 2 + bias

    draws0, acc0, _ = _run(field, seed=4, n=1500)
    C = 4
    tgt = GaussTarget(M, S, C)
    smp = hmc.Sampler(tgt, hmc.Prior(ETA0), np.tile(M, (C, 1)) + 0.01, n_leapfrog=8, seed=4)
    smp.warmup(300)
    n0 = tgt.n_exact
    draws, acc, _ = smp.sample(1500, field, anchor=M + 0.5 * S)
    assert tgt.n_exact - n0 == 1500 * 3 * C  # start, anchor, end
    ex, acc_ex, _ = _run(None, seed=4, n=300)
    assert acc.mean() > acc0.mean() + 0.1
    assert abs(acc.mean() - acc_ex.mean()) < 0.05
    _check_posterior(draws)


class CutGaussTarget(GaussTarget):
    """Each location draw adds a random slope x . eta / s to the
    log-likelihood (x ~ N(0, 0.5^2) per chain and iteration)."""

    def __init__(self, m, s, C, seed=0):
        super().__init__(m, s, C)
        self.rng = np.random.default_rng(seed)
        self.x = np.zeros((C, 6))

    def eval(self, eta):
        ll, g = super().eval(eta)
        return ll + np.sum(self.x * eta / self.s, axis=1), g + self.x / self.s

    def resample_eval(self, iteration, eta):
        self.x = 0.5 * self.rng.standard_normal((self.C, 6))
        return self.eval(eta)


def test_anchored_surrogate_raises_acceptance_under_the_cut_scheme():
    def field(eta):  # the draw-averaged surface
        return None, -(eta - M) / S ** 2

    acc = {}
    for anchored in (False, True):
        C = 4
        tgt = CutGaussTarget(M, S, C, seed=5)
        smp = hmc.Sampler(tgt, hmc.Prior(ETA0), np.tile(M, (C, 1)) + 0.01, n_leapfrog=8, seed=5)
        smp.warmup(300)
        _, a, _ = smp.sample(600, field, anchor=M if anchored else None)
        acc[anchored] = a.mean()
    assert acc[True] > acc[False] + 0.1, acc


def test_several_moves_per_location_draw_stay_exact_and_cost_one_evaluation_each():
    """moves=3: three surrogate HMC moves under each location draw; each
    further move starts from the exact value of the state the last one left,
    so an iteration costs 1 + 3 exact evaluations, and the posterior is
    unchanged."""
    def field(eta):  # biased surrogate, as above
        d = (eta - (M + 0.3 * S)) / (1.3 * S)
        return None, -d / (1.3 * S)

    C = 4
    tgt = GaussTarget(M, S, C)
    smp = hmc.Sampler(tgt, hmc.Prior(ETA0), np.tile(M, (C, 1)) + 0.01, n_leapfrog=8, seed=8)
    smp.warmup(300)
    n0 = tgt.n_exact
    draws, acc, _ = smp.sample(1500, field, moves=3)
    assert tgt.n_exact - n0 == 1500 * (1 + 3) * C
    assert 0.05 < acc.mean() < 0.99
    _check_posterior(draws, rhat_max=1.1)


def test_cut_posterior_reference_matches_the_mixture_in_closed_form():
    """Exact HMC under each of many location draws, pooled, is the cut
    posterior: for the random-slope toy, a Gaussian mixture whose mean is the
    fixed-X posterior mean and whose variance adds Var(x / s) / P^2."""
    C = 4
    tgt = CutGaussTarget(M, S, C, seed=9)
    prior = hmc.Prior(ETA0)
    smp = hmc.Sampler(tgt, prior, np.tile(M, (C, 1)) + 0.01, n_leapfrog=8, seed=9, cut=False)
    smp.warmup(200)
    d = hmc.cut_posterior_reference(tgt, prior, smp.q.copy(), smp.cov, smp.eps, rounds=40, burn=20,
                                    draws=60, n_leapfrog=8, seed=3)
    assert d.shape == (C * 40, 60, 6)
    P = 1 / S ** 2 + 1 / hmc.PRIOR_SD ** 2
    mean = (M / S ** 2 + ETA0 / hmc.PRIOR_SD ** 2 + 1.0) / P
    var = 1 / P + 0.25 / (S ** 2 * P ** 2)
    m_cr = d.mean(axis=1)
    se = m_cr.std(axis=0, ddof=1) / np.sqrt(m_cr.shape[0])
    assert np.all(np.abs(m_cr.mean(axis=0) - mean) < 4.5 * se), (m_cr.mean(axis=0), mean, se)
    pooled = d.reshape(-1, 6).var(axis=0)
    assert np.all(np.abs(pooled / var - 1) < 0.25), (pooled, var)


def test_mh_checkpoint_resume_is_bit_identical(tmp_path):
    C = 3
    a = hmc.MHSampler(GaussTarget(M, S, C), hmc.Prior(ETA0), np.tile(M, (C, 1)), seed=11)
    a.warmup(30)
    path = tmp_path / "mh.npz"
    hmc.save(path, a)
    ref = [a.transition().copy() for _ in range(12)]
    b = hmc.MHSampler(GaussTarget(M, S, C), hmc.Prior(ETA0), np.zeros((C, 6)), seed=0)
    hmc.load(path, b)
    got = [b.transition().copy() for _ in range(12)]
    assert np.array_equal(np.stack(ref), np.stack(got)) and np.array_equal(a.q, b.q)


def test_mh_checkpoint_during_warmup_resumes_the_adaptation(tmp_path):
    """A run checkpointed partway through warmup, resumed into a sampler
    built with a different cut setting, continues exactly as the
    uninterrupted run (adaptation schedule, cut setting and RNG restored)."""
    C = 3
    a = hmc.MHSampler(GaussTarget(M, S, C), hmc.Prior(ETA0), np.tile(M, (C, 1)), seed=11)
    a.warmup(12)
    path = tmp_path / "mh_warm.npz"
    hmc.save(path, a)
    a.warmup(18)
    ref = [a.transition().copy() for _ in range(6)]
    b = hmc.MHSampler(GaussTarget(M, S, C), hmc.Prior(ETA0), np.zeros((C, 6)), seed=0, cut=False)
    hmc.load(path, b)
    assert b.cut is True and b.warm_k == 12
    b.warmup(18)
    got = [b.transition().copy() for _ in range(6)]
    assert np.array_equal(a.log_scale, b.log_scale)
    assert np.array_equal(np.stack(ref), np.stack(got)) and np.array_equal(a.q, b.q)


def test_mh_checkpoint_rejects_a_surrogate(tmp_path):
    C = 2
    a = hmc.MHSampler(GaussTarget(M, S, C), hmc.Prior(ETA0), np.tile(M, (C, 1)), seed=1)
    with pytest.raises(ValueError):
        hmc.save(tmp_path / "x.npz", a, mlp=object())
    hmc.save(tmp_path / "y.npz", a)
    with pytest.raises(ValueError):
        hmc.load(tmp_path / "y.npz", a, mlp=object())


def test_mh_uses_the_loglik_only_evaluations_when_offered():
    """A target with eval_loglik / resample_eval_loglik: the MH sampler calls
    only those (it needs no gradient)."""
    class LLOnly(GaussTarget):
        def __init__(self, *a):
            super().__init__(*a)
            self.full_calls = 0

        def eval(self, eta):
            self.full_calls += 1
            return super().eval(eta)

        def resample_eval(self, it, eta):
            self.full_calls += 1
            return super().resample_eval(it, eta)

        def eval_loglik(self, eta):
            ll, g = GaussTarget.eval(self, eta)
            return ll, np.full_like(g, np.nan)

        def resample_eval_loglik(self, it, eta):
            ll, g = GaussTarget.eval(self, eta)
            return ll, np.full_like(g, np.nan)

    C = 2
    t = LLOnly(M, S, C)
    a = hmc.MHSampler(t, hmc.Prior(ETA0), np.tile(M, (C, 1)), seed=3)
    a.warmup(5)
    a.sample(5)
    assert t.full_calls == 0


class SlopeDrawTarget(GaussTarget):
    """Each location draw adds u (w . eta) to the log-likelihood, one scalar
    u ~ N(0, 1.5^2) per chain and draw along a fixed direction w: the
    draw-to-draw change of the surface has one degree of freedom."""

    W = np.array([1.0, -0.5, 0.8, 0.3, -1.0, 0.6]) / 3.0

    def __init__(self, m, s, C, seed=0):
        super().__init__(m, s, C)
        self.rng = np.random.default_rng(seed)
        self.u = np.zeros(C)

    def eval(self, eta):
        ll, g = super().eval(eta)
        return ll + self.u * (eta @ (self.W / S)), g + self.u[:, None] * (self.W / S)

    def resample_eval(self, iteration, eta):
        self.u = 1.5 * self.rng.standard_normal(self.C)
        return self.eval(eta)


class FeatureField:
    """A surrogate that reads the draw from z = ell(a; X): here it knows the
    surface's form, so the feature recovers u exactly."""

    def __init__(self, anchor):
        self.a = anchor
        self.u = 0.0

    def set_feature(self, z):
        base = -0.5 * np.sum(((self.a - M) / S) ** 2)
        self.u = (np.asarray(z) - base) / (self.a @ (SlopeDrawTarget.W / S))

    def __call__(self, eta):
        return None, -(eta - M) / S ** 2 + np.asarray(self.u)[:, None] * (SlopeDrawTarget.W / S)


def test_draw_feature_raises_acceptance_under_the_cut_scheme_and_stays_exact():
    """With the exact log-likelihood at a fixed anchor under each draw as the
    field's input, the field follows the draw-to-draw change and acceptance
    rises; the chains still sample the cut posterior (mean unchanged: the
    slopes average out)."""
    def plain(eta):  # the draw-averaged surface
        return None, -(eta - M) / S ** 2

    C = 4
    acc, means = {}, {}
    for name in ("plain", "feature"):
        tgt = SlopeDrawTarget(M, S, C, seed=21)
        smp = hmc.Sampler(tgt, hmc.Prior(ETA0), np.tile(M, (C, 1)) + 0.01, n_leapfrog=8, seed=22)
        smp.warmup(300)
        a_pt = M + 0.5 * S
        if name == "plain":
            d, a, _ = smp.sample(1500, plain)
        else:
            n0 = tgt.n_exact
            d, a, _ = smp.sample(1500, FeatureField(a_pt), feature_anchor=a_pt)
            assert tgt.n_exact - n0 == 1500 * C * 3  # anchor, start, end per iteration
        acc[name], means[name] = a.mean(), d.reshape(-1, 6).mean(axis=0)
        mu_post, var_post = posterior(M, S, ETA0)
        assert np.all(np.abs(means[name] - mu_post) < 0.15 * S), (name, means[name], mu_post)
    assert acc["feature"] > acc["plain"] + 0.1, acc


def test_training_set_with_feature():
    rec = [(np.zeros((2, 6)) + k, np.array([1.0, 2.0]) + k, np.ones((2, 6)), np.array([5.0, 6.0]) + k)
           for k in range(5)] + [(np.zeros((2, 6)), np.zeros(2), np.ones((2, 6)), None)]
    X, Y, F = hmc.training_set(rec, with_feature=True)
    assert X.shape == (10, 6) and Y.shape == (10, 7) and F.shape == (10,)
    assert np.array_equal(F[:2], [5.0, 6.0])
    X2, Y2 = hmc.training_set(rec)
    assert X2.shape[0] == 12
