"""Hamiltonian Monte Carlo on the cut posterior (Sec. 2.2), exact and
surrogate-driven.

The cut posterior is sampled by alternating (i) a fresh draw of every event
location uniformly in its county, and (ii) a transition that leaves
p(Theta | X, t) invariant.  The paper uses univariate Metropolis-Hastings for
(ii); here it is HMC on eta = log(mu, tau_x, tau_t, theta, omega, h) with
independent Normal(eta0, 2^2) priors (our choice; the paper does not state
its priors) plus the log-transform Jacobian.

Exact HMC evaluates the exact gradient at every leapfrog step.  Surrogate HMC
runs the whole leapfrog trajectory on a neural-network approximation of the
gradient (any fixed vector field gives a reversible, volume-preserving map)
and accepts with the EXACT Hamiltonian at both ends under the current X, so
the chain still targets p(Theta | X, t); a poor surrogate costs acceptance,
not correctness.

Anchored surrogate (cut posterior).  The network sees only Theta, so it
predicts the likelihood surface averaged over location draws, while the
exact surface moves with every draw of X.  With an anchor point a (fixed
for the whole run, e.g. a warmup estimate of the posterior mean), each
iteration evaluates the exact gradient at a under the freshly drawn X and
adds the constant c = grad_exact(a; X) - grad_net(a) to the network's
field for that iteration's trajectory.  c depends on X and a only, never on
the chain's state, so the field is still a fixed conservative field during
the trajectory and the exact accept step keeps p(Theta | X, t) invariant;
the shift removes the part of the X-dependence that is locally a change of
slope.  Cost: one more exact evaluation per iteration (3 instead of 2).

Draw feature (cut posterior).  Instead of a shift, the network can be told
about the draw: its seventh input is z = ell_exact(a; X), the exact
log-likelihood at a fixed anchor a under the iteration's locations (one more
exact evaluation per iteration), and it is trained on (eta, z) -> (ell,
grad) pairs recorded with their draw's z.  z depends on X and a only, so the
field is again fixed for the whole trajectory and the exact accept step
keeps p(Theta | X, t) invariant.

Chains advance in lockstep: the exact evaluations of all chains are one
batched launch (``Batch``), the surrogate's predictions one network call.
Step size: dual averaging (Hoffman and Gelman 2014); metric: a dense
covariance estimate from windows of warmup draws.  Checkpoints (``save``/``load``) hold every piece of
state, so a resumed run continues bit for bit.
"""
import time

import numpy as np

NAMES = ("mu", "tau_x", "tau_t", "theta", "omega", "h")
PRIOR_SD = 2.0
ETA_MAX = 30.0  # |log p| beyond this is treated as a divergent trajectory


class Prior:
    """Independent Normal(eta0, sd^2) on eta = log p, plus the Jacobian sum(eta)."""

    def __init__(self, eta0, sd=PRIOR_SD):
        self.eta0 = np.asarray(eta0, dtype=np.float64)
        self.sd = float(sd)

    def __call__(self, eta):
        d = (eta - self.eta0) / self.sd
        lp = -0.5 * np.sum(d * d, axis=-1) + np.sum(eta, axis=-1)
        g = -d / self.sd + 1.0
        return lp, g


class HawkesTarget:
    """Exact log-likelihood and gradient for C chains on one GPU.

    Each chain owns a context with the same events and its own resample
    stream; ``resample_eval`` draws new locations for every chain and then
    evaluates (one captured graph), ``eval`` evaluates at fixed locations.
    Returns the log-likelihood and its gradient in eta = log p.  ``flags``:
    extra batch flags (model options, the exact underflow skip).
    """

    def __init__(self, ds, n_chains, seed=0, device=0, flags=0):
        import torch

        from .hawkes import HAWKES_F32, HAWKES_SKIP_SPATIAL, Batch, Hawkes, HawkesError

        self.torch = torch
        self.HawkesError = HawkesError
        self.n_failed = 0
        self.C = n_chains
        self.stream = torch.cuda.Stream(device=device)
        s = self.stream.cuda_stream
        self.hks = [Hawkes(device, s).load(ds) for _ in range(n_chains)]
        self.dp = torch.zeros((n_chains, 6), dtype=torch.float64, device=f"cuda:{device}")
        self.dout = torch.zeros((n_chains, 7), dtype=torch.float64, device=f"cuda:{device}")
        self.host = torch.zeros((n_chains, 7), dtype=torch.float64).pin_memory()
        self.flags = HAWKES_F32 | flags
        self.seed = seed
        # the spatial skip runs on single contexts: evaluate chain by chain
        self.sequential = bool(flags & HAWKES_SKIP_SPATIAL)
        if not self.sequential:
            self.b_rs = Batch(self.hks, [seed] * n_chains, list(range(n_chains)), self.flags, s)
            self.b_ev = Batch(self.hks, None, None, self.flags, s)
            self.b_rs.capture(self.dp.data_ptr(), self.dout.data_ptr())
            self.b_ev.capture(self.dp.data_ptr(), self.dout.data_ptr())
        self.b_ll = None
        self.n_exact = 0
        self.n_events = ds.n

    def _run(self, batch, eta, iteration):
        torch = self.torch
        p = np.exp(np.asarray(eta, dtype=np.float64))
        with torch.cuda.stream(self.stream):
            self.dp.copy_(torch.from_numpy(p), non_blocking=False)
        self.stream.synchronize()
        batch.run(self.dp.data_ptr(), iteration, self.dout.data_ptr())
        try:
            batch.wait()
        except self.HawkesError:
            # a problem with unusable parameters or a non-finite result: its
            # outputs are NaN and the sampler rejects that chain's move
            self.n_failed += 1
        with torch.cuda.stream(self.stream):
            self.host.copy_(self.dout)
        self.stream.synchronize()
        out = self.host.numpy().copy()
        self.n_exact += self.C
        return out[:, 0], out[:, 1:] * p

    def _run_sequential(self, eta, iteration, resample, loglik_only=False):
        from .hawkes import HAWKES_LOGLIK_ONLY
        p = np.exp(np.asarray(eta, dtype=np.float64))
        out = np.full((self.C, 7), np.nan)
        fl = self.flags | (HAWKES_LOGLIK_ONLY if loglik_only else 0)
        for c, h in enumerate(self.hks):
            try:
                if resample:
                    h.resample(self.seed, c, iteration)
                ll, g = h.loglik_grad(p[c], fl)
                out[c, 0], out[c, 1:] = ll, g
            except self.HawkesError:
                self.n_failed += 1
        self.n_exact += self.C
        return out[:, 0], out[:, 1:] * p

    def resample_eval(self, iteration, eta):
        if self.sequential:
            return self._run_sequential(eta, iteration, True)
        return self._run(self.b_rs, eta, iteration)

    def eval(self, eta):
        if self.sequential:
            return self._run_sequential(eta, 0, False)
        return self._run(self.b_ev, eta, 0)

    def _ll_batches(self):
        """Batches with the log-likelihood-only flag (built on first use)."""
        if self.b_ll is None:
            from .hawkes import HAWKES_LOGLIK_ONLY, Batch
            s = self.stream.cuda_stream
            fl = self.flags | HAWKES_LOGLIK_ONLY
            self.b_ll = (Batch(self.hks, [self.seed] * self.C, list(range(self.C)), fl, s),
                         Batch(self.hks, None, None, fl, s))
            for b in self.b_ll:
                b.capture(self.dp.data_ptr(), self.dout.data_ptr())
        return self.b_ll

    def resample_eval_loglik(self, iteration, eta):
        """As resample_eval, log-likelihood only (its gradient is NaN): the
        sweep forms two moment sums per row instead of six."""
        if self.sequential:
            return self._run_sequential(eta, iteration, True, loglik_only=True)
        return self._run(self._ll_batches()[0], eta, iteration)

    def eval_loglik(self, eta):
        if self.sequential:
            return self._run_sequential(eta, 0, False, loglik_only=True)
        return self._run(self._ll_batches()[1], eta, 0)

    def close(self):
        if not self.sequential:
            self.b_rs.close()
            self.b_ev.close()
        if self.b_ll is not None:
            for b in self.b_ll:
                b.close()
        for h in self.hks:
            h.close()


class SurrogateField:
    """The network's (log-likelihood, eta-gradient) prediction for C chains.
    feature=True: the network was trained with a seventh-input feature, and
    ``set_feature`` gives each chain's value for the coming trajectory."""

    def __init__(self, mlp, n_chains, device=0, feature=False):
        import torch

        self.torch = torch
        self.mlp = mlp
        self.C = n_chains
        self.dq = torch.zeros((n_chains, 6), dtype=torch.float64, device=f"cuda:{device}")
        self.dout = torch.zeros((n_chains, 7), dtype=torch.float64, device=f"cuda:{device}")
        self.df = torch.zeros(n_chains, dtype=torch.float64, device=f"cuda:{device}") if feature else None
        self.n_calls = 0

    def set_feature(self, z):
        self.df.copy_(self.torch.from_numpy(np.asarray(z, dtype=np.float64)))

    def __call__(self, eta):
        torch = self.torch
        self.dq.copy_(torch.from_numpy(np.asarray(eta, dtype=np.float64)))
        torch.cuda.synchronize()
        self.mlp.predict(self.dq.data_ptr(), self.C, self.dout.data_ptr(),
                         0 if self.df is None else self.df.data_ptr())
        self.mlp.wait()
        out = self.dout.cpu().numpy()
        self.n_calls += 1
        return out[:, 0], out[:, 1:]


class DualAveraging:
    """Step-size adaptation of Hoffman and Gelman (2014), per chain."""

    def __init__(self, eps0, delta=0.8, gamma=0.05, t0=10.0, kappa=0.75):
        self.mu = np.log(10.0 * eps0)
        self.delta, self.gamma, self.t0, self.kappa = delta, gamma, t0, kappa
        self.hbar = np.zeros_like(eps0)
        self.logeps_bar = np.zeros_like(eps0)
        self.t = 0
        self.logeps = np.log(eps0)

    def update(self, accept_stat):
        self.t += 1
        w = 1.0 / (self.t + self.t0)
        self.hbar = (1 - w) * self.hbar + w * (self.delta - accept_stat)
        self.logeps = self.mu - np.sqrt(self.t) / self.gamma * self.hbar
        eta = self.t ** (-self.kappa)
        self.logeps_bar = eta * self.logeps + (1 - eta) * self.logeps_bar
        return np.exp(self.logeps)

    def final(self):
        return np.exp(self.logeps_bar)


class Sampler:
    """Lockstep HMC for C chains on the cut posterior.

    target:  object with resample_eval(iteration, eta) and eval(eta), each
             returning (loglik[C], grad_eta[C, 6])
    prior:   Prior
    """

    def __init__(self, target, prior, eta_init, n_leapfrog=10, seed=0, jitter=0.2, cut=True):
        self.target = target
        self.cut = bool(cut)  # False: keep the locations fixed (samples p(Theta | X, t) for one X)
        self.prior = prior
        self.q = np.array(eta_init, dtype=np.float64, copy=True)
        self.C = self.q.shape[0]
        self.L = int(n_leapfrog)
        self.eps = np.full(self.C, 0.05)
        self.cov = np.tile(np.eye(6), (self.C, 1, 1))  # metric: inverse mass (posterior covariance estimate)
        self.chol = np.linalg.cholesky(self.cov)
        self.rng = np.random.default_rng(seed)
        self.jitter = float(jitter)  # step size drawn from eps * U(1 - jitter, 1 + jitter)
        self.iteration = 0
        self.divergent = 0
        # list of (eta, loglik, grad, z) exact evaluations, when collecting; z
        # is the draw feature of the evaluation's locations (None without one)
        self.record = None
        self.z = None

    def _exact(self, eta, resample=False):
        if resample:
            ll, g = self.target.resample_eval(self.iteration, eta)
        else:
            ll, g = self.target.eval(eta)
        if self.record is not None:
            self.record.append((eta.copy(), ll.copy(), g.copy(), None if self.z is None else self.z.copy()))
        lp, gp = self.prior(eta)
        return ll + lp, g + gp

    def _init_scale(self):
        """Initial inverse mass from the gradient at the starting point: a
        component whose log-density changes by g per unit starts with a
        scale ~ 1/|g| (the posterior in eta is very narrow at large N)."""
        _, g = self._exact(self.q, resample=self.cut)
        self.set_cov(np.stack([np.diag(np.clip(1.0 / (gc * gc + 1e-12), 1e-12, 1.0)) for gc in g]))
        self.eps = np.full(self.C, 0.1)

    def set_cov(self, cov):
        self.cov = np.array(cov, dtype=np.float64)
        self.chol = np.linalg.cholesky(self.cov)

    def _momentum(self):
        # p ~ N(0, cov^-1): p = L^-T z with cov = L L^T
        z = self.rng.standard_normal((self.C, 6))
        return np.stack([np.linalg.solve(self.chol[c].T, z[c]) for c in range(self.C)])

    def _kinetic(self, p):
        return 0.5 * np.einsum("ci,cij,cj->c", p, self.cov, p)

    def _velocity(self, p):
        return np.einsum("cij,cj->ci", self.cov, p)

    def transition(self, field=None, anchor=None, moves=1, feature_anchor=None):
        """One cut-posterior iteration: new locations, then `moves` HMC moves
        under them (the paper's scheme has one).  field(eta) -> (loglik, grad)
        drives the trajectories (None: exact).  anchor (6,) or (C, 6), with a
        field: shift the field by the exact minus the field's gradient at the
        anchor under this iteration's locations (see the module notes).
        feature_anchor (6,) or (C, 6): evaluate the exact log-likelihood there
        under the new locations as this iteration's draw feature z (recorded
        with the exact evaluations, and given to a field that takes one).
        Every move under the same locations starts from the exact value of
        the state the previous move left, so a further surrogate move costs
        one exact evaluation.  A trajectory that leaves |eta| <= ETA_MAX or
        turns non-finite is divergent: it is rejected (its exact evaluations
        use the current state instead).  Returns the acceptance probability
        of each chain, averaged over the moves."""
        self.iteration += 1
        self.z = None
        if feature_anchor is not None:
            # the new locations, evaluated first at the anchor: this draw's feature
            f_pt = np.array(np.broadcast_to(feature_anchor, self.q.shape), dtype=np.float64)
            if self.cut:
                self.z = self.target.resample_eval(self.iteration, f_pt)[0]
            else:
                self.z = self.target.eval(f_pt)[0]
            if field is not None:
                field.set_feature(self.z)
            lp0, g0 = self._exact(self.q)
        else:
            lp0, g0 = self._exact(self.q, resample=self.cut)
        shift = 0.0
        if field is not None and anchor is not None:
            a_pt = np.array(np.broadcast_to(anchor, self.q.shape), dtype=np.float64)
            _, g_a = self.target.eval(a_pt)  # exact, under the locations just drawn
            shift = g_a - field(a_pt)[1]
            shift = np.where(np.isfinite(shift), shift, 0.0)
        acc = np.zeros(self.C)
        self.divergent = 0
        for _ in range(int(moves)):
            a, lp0, g0 = self._move(lp0, g0, field, shift)
            acc += a
        return acc / int(moves)

    def _move(self, lp0, g0, field, shift):
        """One HMC move from self.q, whose exact log-posterior and gradient
        are (lp0, g0) under the current locations.  Returns the acceptance
        probability and the exact (log-posterior, gradient) of the new state
        (the gradient is None where a surrogate move was accepted; it is only
        needed to start exact trajectories)."""
        p0 = self._momentum()
        # a random step size per move (independent of the state) avoids
        # trajectories that return to their start on near-Gaussian targets
        eps = (self.eps * (1.0 + self.jitter * (2.0 * self.rng.random(self.C) - 1.0)))[:, None]
        bad = np.zeros(self.C, dtype=bool)

        def safe(q):
            nonlocal bad
            bad |= ~np.all(np.isfinite(q) & (np.abs(q) <= ETA_MAX), axis=1)
            return np.where(bad[:, None], self.q, q)

        def grad(q):
            if field is None:
                lp, g = self._exact(safe(q))
            else:
                lp, g = None, field(safe(q))[1] + shift + self.prior(safe(q))[1]
            bad[:] |= ~np.all(np.isfinite(g), axis=1)
            return lp, np.where(bad[:, None], 0.0, g)

        q = self.q.copy()
        p = p0 + 0.5 * eps * (g0 if field is None else grad(q)[1])
        lp1, g1 = None, None
        for step in range(self.L):
            q = q + eps * self._velocity(p)
            lpq, gq = grad(q)
            p = p + (eps if step < self.L - 1 else 0.5 * eps) * gq
            lp1, g1 = lpq, gq
        if field is not None:
            lp1, g1 = self._exact(safe(q))
        H0 = -lp0 + self._kinetic(p0)
        H1 = -lp1 + self._kinetic(p)
        log_a = np.where(np.isfinite(H1) & ~bad, H0 - H1, -np.inf)
        a = np.exp(np.minimum(0.0, log_a))
        u = self.rng.random(self.C)
        take = (u < a) & ~bad
        self.q[take] = q[take]
        self.divergent += int(bad.sum())
        lp_new = np.where(take, lp1, lp0)
        g_new = np.where(take[:, None], g1, g0) if (g1 is not None and g0 is not None) else None
        return a, lp_new, g_new

    def warmup(self, n, field=None, anchor=None, moves=1, feature_anchor=None):
        """Adapt the step size (dual averaging, every iteration) and the dense
        metric: a fast window (first 15%), slow windows of doubling length
        whose draws give a covariance estimate (shrunk towards its diagonal),
        and a final fast window (last 10%).  Returns the iteration at which
        the last slow window began (its draws are in the posterior's bulk)."""
        self._init_scale()
        da = DualAveraging(self.eps.copy())
        start, end = int(0.15 * n), int(0.90 * n)
        bounds, w, b = [], 25, start
        while b < end:
            e = end if end - (b + w) < 2 * w else b + w
            bounds.append((b, e))
            b, w = e, 2 * w
        draws, last_start = [], start
        for k in range(n):
            a = self.transition(field, anchor, moves, feature_anchor)
            self.eps = da.update(a)
            for (w0, w1) in bounds:
                if w0 <= k < w1:
                    draws.append(self.q.copy())
                if k == w1 - 1 and len(draws) > 10:
                    D = np.stack(draws)  # (draws, C, 6)
                    m = D.shape[0]
                    cov = np.stack([np.cov(D[:, c].T) for c in range(self.C)])
                    diag = np.stack([np.diag(np.diag(cv)) for cv in cov])
                    cov = (m / (m + 5.0)) * cov + (5.0 / (m + 5.0)) * diag
                    cov += np.stack([1e-10 * np.trace(cv) / 6 * np.eye(6) for cv in cov])
                    self.set_cov(cov)
                    draws = []
                    da = DualAveraging(self.eps.copy())
                    last_start = w0
        self.eps = da.final()
        return last_start

    def sample(self, n, field=None, anchor=None, moves=1, feature_anchor=None):
        out = np.zeros((self.C, n, 6))
        acc = np.zeros(n)
        t0 = time.perf_counter()
        for k in range(n):
            acc[k] = self.transition(field, anchor, moves, feature_anchor).mean()
            out[:, k] = self.q
        return out, acc, time.perf_counter() - t0

    # ---- checkpoint -----------------------------------------------------
    def state(self):
        return {"q": self.q.copy(), "eps": self.eps.copy(), "cov": self.cov.copy(),
                "iteration": self.iteration, "L": self.L, "jitter": self.jitter,
                "rng": self.rng.bit_generator.state}

    def set_state(self, st):
        self.q = np.array(st["q"], dtype=np.float64)
        self.eps = np.array(st["eps"], dtype=np.float64)
        self.set_cov(st["cov"])
        self.iteration = int(st["iteration"])
        self.L = int(st["L"])
        self.jitter = float(st.get("jitter", self.jitter))
        self.rng.bit_generator.state = st["rng"]


class MHSampler:
    """The paper's sampler (Sec. 2.2): univariate-update random-walk
    Metropolis-Hastings on eta = log p, one coordinate at a time, after a
    fresh location draw each iteration (cut scheme).  Each coordinate's
    proposal scale adapts during warmup towards an acceptance rate of 0.44
    (Robbins-Monro on its log).  Chains advance in lockstep: each univariate
    update is one batched exact evaluation of all chains, of the
    log-likelihood only when the target offers that (the sampler needs no
    gradient)."""

    def __init__(self, target, prior, eta_init, seed=0, cut=True):
        self.target = target
        self.prior = prior
        self.q = np.array(eta_init, dtype=np.float64, copy=True)
        self.C = self.q.shape[0]
        self.cut = bool(cut)
        self.rng = np.random.default_rng(seed)
        self.log_scale = np.full((self.C, 6), np.log(0.01))
        self.iteration = 0
        self.warm_k = 0  # warmup iterations done (the adaptation schedule's position)

    def _logpost(self, eta, resample=False):
        ll_only = hasattr(self.target, "eval_loglik")
        if resample:
            f = self.target.resample_eval_loglik if ll_only else self.target.resample_eval
            ll, _ = f(self.iteration, eta)
        else:
            ll, _ = (self.target.eval_loglik if ll_only else self.target.eval)(eta)
        return ll + self.prior(eta)[0]

    def transition(self, adapt_rate=0.0):
        """One iteration: new locations, then six univariate updates.
        Returns the acceptance indicator array (C, 6)."""
        self.iteration += 1
        lp = self._logpost(self.q, resample=self.cut)
        acc = np.zeros((self.C, 6))
        for k in range(6):
            prop = self.q.copy()
            prop[:, k] += np.exp(self.log_scale[:, k]) * self.rng.standard_normal(self.C)
            ok = np.all(np.abs(prop) <= ETA_MAX, axis=1)
            lp_new = self._logpost(np.where(ok[:, None], prop, self.q))
            log_a = np.where(ok & np.isfinite(lp_new), lp_new - lp, -np.inf)
            take = np.log(self.rng.random(self.C)) < log_a
            self.q[take] = prop[take]
            lp = np.where(take, lp_new, lp)
            acc[:, k] = take
            if adapt_rate > 0:
                a = np.exp(np.minimum(0.0, log_a))
                self.log_scale[:, k] += adapt_rate * (a - 0.44)
        return acc

    def warmup(self, n):
        """n more adaptation iterations, continuing the schedule (rate
        1/sqrt(k + 1) at the k-th warmup iteration overall), so a run resumed
        from a checkpoint taken during warmup adapts as an uninterrupted one."""
        for _ in range(n):
            self.transition(adapt_rate=1.0 / np.sqrt(self.warm_k + 1.0))
            self.warm_k += 1

    # ---- checkpoint -----------------------------------------------------
    def state(self):
        return {"kind": "mh", "q": self.q.copy(), "log_scale": self.log_scale.copy(),
                "iteration": self.iteration, "warm_k": self.warm_k, "cut": self.cut,
                "rng": self.rng.bit_generator.state}

    def set_state(self, st):
        self.q = np.array(st["q"], dtype=np.float64)
        self.log_scale = np.array(st["log_scale"], dtype=np.float64)
        self.iteration = int(st["iteration"])
        self.warm_k = int(st.get("warm_k", 0))
        self.cut = bool(st.get("cut", self.cut))
        self.rng.bit_generator.state = st["rng"]

    def sample(self, n):
        out = np.zeros((self.C, n, 6))
        acc = np.zeros(n)
        t0 = time.perf_counter()
        for k in range(n):
            acc[k] = self.transition().mean()
            out[:, k] = self.q
        return out, acc, time.perf_counter() - t0


def cut_posterior_reference(target, prior, q_start, cov, eps, rounds, burn, draws, n_leapfrog=10,
                            seed=0, first_iteration=10_000):
    """Draws from the cut posterior itself, the mixture over location draws X
    of p(Theta | X, t) (Sec. 2.2), independent of how well one MCMC move
    mixes under one X: for each of `rounds` rounds, draw new locations for
    every chain (resample counter first_iteration + round), then run exact HMC
    with those locations held fixed (`burn` moves, then `draws` kept), which
    samples p(Theta | X, t) exactly.  Returns (C * rounds, draws, 6): one
    chain per (chain, round), each with its own X."""
    C = q_start.shape[0]
    out = []
    for r in range(rounds):
        target.resample_eval(first_iteration + r, q_start)  # new X for every chain
        smp = Sampler(target, prior, q_start, n_leapfrog=n_leapfrog, seed=seed + r, cut=False)
        smp.eps = np.array(eps, dtype=np.float64, copy=True)
        smp.set_cov(cov)
        for _ in range(burn):
            smp.transition()
        d, _, _ = smp.sample(draws)
        out.append(d)
    return np.concatenate(out, axis=0)


def save(path, sampler, mlp=None, train_X=None, train_Y=None, train_F=None):
    """Checkpoint the sampler (HMC or univariate MH; and the surrogate:
    weights + its training set, with the draw features of a network trained
    on them, from which its standardisation is recomputed) to an .npz file.
    The MH sampler has no surrogate: passing one with it raises ValueError."""
    import json
    st = sampler.state()
    if st.get("kind") == "mh":
        if mlp is not None or train_X is not None or train_Y is not None or train_F is not None:
            raise ValueError("the univariate MH sampler has no surrogate to save")
        np.savez(path, kind="mh", q=st["q"], log_scale=st["log_scale"], iteration=st["iteration"],
                 warm_k=st["warm_k"], cut=st["cut"], rng=json.dumps(st["rng"]))
        return
    extra = {}
    if mlp is not None:
        extra["mlp_params"] = mlp.get_params()
        extra["train_X"] = np.asarray(train_X)
        extra["train_Y"] = np.asarray(train_Y)
        if train_F is not None:
            extra["train_F"] = np.asarray(train_F)
    np.savez(path, q=st["q"], eps=st["eps"], cov=st["cov"], iteration=st["iteration"], L=st["L"],
             jitter=st["jitter"], rng=json.dumps(st["rng"]), **extra)


def load(path, sampler, mlp=None):
    """Restore a checkpoint written by ``save`` into a sampler of the same
    kind (and, for HMC, the surrogate).  A univariate MH checkpoint also
    restores the sampler's cut setting; passing a surrogate with it raises
    ValueError."""
    import json
    z = np.load(path, allow_pickle=False)
    if "kind" in z and str(z["kind"]) == "mh":
        if mlp is not None:
            raise ValueError("the univariate MH sampler has no surrogate to load")
        sampler.set_state({"q": z["q"], "log_scale": z["log_scale"], "iteration": int(z["iteration"]),
                           "warm_k": int(z["warm_k"]) if "warm_k" in z else 0,
                           "cut": bool(z["cut"]) if "cut" in z else sampler.cut,
                           "rng": json.loads(str(z["rng"]))})
        return
    sampler.set_state({"q": z["q"], "eps": z["eps"], "cov": z["cov"], "iteration": int(z["iteration"]),
                       "L": int(z["L"]), "jitter": float(z["jitter"]), "rng": json.loads(str(z["rng"]))})
    if mlp is not None and "mlp_params" in z:
        mlp.set_data(z["train_X"], z["train_Y"], z["train_F"] if "train_F" in z else None)
        mlp.set_params(z["mlp_params"])


def training_set(record, k_mad=25.0, with_feature=False):
    """Stack recorded exact evaluations into (X[n x 6], Y[n x 7]), and with
    with_feature also F[n], the draw feature of each evaluation (records
    without one are skipped).  Rows with a non-finite value, or with any
    column more than k_mad median absolute deviations from that column's
    median, are dropped: leapfrog excursions far outside the posterior
    (log-likelihoods many orders of magnitude below the bulk) would
    otherwise set the network's standardisation."""
    if with_feature:
        record = [r for r in record if len(r) > 3 and r[3] is not None]
    X = np.concatenate([r[0] for r in record])
    Y = np.concatenate([np.column_stack([r[1], r[2]]) for r in record])
    F = np.concatenate([r[3] for r in record]) if with_feature else np.zeros(X.shape[0])
    ok = np.all(np.isfinite(X), axis=1) & np.all(np.isfinite(Y), axis=1) & np.isfinite(F)
    X, Y, F = X[ok], Y[ok], F[ok]
    Z = np.column_stack([X, Y, F])
    med = np.median(Z, axis=0)
    mad = np.median(np.abs(Z - med), axis=0)
    mad = np.where(mad > 0, mad, np.maximum(np.abs(med), 1.0) * 1e-12)
    keep = np.all(np.abs(Z - med) <= k_mad * mad, axis=1)
    if with_feature:
        return X[keep], Y[keep], F[keep]
    return X[keep], Y[keep]
