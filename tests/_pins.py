"""Checks that pin the CPU oracle to things other than itself.

Each check takes a loaded oracle library ``L`` (the real one, or a copy with a
planted mistake) and returns (ok, message).  None of them retypes the oracle's
loop: they use closed forms for N = 1 and N = 2 written through scipy's
density functions, the same model assembled from scipy.stats densities with
boolean masks, numerical quadrature of the temporal intensity, invariances of
the model, finite differences of the oracle's own value, and the long-double
build.
"""
import math

import numpy as np
from scipy import integrate
from scipy.stats import expon, norm, uniform

import oracle

P0 = (0.5, 20.0, 7.0, 0.3, 0.2, 2.0)
CLIP = 1e-40


def small_events(n, seed, T=30.0, L=60.0, ties=False):
    rng = np.random.default_rng(seed)
    t = np.sort(T * (1.0 - rng.random(n)))
    if ties:
        t = np.sort(np.ceil(t / 3.0) * 3.0)
    x = rng.uniform(0, L, n)
    y = rng.uniform(0, L, n)
    s = np.exp(rng.normal(0, 0.5, n))
    return t, x, y, s


# ---------------------------------------------------------------------------
# Independent formulations
# ---------------------------------------------------------------------------

def scipy_loglam(t, x, y, s, p, bg_time_only=False):
    """log lambda_i from scipy.stats densities (product of 1-D normals for the
    spherical 2-D Gaussian, expon for the temporal decay), masks as eq. 2-3.
    bg_time_only: eq. 2's background, a uniform density over a domain of area
    tau_x^2 times a normal density in time."""
    mu, tx, tt, th, om, h = p
    n = t.shape[0]
    s = np.ones(n) if s is None else s
    out = np.empty(n)
    for i in range(n):
        dt, dx, dy = t[i] - t, x[i] - x, y[i] - y
        bg = (t != t[i])
        if bg_time_only:
            b = norm.pdf(dt, scale=tt) * uniform.pdf(0.0, scale=tx * tx)
        else:
            b = norm.pdf(dx, scale=tx) * norm.pdf(dy, scale=tx) * norm.pdf(dt, scale=tt)
        ex = t < t[i]
        sd = h * s
        e = expon.pdf(dt, scale=1.0 / om) * norm.pdf(dx, scale=sd) * norm.pdf(dy, scale=sd)
        lam = mu * b[bg].sum() + th * e[ex].sum()
        out[i] = math.log(max(lam, CLIP))
    return out


def scipy_Lambda(t, p):
    """Lambda_i = mass of event i's background and triggering kernels on (0, t_N]."""
    mu, tx, tt, th, om, h = p
    tN = t.max()
    return mu * (norm.cdf(tN, loc=t, scale=tt) - norm.cdf(0.0, loc=t, scale=tt)) + \
        th * expon.cdf(tN - t, scale=1.0 / om)


def quad_Lambda(ti, tN, p):
    mu, tx, tt, th, om, h = p
    a, _ = integrate.quad(lambda u: norm.pdf(u, loc=ti, scale=tt), 0.0, tN,
                          points=[ti], epsabs=1e-14, epsrel=1e-13, limit=200)
    b = 0.0
    if tN > ti:
        b, _ = integrate.quad(lambda u: om * math.exp(-om * (u - ti)), ti, tN,
                              epsabs=1e-14, epsrel=1e-13)
    return mu * a + th * b


def rel(a, b, floor=0.0):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.max(np.abs(a - b) / np.maximum(np.maximum(np.abs(b), floor), 1e-300)))


# ---------------------------------------------------------------------------
# Pins
# ---------------------------------------------------------------------------

def pin_n1(L):
    p = P0
    t = np.array([3.5]); x = np.array([10.0]); y = np.array([-4.0])
    out = oracle.loglik_grad(t, x, y, p, L=L)
    mu, tx, tt, th, om, h = p
    bq = -t[0] / tt
    ell = math.log(CLIP) - mu * (0.5 - norm.cdf(bq))
    g = [-(0.5 - norm.cdf(bq)), 0.0, -mu * norm.pdf(bq) * bq / tt, 0.0, 0.0, 0.0]
    exp = np.array([ell] + g)
    err = float(np.max(np.abs(out - exp)))
    return err < 1e-12, f"N=1 closed form: max abs err {err:.3g}"


def pin_n2(L):
    p = (0.7, 15.0, 4.0, 0.4, 0.3, 3.0)
    mu, tx, tt, th, om, h = p
    t = np.array([2.0, 5.5]); x = np.array([1.0, 4.0]); y = np.array([2.0, -1.5])
    s = np.array([1.7, 0.6])
    d = t[1] - t[0]
    # phi2(r; sd) = pdf_x * pdf_y for the 2-D spherical Gaussian at offset (dx, dy)
    B = mu * norm.pdf(x[1] - x[0], scale=tx) * norm.pdf(y[1] - y[0], scale=tx) * norm.pdf(d, scale=tt)
    E = th * expon.pdf(d, scale=1 / om) * norm.pdf(x[1] - x[0], scale=h * s[0]) * \
        norm.pdf(y[1] - y[0], scale=h * s[0])
    lam1, lam2 = B, B + E
    tN = t[1]
    Lam = [mu * (norm.cdf((tN - ti) / tt) - norm.cdf(-ti / tt)) + th * (1 - math.exp(-om * (tN - ti)))
           for ti in t]
    ell = math.log(lam1) + math.log(lam2) - Lam[0] - Lam[1]
    out = oracle.loglik_grad(t, x, y, p, s=s, L=L)
    e1 = abs(out[0] - ell) / abs(ell)
    # swapped input order must not matter (the oracle does not need sorting)
    out2 = oracle.loglik_grad(t[::-1], x[::-1], y[::-1], p, s=s[::-1], L=L)
    e2 = abs(out2[0] - ell) / abs(ell)
    # tie: both rates are zero and clipped
    tt2 = np.array([2.0, 2.0])
    out3 = oracle.loglik_grad(tt2, x, y, p, s=s, L=L)
    ell3 = 2 * math.log(CLIP) - 2 * mu * (norm.cdf(0) - norm.cdf(-2.0 / tt)) - 0.0
    e3 = abs(out3[0] - ell3) / abs(ell3)
    g3 = float(np.max(np.abs(out3[[2, 4, 6]])))          # tau_x, theta, h terms vanish
    ok = e1 < 1e-13 and e2 < 1e-13 and e3 < 1e-13 and g3 == 0.0
    return ok, f"N=2 closed form rel {e1:.3g}, reversed {e2:.3g}, tie {e3:.3g}, tie grads {g3:.3g}"


def pin_scipy_general(L, n=60, seed=1, ties=False, model1=False, p=P0):
    t, x, y, s = small_events(n, seed, ties=ties)
    if model1:
        s = None
    out, rows = oracle.loglik_grad(t, x, y, p, s=s, rows=True, L=L)
    ll = scipy_loglam(t, x, y, s, p)
    La = scipy_Lambda(t, p)
    e_ll = rel(rows[:, 7], ll, floor=1.0)
    e_La = rel(rows[:, 8], La, floor=1e-3)
    e_tot = abs(out[0] - (ll.sum() - La.sum())) / abs(out[0])
    ok = e_ll < 1e-12 and e_La < 1e-12 and e_tot < 1e-12
    return ok, (f"scipy formulation (n={n}, ties={ties}, model1={model1}): log lambda {e_ll:.3g}, "
                f"Lambda {e_La:.3g}, total {e_tot:.3g}")


def pin_bg_time_scipy(L, n=60, seed=14, ties=True):
    """Eq. 2's time-only background against the scipy formulation; Lambda is
    the same as for the space-time background (both kernels have unit mass)."""
    t, x, y, s = small_events(n, seed, ties=ties)
    out, rows = oracle.loglik_grad(t, x, y, P0, s=s, rows=True, L=L, bg_time_only=True)
    ll = scipy_loglam(t, x, y, s, P0, bg_time_only=True)
    La = scipy_Lambda(t, P0)
    e_ll = rel(rows[:, 7], ll, floor=1.0)
    e_La = rel(rows[:, 8], La, floor=1e-3)
    e_tot = abs(out[0] - (ll.sum() - La.sum())) / abs(out[0])
    ok = e_ll < 1e-12 and e_La < 1e-12 and e_tot < 1e-12
    return ok, f"time-only background vs scipy: log lambda {e_ll:.3g}, Lambda {e_La:.3g}, total {e_tot:.3g}"


def pin_bg_time_theta0(L, n=70, seed=15):
    """Time-only background with theta = 0: lambda_i = mu K_i / tau_x^2 with K_i
    a sum over times only, so (a) ell and every partial derivative but d/d theta
    do not depend on the locations at all,
    (b) d ell/d tau_x = -2 m / tau_x and (c) d ell/d mu = m / mu - sum_i
    [Phi((t_N - t_i)/tau_t) - Phi(-t_i/tau_t)], m = number of unclipped rows."""
    t, x, y, s = small_events(n, seed, ties=True)
    p = (0.5, 20.0, 7.0, 0.0, 0.2, 2.0)
    a = oracle.loglik_grad(t, x, y, p, s=s, L=L, bg_time_only=True)
    rng = np.random.default_rng(seed)
    b = oracle.loglik_grad(t, rng.uniform(-1e3, 1e3, n), rng.uniform(-1e3, 1e3, n), p, s=s, L=L,
                           bg_time_only=True)
    keep = [0, 1, 2, 3, 5, 6]
    e1 = rel(b[keep], a[keep], floor=1e-6 * abs(a[0]))
    m = int(np.sum([np.any(t != ti) for ti in t]))
    mu, tx, tt = p[0], p[1], p[2]
    e2 = abs(a[2] - (-2.0 * m / tx)) / (2.0 * m / tx)
    dmu = m / mu - (norm.cdf((t.max() - t) / tt) - norm.cdf(-t / tt)).sum()
    e3 = abs(a[1] - dmu) / abs(dmu)
    ok = e1 < 1e-13 and e2 < 1e-13 and e3 < 1e-12
    return ok, f"time-only theta=0: location-free {e1:.3g}, d/dtau_x {e2:.3g}, d/dmu {e3:.3g}"


def pin_quad_Lambda(L, n=40, seed=2):
    t, x, y, s = small_events(n, seed)
    p = P0
    _, rows = oracle.loglik_grad(t, x, y, p, s=s, rows=True, L=L)
    tN = t.max()
    idx = [0, 7, 19, n - 2, n - 1]
    q = np.array([quad_Lambda(t[i], tN, p) for i in idx])
    e = rel(rows[idx, 8], q, floor=1e-3)
    return e < 1e-10, f"Lambda_i vs quadrature: rel {e:.3g}"


def pin_theta0(L, n=80, seed=3):
    """xi_0 = 0: leave-one-out product-Gaussian KDE score; d ell/d theta stays finite."""
    t, x, y, s = small_events(n, seed)
    p = (0.5, 20.0, 7.0, 0.0, 0.2, 2.0)
    out = oracle.loglik_grad(t, x, y, p, s=s, L=L)
    mu, tx, tt = p[0], p[1], p[2]
    dx = x[:, None] - x[None, :]
    dy = y[:, None] - y[None, :]
    dt = t[:, None] - t[None, :]
    K = norm.pdf(dx, scale=tx) * norm.pdf(dy, scale=tx) * norm.pdf(dt, scale=tt)
    K[t[:, None] == t[None, :]] = 0.0
    lam = mu * K.sum(axis=1)
    ell = np.log(lam).sum() - scipy_Lambda(t, p).sum()
    e = abs(out[0] - ell) / abs(ell)
    # d ell / d theta at theta = 0: sum_i SE_i / lambda_i - sum_i (1 - e^{-omega (t_N - t_i)})
    om, h = p[4], p[5]
    E = expon.pdf(dt, scale=1 / om) * norm.pdf(dx, scale=h * s[None, :]) * norm.pdf(dy, scale=h * s[None, :])
    E[~(t[None, :] < t[:, None])] = 0.0
    dth = (E.sum(axis=1) / lam).sum() - (1 - np.exp(-om * (t.max() - t))).sum()
    e2 = abs(out[4] - dth) / abs(dth)
    return e < 1e-12 and e2 < 1e-11, f"theta=0 KDE: rel {e:.3g}; d/dtheta rel {e2:.3g}"


def pin_mu0(L, n=50, seed=4):
    """mu = 0: pure excitation; the earliest event has no source and is clipped."""
    t, x, y, s = small_events(n, seed)
    p = (0.0, 20.0, 7.0, 0.3, 0.2, 2.0)
    out, rows = oracle.loglik_grad(t, x, y, p, s=s, rows=True, L=L)
    ll = scipy_loglam(t, x, y, s, p)
    e = rel(rows[:, 7], ll, floor=1.0)
    first = rows[0, 7] == math.log(CLIP)
    return e < 1e-12 and first, f"mu=0: log lambda rel {e:.3g}, first event clipped {first}"


def pin_model1_equals_unit_scale(L, n=50, seed=5):
    t, x, y, s = small_events(n, seed)
    a = oracle.loglik_grad(t, x, y, P0, s=None, L=L)
    b = oracle.loglik_grad(t, x, y, P0, s=np.ones(n), L=L)
    return bool(np.all(a == b)), "model 1 == model 2 with s = 1 (bitwise)"


def pin_invariances(L, n=120, seed=6):
    t, x, y, s = small_events(n, seed)
    base = oracle.loglik_grad(t, x, y, P0, s=s, L=L)
    th = 0.7
    c, sn = math.cos(th), math.sin(th)
    xr, yr = c * x - sn * y + 1234.5, sn * x + c * y - 987.25
    rot = oracle.loglik_grad(t, xr, yr, P0, s=s, L=L)
    perm = np.random.default_rng(seed).permutation(n)
    per = oracle.loglik_grad(t[perm], x[perm], y[perm], P0, s=s[perm], L=L)
    e1 = rel(rot, base, floor=1e-3 * abs(base[0]))
    e2 = rel(per, base, floor=1e-3 * abs(base[0]))
    # time translation: only Lambda's lower-limit term moves
    cshift = 2.5
    sh = oracle.loglik_grad(t + cshift, x, y, P0, s=s, L=L)
    mu, tt = P0[0], P0[2]
    d_exp = -mu * (norm.cdf(-t / tt) - norm.cdf(-(t + cshift) / tt)).sum()
    e3 = abs((sh[0] - base[0]) - d_exp) / abs(d_exp)
    ok = e1 < 1e-10 and e2 < 1e-11 and e3 < 1e-8
    return ok, f"rotation+translation {e1:.3g}, permutation {e2:.3g}, time shift vs closed form {e3:.3g}"


def pin_finite_differences(L, n=150, seed=7, ties=False, p=P0, bg_time_only=False):
    """Central differences in log-parameter space with one Richardson step."""
    t, x, y, s = small_events(n, seed, ties=ties)
    g = oracle.loglik_grad(t, x, y, p, s=s, L=L, bg_time_only=bg_time_only)
    eta = np.log(np.asarray(p, float))
    worst = 0.0
    ok = True
    for k in range(6):
        if p[k] == 0:
            continue

        def f(e):
            q = np.exp(eta.copy())
            q[k] = math.exp(e)
            return oracle.loglik_grad(t, x, y, q, s=s, L=L, bg_time_only=bg_time_only)[0]

        def D(hh):
            return (f(eta[k] + hh) - f(eta[k] - hh)) / (2 * hh)

        fd = (4 * D(5e-4) - D(1e-3)) / 3
        an = p[k] * g[1 + k]
        err = abs(fd - an) / (abs(an) + 1e-6 * abs(g[0]) + 1e-8)
        worst = max(worst, err)
        ok = ok and err < 1e-7
    return ok, (f"finite differences (n={n}, ties={ties}, time-only background {bg_time_only}): "
                f"worst rel {worst:.3g}")


def pin_long_double(L, n=100, seed=8):
    t, x, y, s = small_events(n, seed)
    a = oracle.loglik_grad(t, x, y, P0, s=s, L=L)
    b = oracle.loglik_grad(t, x, y, P0, s=s, precision="ld", L=L)
    e = rel(a, b, floor=1e-6 * abs(b[0]))
    return e < 1e-12, f"double vs long double: rel {e:.3g}"


def pin_row_window(L, n=90, seed=9):
    t, x, y, s = small_events(n, seed)
    full = oracle.loglik_grad(t, x, y, P0, s=s, L=L)
    parts = sum(oracle.loglik_grad(t, x, y, P0, s=s, row_begin=a, row_end=b, L=L)
                for a, b in ((0, 17), (17, 60), (60, n)))
    e = rel(parts, full, floor=1e-6 * abs(full[0]))
    return e < 1e-12, f"row windows sum to the whole: rel {e:.3g}"


ALL_PINS = [
    pin_n1, pin_n2, pin_scipy_general,
    lambda L: pin_scipy_general(L, n=70, seed=11, ties=True),
    lambda L: pin_scipy_general(L, n=50, seed=12, model1=True),
    pin_quad_Lambda, pin_theta0, pin_mu0, pin_model1_equals_unit_scale, pin_invariances,
    pin_finite_differences,
    lambda L: pin_finite_differences(L, n=90, seed=13, ties=True),
    pin_long_double, pin_row_window,
    pin_bg_time_scipy, pin_bg_time_theta0,
    lambda L: pin_finite_differences(L, n=90, seed=16, ties=True, bg_time_only=True),
]
