"""MCMC convergence diagnostics: rank-normalised split-R-hat, bulk and tail
effective sample size (Vehtari, Gelman, Simpson, Carpenter, Buerkner 2021,
"Rank-normalization, folding, and localization"), as used in Sec. 3.2 to
report the worst parameter's bulk/tail ESS and R-hat.

Chains are arrays of shape (chains, draws).  Host-side statistics on a few
thousand numbers per parameter.
"""
import numpy as np
from scipy.special import ndtri


def _split(x):
    x = np.asarray(x, dtype=np.float64)
    if x.ndim == 1:
        x = x[None, :]
    n = x.shape[1] // 2
    return np.concatenate([x[:, :n], x[:, x.shape[1] - n:]], axis=0)


def _rank_normalise(x):
    """z-scores of the pooled ranks (average ranks for ties), offset 3/8."""
    from scipy.stats import rankdata
    flat = x.reshape(-1)
    r = rankdata(flat, method="average")
    S = flat.size
    return ndtri((r - 0.375) / (S + 0.25)).reshape(x.shape)


def _autocov(v):
    """Autocovariance of one chain at all lags (biased, FFT)."""
    n = v.size
    v = v - v.mean()
    m = 1 << (2 * n - 1).bit_length()
    f = np.fft.rfft(v, m)
    ac = np.fft.irfft(f * np.conj(f), m)[:n]
    return ac / n


def ess(x):
    """Effective sample size of (chains, draws) via Geyer's initial monotone
    sequence on the multi-chain autocorrelation estimate."""
    x = np.asarray(x, dtype=np.float64)
    if x.ndim == 1:
        x = x[None, :]
    M, N = x.shape
    if N < 4:
        return np.nan
    acov = np.stack([_autocov(c) for c in x])
    chain_var = acov[:, 0] * N / (N - 1.0)
    W = chain_var.mean()
    mean_c = x.mean(axis=1)
    B_over_N = mean_c.var(ddof=1) if M > 1 else 0.0
    var_plus = W * (N - 1.0) / N + B_over_N
    if not var_plus > 0:
        return np.nan
    rho = 1.0 - (W - acov.mean(axis=0)) / var_plus
    rho[0] = 1.0
    # Geyer: sum consecutive pairs while positive, then make them monotone.
    pairs = []
    t = 0
    while t + 1 < N:
        p = rho[t] + rho[t + 1]
        if p < 0:
            break
        pairs.append(p)
        t += 2
    pairs = np.minimum.accumulate(np.asarray(pairs)) if pairs else np.asarray([1.0])
    tau = -1.0 + 2.0 * pairs.sum()
    tau = max(tau, 1.0 / np.log10(M * N)) if M * N > 1 else tau
    return M * N / tau


def bulk_ess(x):
    return ess(_rank_normalise(_split(x)))


def tail_ess(x, prob=0.05):
    """Minimum ESS of the 5% and 95% quantile indicators."""
    s = _split(x)
    lo, hi = np.quantile(s, [prob, 1 - prob])
    return min(ess((s <= lo).astype(float)), ess((s <= hi).astype(float)))


def rhat(x):
    """Rank-normalised split-R-hat: the larger of the bulk and the folded value."""
    def _rh(y):
        M, N = y.shape
        W = y.var(axis=1, ddof=1).mean()
        B = N * y.mean(axis=1).var(ddof=1)
        return np.sqrt(((N - 1) / N * W + B / N) / W)

    s = _split(x)
    bulk = _rh(_rank_normalise(s))
    folded = _rh(_rank_normalise(np.abs(s - np.median(s))))
    return max(bulk, folded)


def mcse_mean(x):
    x = np.asarray(x, dtype=np.float64)
    return x.std(ddof=1) / np.sqrt(ess(_split(x)))


def summary(draws, names):
    """Per-parameter mean, sd, MCSE of the mean, bulk/tail ESS, R-hat.
    draws: (chains, draws, params)."""
    out = {}
    for k, nm in enumerate(names):
        x = draws[:, :, k]
        out[nm] = {"mean": float(x.mean()), "sd": float(x.std(ddof=1)), "mcse": float(mcse_mean(x)),
                   "bulk_ess": float(bulk_ess(x)), "tail_ess": float(tail_ess(x)), "rhat": float(rhat(x))}
    return out
