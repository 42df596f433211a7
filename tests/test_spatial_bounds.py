"""The bound behind HAWKES_SKIP_SPATIAL, restated on the host (no GPU): order
events as the library does (time windows cut between distinct times, a
Morton curve inside each), and for every (row tile, column tile) pair that
the tile test declares all-zero, check every pair's exact exponents: the
background exponent dt~^2 + r~^2 above 126 and the excitation exponent
ce - omega~ dt~ - beta r~^2 below -126 (or no earlier source), so that every
term flushes to zero in FP32.  The test uses 2 units of margin, as the
kernel does."""
import numpy as np
import pytest

from paper_2407_11349_gb300 import synth

LOG2E = 1.4426950408889634
TC = 256


def _spread16(v):
    v = v & 0xFFFF
    v = (v | (v << 8)) & 0x00FF00FF
    v = (v | (v << 4)) & 0x0F0F0F0F
    v = (v | (v << 2)) & 0x33333333
    v = (v | (v << 1)) & 0x55555555
    return v


def _order(ds, window):
    n = ds.n
    gx = np.clip((ds.x - ds.x.min()) * (65535.0 / max(np.ptp(ds.x), 1e-300)), 0, 65535).astype(np.int64)
    gy = np.clip((ds.y - ds.y.min()) * (65535.0 / max(np.ptp(ds.y), 1e-300)), 0, 65535).astype(np.int64)
    key = (_spread16(gx) | (_spread16(gy) << 1)).astype(np.int64)
    perm = []
    a = 0
    while a < n:
        b = min(n, a + window)
        while b < n and ds.t[b] == ds.t[b - 1]:
            b += 1
        idx = np.arange(a, b)
        perm.extend(idx[np.lexsort((idx, key[a:b]))])
        a = b
    return np.asarray(perm)


def _zero(rw, col, p, model1=False):
    """The kernel's tile test, restated."""
    mu, tx, tt, th, om, h = p
    ax = LOG2E / (2 * tx * tx)
    kt = np.sqrt(LOG2E / (2 * tt * tt))
    omt = om * LOG2E / kt
    dx = max(0.0, col["x0"] - rw["x1"], rw["x0"] - col["x1"])
    dy = max(0.0, col["y0"] - rw["y1"], rw["y0"] - col["y1"])
    r2 = (dx * dx + dy * dy) * ax
    gap = max(0.0, col["t0"] - rw["t1"], rw["t0"] - col["t1"]) * kt
    if gap * gap + r2 <= 128.0:
        return False
    if col["t0"] >= rw["t1"]:
        return True
    causal = max(0.0, rw["t0"] - col["t1"]) * kt
    smin, smax = (1.0, 1.0) if model1 else (col["s0"], col["s1"])
    return -2 * np.log2(smin) - omt * causal - (tx * tx) / (h * h * smax * smax) * r2 < -128.0


@pytest.mark.parametrize("seed,window,p", [(1, 512, synth.DEFAULT_PARAMS),
                                           (2, 1024, (2.0, 50.0, 10.0, 0.9, 0.05, 20.0)),
                                           (3, 256, (0.5, 5.0, 2.0, 0.3, 1.5, 0.5))])
def test_skipped_tile_pairs_hold_only_fp32_zeros(seed, window, p):
    ds = synth.integer_day_times(synth.grid_dataset(3000, 1200.0, 20, 20, seed=seed)) if seed == 1 else \
        synth.grid_dataset(3000, 1200.0, 20, 20, seed=seed)
    n = ds.n
    perm = _order(ds, window)
    nt = (n + TC - 1) // TC
    tiles = []
    for k in range(nt):
        e = perm[k * TC:(k + 1) * TC]
        tiles.append({"e": e, "x0": ds.x[e].min(), "x1": ds.x[e].max(), "y0": ds.y[e].min(), "y1": ds.y[e].max(),
                      "t0": ds.t[e].min(), "t1": ds.t[e].max(), "s0": ds.s[e].min(), "s1": ds.s[e].max()})
    mu, tx, tt, th, om, h = p
    ax = LOG2E / (2 * tx * tx)
    at = LOG2E / (2 * tt * tt)
    skipped = 0
    for a in range(nt):
        ea = tiles[a]["e"]
        for b in range(nt):
            if not _zero(tiles[a], tiles[b], p):
                continue
            skipped += 1
            eb = tiles[b]["e"]
            dt = ds.t[ea][:, None] - ds.t[eb][None, :]
            r2 = (ds.x[ea][:, None] - ds.x[eb][None, :]) ** 2 + (ds.y[ea][:, None] - ds.y[eb][None, :]) ** 2
            bexp = dt * dt * at + r2 * ax
            assert np.all(bexp > 126.0)
            sj = ds.s[eb][None, :]
            earlier = dt > 0
            eexp = -2 * np.log2(sj) - om * LOG2E * dt - r2 * LOG2E / (2 * h * h * sj * sj)
            assert np.all(~earlier | (eexp < -126.0))
    assert skipped >= 10  # the check is exercised
