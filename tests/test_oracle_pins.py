"""The CPU oracle against what the paper and the mathematics fix (no GPU).

Sec. 2.1 (eqs. 2-4 and the closed-form integral), Sec. 2.3.1 (the 1e-40 clip)
and Sec. 2.2 (uniform-in-county location draws).  Every pin is independent of
the oracle's own loop; the mutation test shows the pins catch plausible
mistakes planted in a copy of the oracle source.
"""
import os
import shutil
import tempfile

import numpy as np
import pytest
from scipy import stats

import _pins
import oracle
from oracle import build_oracle

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


@pytest.fixture(scope="module")
def L():
    return oracle.lib()


@pytest.mark.parametrize("k", range(len(_pins.ALL_PINS)))
def test_pin(L, k):
    ok, msg = _pins.ALL_PINS[k](L)
    assert ok, msg


# (description, text in the source, replacement) -- each a plausible slip.
MUTATIONS = [
    ("2-D normalisation missing 2", "/ (2 * PI_R * sd * sd)", "/ (PI_R * sd * sd)"),
    ("1-D normalisation missing sqrt(2 pi)", "/ (SQRT(2 * PI_R) * sd)", "/ (sd)"),
    ("excitation on ties", "if (tj < ti) {", "if (tj <= ti) {"),
    ("background on ties", "if (tj != ti) {", "if (1) {"),
    ("bandwidth of the target event", "s ? (REAL)s[j]", "s ? (REAL)s[i]"),
    ("no clip", "if (lam < CLIP_R) {", "if (lam < 0) {"),
    ("integral sign", "th * (1 - ea);", "th * (ea - 1);"),
    ("tau_t power", "SBt / (tt * tt * tt)", "SBt / (tt * tt)"),
    ("omega sign", "(SE / om - SEt)", "(SE / om + SEt)"),
    ("dLambda/dtau_t sign", "(-std_normal_pdf(a) * a + std_normal_pdf(b) * b)",
     "(std_normal_pdf(a) * a + std_normal_pdf(b) * b)"),
    ("h moment without 1/s^2", "e * r2 / (sj * sj)", "e * r2"),
    ("time difference reversed", "const REAL dt = ti - tj;", "const REAL dt = tj - ti;"),
    ("t_N from the last input", "if (t[j] > tN) tN = t[j];", "tN = t[j];"),
    ("dropped tau_x factor 2", "- 2 * SB / tx", "- SB / tx"),
    ("time-only background keeps the spatial Gaussian", "const REAL b = phi1(dt, tt) / (tx * tx);",
     "const REAL b = phi2(r2, tx) * phi1(dt, tt);"),
    ("time-only area factor not squared", "phi1(dt, tt) / (tx * tx)", "phi1(dt, tt) / tx"),
    ("time-only background with a spatial moment", "SB += b;                            /*",
     "SB += b; SBr += b * r2; /*"),
]


@pytest.fixture(scope="module")
def mutant_dir():
    d = tempfile.mkdtemp(prefix="oracle_mut_")
    yield d
    shutil.rmtree(d, ignore_errors=True)


@pytest.mark.parametrize("desc,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_mutation(mutant_dir, desc, old, new):
    src = open(build_oracle.SRC).read()
    assert src.count(old) == 1, f"mutation anchor not unique: {old!r}"
    tag = "".join(ch if ch.isalnum() else "_" for ch in desc)
    path = os.path.join(mutant_dir, tag + ".c")
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    so = build_oracle.compile_oracle(src=path, out=os.path.join(mutant_dir, tag, "lib.so"))
    Lm = oracle.lib(so)
    failed = []
    for k, pin in enumerate(_pins.ALL_PINS):
        try:
            ok, msg = pin(Lm)
        except Exception as e:  # a crash of a mutant counts as a caught mistake
            ok, msg = False, repr(e)
        if not ok:
            failed.append(msg)
    assert failed, f"no pin caught the planted mistake: {desc}"


# ---------------------------------------------------------------------------
# Resample: Philox4x64-10 against numpy's independent implementation, and the
# draw's distribution against the uniform law on the polygon.
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("ctr,key", [
    ([0, 0, 0, 0], [0, 0]),
    ([5, 17, 0, 0], [123456789, 42]),
    ([2**64 - 2, 3, 2**63, 1], [2**64 - 1, 2**62 + 5]),
])
def test_philox_matches_numpy(ctr, key):
    # numpy's Philox bit generator (4x64, 10 rounds) increments the counter before
    # each block, so its first output for counter c is the block for c + 1.
    g = np.random.Philox(counter=np.array(ctr, dtype=np.uint64), key=np.array(key, dtype=np.uint64))
    ref = g.random_raw(8)
    c1 = list(ctr)
    for blk in range(2):
        c1[0] = (c1[0] + 1) % 2**64
        if c1[0] == 0:
            c1[1] = (c1[1] + 1) % 2**64
        got = oracle.philox4x64_10(c1, key)
        assert np.array_equal(got, ref[4 * blk:4 * blk + 4])


def _square_and_hexagon():
    sq = np.array([[0, 0], [10, 0], [10, 10], [0, 10]], float)
    ang = np.linspace(0, 2 * np.pi, 7)[:-1]
    hexa = np.column_stack([30 + 8 * np.cos(ang), 5 + 8 * np.sin(ang)])
    from paper_2407_11349_gb300.synth import Counties
    return Counties([sq, hexa], np.array([1.0, 2.0]))


def _inside(poly, x, y):
    e = np.roll(poly, -1, axis=0) - poly
    cross = e[None, :, 0] * (y[:, None] - poly[None, :, 1]) - e[None, :, 1] * (x[:, None] - poly[None, :, 0])
    return np.all(cross >= -1e-9, axis=1)


def test_resample_uniform_in_polygon():
    cs = _square_and_hexagon()
    n = 200_000
    county = np.repeat(np.array([0, 1], np.int32), n // 2)
    x, y = oracle.resample(county, cs.n, cs.tri_county, cs.tri_xy, seed=7, stream=3, iteration=11)
    for c in range(2):
        m = county == c
        assert _inside(cs.polygons[c], x[m], y[m]).all()
    # square: chi-square on a 10 x 10 grid of sub-cells
    m = county == 0
    h, _, _ = np.histogram2d(x[m], y[m], bins=10, range=[[0, 10], [0, 10]])
    chi2 = ((h - h.mean()) ** 2 / h.mean()).sum()
    assert stats.chi2.sf(chi2, 99) > 1e-4
    # hexagon: mean at the centre, and the six fan triangles (unequal angles
    # from vertex 0) hit in proportion to their area: compare the fraction in
    # each 60-degree sector (equal areas) with 1/6.
    m = county == 1
    mx, my = x[m].mean(), y[m].mean()
    se = 8 / np.sqrt(m.sum())
    assert abs(mx - 30) < 5 * se and abs(my - 5) < 5 * se
    sector = np.floor((np.arctan2(y[m] - 5, x[m] - 30) % (2 * np.pi)) / (np.pi / 3)).astype(int)
    cnt = np.bincount(sector, minlength=6)
    chi2 = ((cnt - m.sum() / 6) ** 2 / (m.sum() / 6)).sum()
    assert stats.chi2.sf(chi2, 5) > 1e-4


def test_resample_keying():
    cs = _square_and_hexagon()
    county = np.array([0, 1, 0, 1], np.int32)
    a = oracle.resample(county, cs.n, cs.tri_county, cs.tri_xy, 1, 0, 0)
    b = oracle.resample(county, cs.n, cs.tri_county, cs.tri_xy, 1, 0, 0)
    c = oracle.resample(county, cs.n, cs.tri_county, cs.tri_xy, 1, 0, 1)
    d = oracle.resample(county, cs.n, cs.tri_county, cs.tri_xy, 1, 1, 0)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert not np.array_equal(a[0], c[0]) and not np.array_equal(a[0], d[0])
    # the draw for event i depends only on (i, iteration, seed, stream, its county)
    e = oracle.resample(county[:2], cs.n, cs.tri_county, cs.tri_xy, 1, 0, 0)
    assert np.array_equal(e[0], a[0][:2])


def test_resample_rejects_bad_input():
    cs = _square_and_hexagon()
    with pytest.raises(ValueError):
        oracle.resample(np.array([2], np.int32), cs.n, cs.tri_county, cs.tri_xy, 1, 0, 0)
    with pytest.raises(ValueError):
        oracle.resample(np.array([0], np.int32), cs.n, cs.tri_county[::-1].copy(), cs.tri_xy, 1, 0, 0)
