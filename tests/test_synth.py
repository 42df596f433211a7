"""The synthetic workloads against their stated recipe (CPU, no GPU): sorted
positive times inside (0, T], every location inside its county polygon,
county scales s_c = (density / median)^(-1/2), the Voronoi map's 3,143
convex cells tiling the box, integer-day ties, the regional subset sizes and
the per-chain parameter spread."""
import numpy as np
import pytest

from paper_2407_11349_gb300 import synth


def _inside_convex(poly, x, y, tol=1e-9):
    """Point in a counter-clockwise convex polygon (cross products >= -tol)."""
    ok = np.ones(x.shape, dtype=bool)
    k = len(poly)
    for a in range(k):
        b = (a + 1) % k
        cr = (poly[b, 0] - poly[a, 0]) * (y - poly[a, 1]) - (poly[b, 1] - poly[a, 1]) * (x - poly[a, 0])
        ok &= cr >= -tol * max(1.0, np.max(np.abs(poly)))
    return ok


def _check_dataset(ds, T):
    assert np.all(np.diff(ds.t) >= 0) and ds.t[0] > 0 and ds.t[-1] <= T + 1e-9
    for c in np.unique(ds.county)[:200]:
        m = ds.county == c
        assert np.all(_inside_convex(ds.counties.polygons[c], ds.x[m], ds.y[m])), c
    s = ds.counties.scale()
    assert np.allclose(s, (ds.counties.density / np.median(ds.counties.density)) ** -0.5)
    assert np.allclose(ds.s, s[ds.county])


def test_grid_workload_c1():
    ds = synth.config_dataset("c1")
    assert ds.n == 2000 and ds.counties.n == 400
    _check_dataset(ds, 100.0)
    assert np.allclose(ds.counties.areas(), 50.0 * 50.0)


def test_voronoi_workload_cells():
    ds = synth.voronoi_dataset(20_000, seed=2)
    assert ds.counties.n == 3143
    _check_dataset(ds, 1200.0)
    areas = ds.counties.areas()
    assert np.all(areas > 0)
    assert abs(areas.sum() - 4500.0 * 2800.0) < 1e-6 * 4500.0 * 2800.0  # the cells tile the box
    tri = ds.counties.tri_xy
    cr = (tri[:, 2] - tri[:, 0]) * (tri[:, 5] - tri[:, 1]) - (tri[:, 4] - tri[:, 0]) * (tri[:, 3] - tri[:, 1])
    assert np.all(cr >= 0)  # fan triangles keep the polygons' orientation
    assert np.all(np.diff(ds.counties.tri_county) >= 0)
    ld = np.log(ds.counties.density)
    assert 0.9 < ld.std() / 1.3 < 1.1  # ln D ~ N(0, 1.3^2)


def test_clustered_workload():
    ds = synth.clustered_dataset(5000, seed=41)
    assert ds.n == 5000
    _check_dataset(ds, 100.0)


def test_integer_days_regions_and_chain_parameters():
    ds = synth.integer_day_times(synth.config_dataset("c1"))
    assert np.all(ds.t == np.round(ds.t)) and np.sum(np.diff(ds.t) == 0) > 1800
    sizes = synth.regional_sizes()
    assert len(sizes) == 16 and sizes[0] == 5000 and sizes[-1] == 200_000
    base = synth.voronoi_dataset(30_000, seed=3)
    regs = synth.regional_subsets(base, [3000, 7000], seed=4)
    assert [r.n for r in regs] == [3000, 7000]
    for r in regs:
        assert np.all(np.diff(r.t) >= 0)
    p = synth.chain_params(30, seed=3)
    ratio = np.log(p / np.asarray(synth.DEFAULT_PARAMS))
    assert p.shape == (30, 6) and 0.03 < ratio.std() < 0.07
