"""Seeded synthetic county-structured event data.

These inputs stand in for the paper's COVID-19 hospital data and US county
maps (Sec. 3.2), which are not available: times on (0, T] days, counties as
convex polygons (square grids or Voronoi cells) given as fans of triangles,
per-county population densities, and events assigned to counties by a
multinomial draw.  This module only generates data.  It evaluates no part of
the likelihood, its gradient or the location resample; both the CUDA library
and the CPU oracle take what it returns as plain arrays.

Workloads (units: km and days):
  * ``grid_dataset``: uniform times on (0, T], an nx x ny grid of square
    counties, county weights w_c ~ LogNormal(0, 1), counts ~ Multinomial(N,
    w / sum w), locations uniform in the square, density_c = w_c / area.
  * ``voronoi_dataset``: times from a temporal Hawkes process with
    exponential kernel (branching construction, theta = 0.6, omega = 0.2/d)
    rescaled to span (0, T]; Voronoi cells of seeded uniform points in a
    W x H box clipped to the box; ln D_c ~ N(0, 1.3^2); counts ~
    Multinomial(N, D_c area_c / sum); locations uniform in the cell.
  * ``regional_subsets``: square windows of a dataset grown until they hold
    at least N_k events, subsampled to N_k.
In every case s_c = (density_c / median density)^(-1/2), the per-county
source bandwidth scale of the spatially varying model (eq. 3).
"""
from dataclasses import dataclass, field

import math

import numpy as np

# Parameter vector used by every workload: mu, tau_x (km), tau_t (d), theta,
# omega (1/d), h (km).
DEFAULT_PARAMS = (0.5, 20.0, 7.0, 0.3, 0.2, 2.0)
PARAM_NAMES = ("mu", "tau_x", "tau_t", "theta", "omega", "h")


@dataclass
class Counties:
    """Convex county polygons and their fan triangulation."""
    polygons: list                 # per county: (k, 2) vertex array, counter-clockwise
    density: np.ndarray            # per county density (arbitrary units)
    tri_county: np.ndarray = field(default=None)   # int32 [T], non-decreasing
    tri_xy: np.ndarray = field(default=None)       # float64 [T, 6]: ax ay bx by cx cy

    def __post_init__(self):
        tc, tx = [], []
        for c, poly in enumerate(self.polygons):
            for k in range(1, len(poly) - 1):
                tc.append(c)
                tx.append([poly[0, 0], poly[0, 1], poly[k, 0], poly[k, 1],
                           poly[k + 1, 0], poly[k + 1, 1]])
        self.tri_county = np.asarray(tc, dtype=np.int32)
        self.tri_xy = np.asarray(tx, dtype=np.float64).reshape(-1, 6)

    @property
    def n(self):
        return len(self.polygons)

    def areas(self):
        out = np.zeros(self.n)
        for c, p in enumerate(self.polygons):
            x, y = p[:, 0], p[:, 1]
            out[c] = 0.5 * abs(np.dot(x, np.roll(y, -1)) - np.dot(y, np.roll(x, -1)))
        return out

    def scale(self):
        """s_c = (density_c / median)^(-1/2), through a correctly rounded
        square root and division, so that the values are the same on every
        platform (a power function is not correctly rounded)."""
        return 1.0 / np.sqrt(self.density / np.median(self.density))


@dataclass
class Dataset:
    """Events sorted by time plus their county structure."""
    t: np.ndarray          # float64 [N], non-decreasing, > 0
    x: np.ndarray          # float64 [N] initial locations (uniform in county)
    y: np.ndarray
    county: np.ndarray     # int32 [N]
    counties: Counties
    params: tuple = DEFAULT_PARAMS
    name: str = ""

    @property
    def n(self):
        return self.t.shape[0]

    @property
    def county_scale(self):
        return self.counties.scale()

    @property
    def s(self):
        """Per-event source scale s_j = s_{c(j)}."""
        return self.county_scale[self.county]

    def subset(self, idx, name=""):
        idx = np.sort(np.asarray(idx))
        return Dataset(self.t[idx].copy(), self.x[idx].copy(), self.y[idx].copy(),
                       self.county[idx].copy(), self.counties, self.params, name or self.name)


# ----------------------------------------------------------------------------
# County geometry
# ----------------------------------------------------------------------------

def grid_counties(nx, ny, cell, rng):
    polys = []
    for j in range(ny):
        for i in range(nx):
            x0, y0 = i * cell, j * cell
            polys.append(np.array([[x0, y0], [x0 + cell, y0], [x0 + cell, y0 + cell],
                                   [x0, y0 + cell]], dtype=np.float64))
    w = rng.lognormal(0.0, 1.0, size=nx * ny)
    return Counties(polys, w / (cell * cell))


def _clip_halfplane(poly, a, b, c):
    """Keep the part of a convex polygon with a x + b y <= c."""
    out = []
    m = len(poly)
    for k in range(m):
        p, q = poly[k], poly[(k + 1) % m]
        fp = a * p[0] + b * p[1] - c
        fq = a * q[0] + b * q[1] - c
        if fp <= 0:
            out.append(p)
        if (fp < 0 < fq) or (fq < 0 < fp):
            s = fp / (fp - fq)
            out.append(p + s * (q - p))
    return np.array(out, dtype=np.float64).reshape(-1, 2)


def voronoi_counties(n_cells, width, height, rng, log_sd=1.3):
    """Voronoi cells of uniform seeds in [0, width] x [0, height], clipped to the box."""
    from scipy.spatial import Delaunay

    pts = np.column_stack([rng.uniform(0, width, n_cells), rng.uniform(0, height, n_cells)])
    tri = Delaunay(pts)
    indptr, nbrs = tri.vertex_neighbor_vertices
    box = np.array([[0, 0], [width, 0], [width, height], [0, height]], dtype=np.float64)
    polys = []
    for c in range(n_cells):
        poly = box.copy()
        p = pts[c]
        for q in pts[nbrs[indptr[c]:indptr[c + 1]]]:
            d = q - p
            mid = 0.5 * (p + q)
            poly = _clip_halfplane(poly, d[0], d[1], float(d @ mid))
        # drop near-duplicate vertices produced by clipping through a vertex
        keep = [0]
        for k in range(1, len(poly)):
            if np.hypot(*(poly[k] - poly[keep[-1]])) > 1e-9:
                keep.append(k)
        if len(keep) > 1 and np.hypot(*(poly[keep[-1]] - poly[0])) <= 1e-9:
            keep.pop()
        polys.append(poly[keep])
    # exp of each draw through the C library, element by element: vectorised
    # exp implementations differ in the last bit between platforms
    dens = np.array([math.exp(v) for v in rng.normal(0.0, log_sd, size=n_cells)])
    return Counties(polys, dens)


def _uniform_in_polygons(counties, county, rng):
    """Rejection sampling in each county's bounding box (convex polygons)."""
    n = county.shape[0]
    x, y = np.empty(n), np.empty(n)
    order = np.argsort(county, kind="stable")
    bounds = np.searchsorted(county[order], np.arange(counties.n + 1))
    for c in range(counties.n):
        idx = order[bounds[c]:bounds[c + 1]]
        if idx.size == 0:
            continue
        poly = counties.polygons[c]
        lo, hi = poly.min(axis=0), poly.max(axis=0)
        e = np.roll(poly, -1, axis=0) - poly
        todo = idx
        while todo.size:
            px = rng.uniform(lo[0], hi[0], todo.size)
            py = rng.uniform(lo[1], hi[1], todo.size)
            cross = e[None, :, 0] * (py[:, None] - poly[None, :, 1]) - \
                e[None, :, 1] * (px[:, None] - poly[None, :, 0])
            ok = np.all(cross >= 0, axis=1)
            x[todo[ok]], y[todo[ok]] = px[ok], py[ok]
            todo = todo[~ok]
    return x, y


# ----------------------------------------------------------------------------
# Times
# ----------------------------------------------------------------------------

def uniform_times(n, T, rng):
    """n sorted times, uniform on (0, T]."""
    return np.sort(T * (1.0 - rng.random(n)))


def hawkes_times(n, T, rng, theta=0.6, omega=0.2):
    """First n events of a temporal Hawkes process with kernel theta*omega*e^{-omega s}
    and base rate n (1 - theta) / T, built generation by generation (each event
    has Poisson(theta) children after Exp(omega) delays), rescaled to span (0, T]."""
    horizon = 1.3 * T
    base = n * (1.0 - theta) / T
    while True:
        gen = rng.uniform(0.0, horizon, rng.poisson(base * horizon))
        allt = [gen]
        while gen.size:
            k = rng.poisson(theta, gen.size)
            par = np.repeat(gen, k)
            kids = par + rng.exponential(1.0 / omega, par.size)
            gen = kids[kids < horizon]
            allt.append(gen)
        t = np.sort(np.concatenate(allt))
        if t.size >= n:
            t = t[:n]
            return t * (T / t[-1])
        horizon *= 1.5


# ----------------------------------------------------------------------------
# Workloads
# ----------------------------------------------------------------------------

def _assign(n, weights, rng):
    counts = rng.multinomial(n, weights / weights.sum())
    return np.repeat(np.arange(weights.size, dtype=np.int32), counts)


def grid_dataset(n, T, nx, ny, cell=50.0, seed=0, name=""):
    """Uniform times on (0, T], nx x ny square counties of side ``cell`` km."""
    rng = np.random.default_rng(seed)
    counties = grid_counties(nx, ny, cell, rng)
    t = uniform_times(n, T, rng)
    county = rng.permutation(_assign(n, counties.density * cell * cell, rng)).astype(np.int32)
    x, y = _uniform_in_polygons(counties, county, rng)
    return Dataset(t, x, y, county, counties, DEFAULT_PARAMS, name)


def voronoi_dataset(n, T=1200.0, n_cells=3143, width=4500.0, height=2800.0, seed=2,
                    name="", counties=None):
    """Hawkes-burst times, Voronoi counties with lognormal densities (sd 1.3)."""
    rng = np.random.default_rng(seed)
    if counties is None:
        counties = voronoi_counties(n_cells, width, height, rng)
    t = hawkes_times(n, T, rng)
    county = rng.permutation(_assign(n, counties.density * counties.areas(), rng)).astype(np.int32)
    x, y = _uniform_in_polygons(counties, county, rng)
    return Dataset(t, x, y, county, counties, DEFAULT_PARAMS, name)


def clustered_dataset(n, T=100.0, nx=20, ny=20, cell=50.0, seed=0, params=DEFAULT_PARAMS,
                      events_per_centre=40, name=""):
    """Events whose structure matches the model's parameters (for samplers):
    background events scattered around uniform space-time centres with
    Gaussian offsets (sd tau_x in space, tau_t in time), plus branching
    offspring (Poisson(theta) children per event, Exp(omega) delays, Gaussian
    spatial offsets of sd h s_c of the parent's county), kept inside the
    box and (0, T], subsampled to exactly n events.  Counties: an nx x ny
    grid of squares with LogNormal(0, 1) densities."""
    rng = np.random.default_rng(seed)
    mu, tx, tt, th, om, h = params
    counties = grid_counties(nx, ny, cell, rng)
    sc = counties.scale()
    W, H = nx * cell, ny * cell

    def county_of(x, y):
        i = np.clip((x // cell).astype(int), 0, nx - 1)
        j = np.clip((y // cell).astype(int), 0, ny - 1)
        return (j * nx + i).astype(np.int32)

    m_imm = int(1.3 * n * (1.0 - th)) + 10
    while True:
        K = max(1, m_imm // events_per_centre)
        cx, cy, ct = rng.uniform(0, W, K), rng.uniform(0, H, K), rng.uniform(0, T, K)
        k = rng.integers(0, K, m_imm)
        x = cx[k] + rng.normal(0, tx, m_imm)
        y = cy[k] + rng.normal(0, tx, m_imm)
        t = ct[k] + rng.normal(0, tt, m_imm)
        ok = (x >= 0) & (x < W) & (y >= 0) & (y < H) & (t > 0) & (t <= T)
        X, Y, Tt = [x[ok]], [y[ok]], [t[ok]]
        gx, gy, gt = x[ok], y[ok], t[ok]
        while gt.size:
            kids = rng.poisson(th, gt.size)
            px, py, pt = np.repeat(gx, kids), np.repeat(gy, kids), np.repeat(gt, kids)
            sd = h * sc[county_of(px, py)]
            cxk = px + rng.normal(0, 1, px.size) * sd
            cyk = py + rng.normal(0, 1, py.size) * sd
            ctk = pt + rng.exponential(1.0 / om, pt.size)
            ok = (cxk >= 0) & (cxk < W) & (cyk >= 0) & (cyk < H) & (ctk <= T)
            gx, gy, gt = cxk[ok], cyk[ok], ctk[ok]
            X.append(gx), Y.append(gy), Tt.append(gt)
        x, y, t = np.concatenate(X), np.concatenate(Y), np.concatenate(Tt)
        if t.size >= n:
            break
        m_imm = int(m_imm * 1.5)
    keep = np.sort(rng.choice(t.size, n, replace=False))
    x, y, t = x[keep], y[keep], t[keep]
    order = np.argsort(t, kind="stable")
    x, y, t = x[order], y[order], t[order]
    return Dataset(t, x, y, county_of(x, y), counties, params, name or f"clustered{n}")


def integer_day_times(ds, seed=0):
    """Copy of ``ds`` with times rounded up to whole days (many exact ties)."""
    t = np.maximum(np.ceil(ds.t), 1.0)
    return Dataset(np.sort(t), ds.x.copy(), ds.y.copy(), ds.county.copy(), ds.counties,
                   ds.params, ds.name + "-ties")


def chain_params(n_chains, seed=3, sd=0.05, base=DEFAULT_PARAMS):
    """Per-chain parameter vectors: base * exp(N(0, sd^2)) per coordinate."""
    rng = np.random.default_rng(seed)
    return np.asarray(base)[None, :] * np.exp(rng.normal(0.0, sd, size=(n_chains, 6)))


def regional_sizes(k=16, lo=5000, ratio=40.0):
    return [int(round(lo * ratio ** (i / (k - 1)))) for i in range(k)]


def regional_subsets(ds, sizes, seed=3):
    """For each size, a square window around a random event grown until it holds
    at least that many events, subsampled to exactly that many."""
    rng = np.random.default_rng(seed)
    out = []
    for k, m in enumerate(sizes):
        c = rng.integers(ds.n)
        cx, cy = ds.x[c], ds.y[c]
        half = 10.0
        while True:
            inside = np.flatnonzero((np.abs(ds.x - cx) <= half) & (np.abs(ds.y - cy) <= half))
            if inside.size >= m:
                break
            half *= 1.25
        pick = rng.choice(inside, size=m, replace=False)
        out.append(ds.subset(pick, name=f"region{k}-{m}"))
    return out


def config_dataset(which, seed=None):
    """The five named workloads (sizes as documented in the design notes).

    c1: N=2,000 over 100 d, 20x20 grid of 50 km squares, seed 0
    c2: N=100,000 over 1,200 d, 60x60 grid, seed 1
    c3: N=1,000,000 over 1,200 d, 3,143 Voronoi counties, seed 2
    c4: N=250,000 C3-type dataset (the 30 chains' data), seed 3
    """
    if which == "c1":
        return grid_dataset(2000, 100.0, 20, 20, seed=0 if seed is None else seed, name="c1")
    if which == "c2":
        return grid_dataset(100_000, 1200.0, 60, 60, seed=1 if seed is None else seed, name="c2")
    if which == "c3":
        return voronoi_dataset(1_000_000, seed=2 if seed is None else seed, name="c3")
    if which == "c4":
        return voronoi_dataset(250_000, seed=3 if seed is None else seed, name="c4")
    raise ValueError(which)


def fingerprint(arrays):
    """Identify a workload's input arrays (name -> float64 array).

    ``sha256`` is the exact bytes.  ``stats`` are, per array, its length, the
    sums of a, a^2 and a * w (w_k = 1 + (k mod 97), fixed weights) and the
    values at eleven evenly spaced positions: two workloads whose arrays
    differ only in the last bit of a few elements (a platform's library exp
    or log) agree on them to about 1e-15 relative, while any other change
    moves them grossly.  ``same_inputs`` compares two stats records."""
    import hashlib
    h = hashlib.sha256()
    stats = {}
    for name in sorted(arrays):
        a = np.ascontiguousarray(arrays[name], dtype=np.float64)
        h.update(name.encode())
        h.update(a.tobytes())
        w = 1.0 + (np.arange(a.size) % 97)
        pos = np.linspace(0, max(a.size - 1, 0), 11).astype(np.int64)
        stats[name] = {"n": int(a.size), "sum": float(a.sum()), "sum2": float((a * a).sum()),
                       "sumw": float((a * w).sum()), "at": [float(a[k]) for k in pos] if a.size else []}
    return {"sha256": h.hexdigest(), "stats": stats}


def same_inputs(a, b, rel=1e-12):
    """True if two ``fingerprint(...)['stats']`` records describe the same
    arrays up to last-bit differences."""
    if sorted(a) != sorted(b):
        return False
    for k in a:
        x, y = a[k], b[k]
        if x["n"] != y["n"] or len(x["at"]) != len(y["at"]):
            return False
        for u, v in [(x["sum"], y["sum"]), (x["sum2"], y["sum2"]), (x["sumw"], y["sumw"])] + list(zip(x["at"], y["at"])):
            if abs(u - v) > rel * max(abs(u), abs(v), 1e-300):
                return False
    return True
