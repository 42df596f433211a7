"""The HAWKES_DEBUG build (device-side index checks, the library's stand-in
for a memory checker) on the GPU.

In a child process that loads lib/libhawkes_debug.so: every regular path
(symmetric sweep, row windows, ties, Model 1, the time-only background, the
FP64 path, a batch, a batch with two chains per CTA, the allocation-free
entry point) runs with no check
firing and matches the oracle at the FP32-path tolerances; then one work item
is overwritten to end one column tile past its row tile's causal triangle.
That tile is still inside the padded arrays, so the planted item is memory
safe even if a check missed it; the debug kernel must refuse it and report
HAWKES_ERR_BOUNDS, and the context must work again once the list is rebuilt."""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent('''
    import numpy as np
    import torch
    import oracle
    from paper_2407_11349_gb300 import synth
    from paper_2407_11349_gb300.hawkes import (HAWKES_BG_TIME, HAWKES_F32, HAWKES_F64, HAWKES_MODEL1,
                                               Batch, Hawkes, HawkesError, hawkes_debug_build,
                                               hawkes_debug_set_item, hawkes_loglik_grad_noalloc)

    assert hawkes_debug_build() == 1
    P0 = synth.DEFAULT_PARAMS

    def close(got_ll, got_g, ref, rows, tol_ll, tol_g, what):
        scale = np.abs(rows[:, 1:7]).sum(axis=0)
        e_ll = abs(got_ll - ref[0]) / abs(ref[0])
        e_g = np.abs(got_g - ref[1:]) / np.maximum(np.maximum(np.abs(ref[1:]), 1e-3 * scale), 1e-300)
        assert e_ll <= tol_ll and np.all(e_g <= tol_g), (what, e_ll, e_g)

    hk = Hawkes(0)
    for n, ties, fl in ((1, False, 0), (257, False, 0), (5000, False, 0), (3000, True, 0),
                        (2049, False, HAWKES_MODEL1), (4000, True, HAWKES_BG_TIME)):
        ds = synth.grid_dataset(n, 100.0, 20, 20, seed=n)
        if ties:
            ds = synth.integer_day_times(ds)
        hk.load(ds)
        s = None if fl & HAWKES_MODEL1 else ds.s
        ref, rows = oracle.loglik_grad(ds.t, ds.x, ds.y, P0, s=s, rows=True,
                                       bg_time_only=bool(fl & HAWKES_BG_TIME))
        ll, g = hk.loglik_grad(P0, HAWKES_F32 | fl)
        close(ll, g, ref, rows, 1e-6, 1e-5, f"f32 n={n}")
        ll, g = hk.loglik_grad(P0, HAWKES_F64 | fl)
        close(ll, g, ref, rows, 1e-10, 1e-10, f"f64 n={n}")
        if n > 1000:
            wref = oracle.loglik_grad(ds.t, ds.x, ds.y, P0, s=s, row_begin=300, row_end=n - 200,
                                      bg_time_only=bool(fl & HAWKES_BG_TIME))
            ll, g = hk.loglik_grad(P0, HAWKES_F32 | fl, 300, n - 200)
            close(ll, g, wref, rows[300:n - 200], 1e-6, 1e-5, f"window n={n}")

    # a batch of three problems with resampling, against one call each
    dss = [synth.voronoi_dataset(m, n_cells=60, seed=m) for m in (3000, 5000, 1200)]
    hks = [Hawkes(0).load(d) for d in dss]
    params = synth.chain_params(3, seed=1)
    dp = torch.tensor(params, dtype=torch.float64, device="cuda")
    dout = torch.zeros((3, 7), dtype=torch.float64, device="cuda")
    b = Batch(hks, [7] * 3, [0, 1, 2], HAWKES_F32)
    torch.cuda.synchronize()
    b.run(dp.data_ptr(), 2, dout.data_ptr())
    b.wait()
    got = dout.cpu().numpy()
    for p in range(3):
        hks[p].resample(7, p, 2)
        ref, rows = hks[p].loglik_rows(params[p], HAWKES_F32)
        close(got[p, 0], got[p, 1:], ref, rows, 1e-6, 1e-5, f"batch problem {p}")
    b.close()

    # two chains per CTA (the group kernel): two chains of one data set and
    # one other problem
    dss = [dss[0], dss[0], dss[2]]
    hks = [Hawkes(0).load(d) for d in dss]
    b = Batch(hks, [7] * 3, [0, 1, 2], HAWKES_F32)
    b.set_chains_per_cta(2)
    assert b.config()[3:] == (2, 1)
    torch.cuda.synchronize()
    b.run(dp.data_ptr(), 3, dout.data_ptr())
    b.wait()
    got = dout.cpu().numpy()
    for p in range(3):
        hks[p].resample(7, p, 3)
        ref, rows = hks[p].loglik_rows(params[p], HAWKES_F32)
        close(got[p, 0], got[p, 1:], ref, rows, 1e-6, 1e-5, f"group batch problem {p}")
    b.close()

    # the allocation-free entry point (work list built on the device)
    ds = synth.grid_dataset(6000, 100.0, 20, 20, seed=9)
    dev = {k: torch.tensor(getattr(ds, k), dtype=torch.float64, device="cuda") for k in ("t", "x", "y", "s")}
    pp = torch.tensor(P0, dtype=torch.float64, device="cuda")
    out = torch.zeros(7, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    hawkes_loglik_grad_noalloc(dev["t"].data_ptr(), dev["x"].data_ptr(), dev["y"].data_ptr(),
                               dev["s"].data_ptr(), ds.n, pp.data_ptr(), HAWKES_F32, out.data_ptr(),
                               torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    ref, rows = oracle.loglik_grad(ds.t, ds.x, ds.y, P0, s=ds.s, rows=True)
    o = out.cpu().numpy()
    close(o[0], o[1:], ref, rows, 1e-6, 1e-5, "no-alloc")

    # planted: row tile 2 of N = 5000 (rows 4096..4999) has column tiles
    # [0, 20); an item ending at 21 leaves the triangle but not the padded
    # arrays (npad = 6144 = 24 tiles)
    ds = synth.grid_dataset(5000, 100.0, 20, 20, seed=5000)
    hk.load(ds)
    hk.set_variant(0)
    hawkes_debug_set_item(hk.ctx, 0, 2, 16, 21)
    try:
        hk.loglik_grad(P0, HAWKES_F32)
        raise SystemExit("planted item was not reported")
    except HawkesError as e:
        assert e.status == -10, e.status
    hk.set_variant(0)  # rebuilds the work list
    ref, rows = oracle.loglik_grad(ds.t, ds.x, ds.y, P0, s=ds.s, rows=True)
    ll, g = hk.loglik_grad(P0, HAWKES_F32)
    close(ll, g, ref, rows, 1e-6, 1e-5, "after the planted item")
    print("DEBUG-BUILD-OK")
''')


def test_debug_build_checks_pass_and_catch_a_planted_item():
    from paper_2407_11349_gb300 import build as libbuild
    libbuild.build(debug=True)
    env = dict(os.environ, HAWKES_DEBUG="1")
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=1200)
    assert r.returncode == 0 and "DEBUG-BUILD-OK" in r.stdout, r.stdout[-3000:] + r.stderr[-3000:]
