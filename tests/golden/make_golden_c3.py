"""Write oracle_c3.json: the FP64 oracle's log-likelihood and gradient on the
full c3 workload (N = 1,000,000 events over 1,200 days on 3,143 Voronoi
counties, seed 2; paper_2407_11349_gb300/synth.py), after one cut-posterior
location draw (Sec. 2.2) with seed 2, stream 0, iteration 0, at the default
parameters, with the model of Sec. 2.1 (eqs. 2-4, Sec. 2.3.1 clip).

Only oracle/ computes: the location draw is the oracle's resampler and the
values are its ordered-pair double loop, run on every host core (about
10^12 ordered pairs: roughly 20 minutes on 16 Arm cores, 75 on 8 x86
cores).  Beside the seven totals it stores sum_i |.| of each per-row term (the
scale a component that cancels is judged against) and the input arrays'
fingerprint, so a test can check that it evaluates the same inputs before
comparing.

    python tests/golden/make_golden_c3.py
"""
import json
import os
import platform
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2407_11349_gb300 import synth  # noqa: E402

RESAMPLE = (2, 0, 0)  # seed, stream, iteration
ROWS = [0, 1, 2, 999, 123_456, 333_333, 500_000, 654_321, 777_777, 900_001, 999_998, 999_999]


def c3_inputs():
    """The c3 events with the oracle's location draw: (dataset, x, y)."""
    ds = synth.config_dataset("c3")
    x, y = oracle.resample(ds.county, ds.counties.n, ds.counties.tri_county, ds.counties.tri_xy,
                           *RESAMPLE)
    return ds, x, y


def main():
    ds, x, y = c3_inputs()
    fp = synth.fingerprint({"t": ds.t, "x": x, "y": y, "s": ds.s})
    p = list(synth.DEFAULT_PARAMS)
    t0 = time.perf_counter()
    out, rows = oracle.loglik_grad(ds.t, x, y, p, s=ds.s, rows=True)
    sec = time.perf_counter() - t0
    doc = {"workload": "c3 (synth.config_dataset('c3'): N=1,000,000, 1,200 d, 3,143 Voronoi counties, seed 2) "
                       "after oracle.resample(seed=2, stream=0, iteration=0)",
           "model": "Sec. 2.1 eqs. 2-4 with the Sec. 2.3.1 clip; gradient in (mu, tau_x, tau_t, theta, omega, h)",
           "params": p,
           "loglik_grad": [float(v) for v in out],
           "abs_row_sums": [float(v) for v in np.abs(rows[:, :7]).sum(axis=0)],
           "row_fields": "ell_i, six partials, log lambda_i, Lambda_i",
           "rows": {str(i): [float(v) for v in rows[i]] for i in ROWS},
           "inputs": fp,
           "written_by": "tests/golden/make_golden_c3.py (FP64 oracle)",
           "host": {"machine": platform.machine(), "threads": oracle.max_threads(), "seconds": round(sec, 1)}}
    with open(os.path.join(HERE, "oracle_c3.json"), "w") as f:
        json.dump(doc, f, indent=1)
        f.write("\n")
    print(json.dumps({"seconds": sec, "loglik_grad": doc["loglik_grad"]}))


if __name__ == "__main__":
    main()
