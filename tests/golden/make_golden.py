"""Write oracle_c1.json: the FP64 oracle's values on the c1 workload (N = 2,000
events over 100 days on a 20 x 20 grid of 50 km counties, seed 0; the
workload generator in paper_2407_11349_gb300/synth.py), at the default
parameters and one other parameter set, with the model of Sec. 2.1 (eqs. 2-4,
Sec. 2.3.1 clip).  Only oracle/ computes the values; the long-double build is
stored beside them as a bound on their rounding error.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2407_11349_gb300 import synth  # noqa: E402

ROWS = [0, 1, 7, 500, 1234, 1999]
PARAMS = [list(synth.DEFAULT_PARAMS), [2.0, 5.0, 2.0, 0.9, 1.5, 0.7]]


def main():
    ds = synth.config_dataset("c1")
    cases = []
    for p in PARAMS:
        out, rows = oracle.loglik_grad(ds.t, ds.x, ds.y, p, s=ds.s, rows=True)
        outl = oracle.loglik_grad(ds.t, ds.x, ds.y, p, s=ds.s, precision="ld")
        cases.append({"params": p, "loglik_grad": [float(v) for v in out],
                      "loglik_grad_long_double": [float(v) for v in outl],
                      "rows": {str(i): [float(v) for v in rows[i]] for i in ROWS}})
    doc = {"workload": "c1 (synth.config_dataset('c1'): N=2000, 100 d, 20x20 grid of 50 km counties, seed 0)",
           "model": "Sec. 2.1 eqs. 2-4 with the Sec. 2.3.1 clip; gradient in (mu, tau_x, tau_t, theta, omega, h)",
           "row_fields": "ell_i, six partials, log lambda_i, Lambda_i",
           "written_by": "tests/golden/make_golden.py (FP64 oracle)", "cases": cases}
    with open(os.path.join(HERE, "oracle_c1.json"), "w") as f:
        json.dump(doc, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
