"""The oracle against its stored values on the c1 workload
(tests/golden/oracle_c1.json, written by tests/golden/make_golden.py from
the oracle alone).  A change to the oracle's arithmetic, or to the workload
generator, shows up here; the stored long-double values bound the rounding
error of the stored FP64 ones."""
import json
import os

import numpy as np

import oracle
from paper_2407_11349_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_c1.json")


def test_oracle_reproduces_its_stored_c1_values():
    doc = json.load(open(GOLDEN))
    ds = synth.config_dataset("c1")
    for case in doc["cases"]:
        out, rows = oracle.loglik_grad(ds.t, ds.x, ds.y, case["params"], s=ds.s, rows=True)
        ref = np.array(case["loglik_grad"])
        scale = np.maximum(np.abs(ref), 1e-6 * abs(ref[0]))
        assert np.all(np.abs(out - ref) <= 1e-12 * scale), (out, ref)
        ld = np.array(case["loglik_grad_long_double"])
        assert np.all(np.abs(ref - ld) <= 1e-12 * scale)  # the stored values are FP64-accurate
        for i, vals in case["rows"].items():
            v = np.array(vals)
            assert np.all(np.abs(rows[int(i)] - v) <= 1e-12 * np.maximum(np.abs(v), 1.0)), i
