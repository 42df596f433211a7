"""The autotuner's JSON cache file, through the host-only entry points of the
C ABI (no GPU): round trip, replacement, damaged files, stale entries and
errors.  The device-side tuners that use it are covered by the GPU tests."""
import json
import os

import pytest

from paper_2407_11349_gb300 import build as libbuild


@pytest.fixture(scope="module")
def hk():
    libbuild.build()
    from paper_2407_11349_gb300 import hawkes
    return hawkes


KEY = "NVIDIA GB300|sm_103|single|n<=2^20|flags=0"


def test_round_trip_replace_and_valid_json(hk, tmp_path):
    path = str(tmp_path / "tune.json")
    assert hk.hawkes_tune_cache_get(path, KEY) is None  # no file yet
    hk.hawkes_tune_cache_put(path, KEY, 1, 16, 0, 365.4)
    hk.hawkes_tune_cache_put(path, "other|batch|P=46", 0, 64, 1, 737.56)
    assert hk.hawkes_tune_cache_get(path, KEY) == (1, 16, 0, pytest.approx(365.4))
    hk.hawkes_tune_cache_put(path, KEY, 3, 32, 1, 1.25)  # replaces, keeps the other key
    assert hk.hawkes_tune_cache_get(path, KEY) == (3, 32, 1, pytest.approx(1.25))
    assert hk.hawkes_tune_cache_get(path, "other|batch|P=46") == (0, 64, 1, pytest.approx(737.56))
    assert hk.hawkes_tune_cache_get(path, "missing") is None
    doc = json.load(open(path))  # the file is plain JSON
    assert set(doc) == {KEY, "other|batch|P=46"}
    assert doc[KEY]["variant"] == 3 and doc[KEY]["nvariants"] == hk.hawkes_sweep_variants()
    assert doc[KEY]["kc"] == 1  # chains per CTA (batches only; 1 through this entry point)
    assert not os.path.exists(path + ".tmp")


def test_damaged_and_stale_lines_are_misses(hk, tmp_path):
    path = str(tmp_path / "tune.json")
    nv = hk.hawkes_sweep_variants()
    with open(path, "w") as f:
        f.write('{\n'
                'garbage line without quotes\n'
                '"half": {"variant": 1, "chunk":\n'
                f'"stale": {{"variant": 0, "chunk": 16, "order": 0, "ms": 1.0, "nvariants": {nv + 3}}},\n'
                f'"big": {{"variant": 1e400, "chunk": 16, "order": 0, "ms": 1.0, "nvariants": {nv}}},\n'
                f'"range": {{"variant": {nv}, "chunk": 16, "order": 0, "ms": 1.0, "nvariants": {nv}}},\n'
                f'"badkc": {{"variant": 1, "chunk": 16, "order": 0, "ms": 1.0, "nvariants": {nv}, "kc": 0}},\n'
                f'"kc2": {{"variant": 1, "chunk": 16, "order": 0, "ms": 2.0, "nvariants": {nv}, "kc": 2}},\n'
                f'"good": {{"variant": 2, "chunk": 32, "order": 1, "ms": 9.5, "nvariants": {nv}}}\n'
                '}\n')
    assert hk.hawkes_tune_cache_get(path, "kc2") == (1, 16, 0, pytest.approx(2.0))
    for k in ("half", "stale", "big", "range", "badkc"):
        assert hk.hawkes_tune_cache_get(path, k) is None, k
    assert hk.hawkes_tune_cache_get(path, "good") == (2, 32, 1, pytest.approx(9.5))
    # a write rewrites the file with its valid entries only
    hk.hawkes_tune_cache_put(path, KEY, 0, 16, 0, 3.0)
    doc = json.load(open(path))
    assert "good" in doc and KEY in doc and "garbage" not in json.dumps(doc)


def test_bad_arguments_and_unwritable_path(hk, tmp_path):
    path = str(tmp_path / "tune.json")
    with pytest.raises(hk.HawkesError) as e:
        hk.hawkes_tune_cache_put(path, 'bad"key', 0, 16, 0, 1.0)
    assert e.value.status == -1
    with pytest.raises(hk.HawkesError) as e:
        hk.hawkes_tune_cache_put(path, KEY, hk.hawkes_sweep_variants(), 16, 0, 1.0)
    assert e.value.status == -1
    with pytest.raises(hk.HawkesError) as e:
        hk.hawkes_tune_cache_put(path, KEY, 0, 16, 0, float("nan"))
    assert e.value.status == -1
    with pytest.raises(hk.HawkesError) as e:
        hk.hawkes_tune_cache_get(path, "ctrl\x01char")
    assert e.value.status == -1
    with pytest.raises(hk.HawkesError) as e:
        hk.hawkes_tune_cache_put(str(tmp_path / "no_such_dir" / "tune.json"), KEY, 0, 16, 0, 1.0)
    assert e.value.status == -9
