"""Stored fixtures (CPU only).

- oracle_small.json, written by tests/golden/make_golden.py from the FP64 oracle: the
  oracle must keep reproducing it (a regression check; its correctness is what the pins
  establish), with iteration counts and supports exact and values to 1e-9 (the oracle is
  compiled on x86 and Arm, whose compilers may contract a*b+c differently).
- paper_parameters.json: the parameters Section III states, against the library's
  defaults and the bench's configuration.
"""
import json
import os
import sys

import numpy as np

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
sys.path.insert(0, HERE)


def test_oracle_reproduces_stored_results():
    import make_golden
    ref = json.load(open(os.path.join(HERE, "oracle_small.json")))
    got = make_golden.results()
    assert abs(got["lipschitz"] - ref["lipschitz"]) <= 1e-12 * ref["lipschitz"]
    for k in ("gomp_iters", "biht_iters", "cosamp_iters", "sparsify_kappa"):
        assert np.array_equal(got[k], np.array(ref[k])), k
    for k in ("cgomp_iters", "cbiht_iters", "ccosamp_iters"):
        assert np.array_equal(got[k], np.array(ref[k])), k
    for k in ("cfista", "cadmm", "cgomp", "cbiht", "ccosamp"):
        r = np.array(ref[k]["re"]) + 1j * np.array(ref[k]["im"])
        if k not in ("cfista", "cadmm"):
            assert np.array_equal(got[k] != 0, r != 0), k
        assert np.abs(got[k] - r).max() <= 1e-9 * max(1.0, np.abs(r).max()), k
    for k in ("fista", "admm", "gomp", "biht", "cosamp", "sparsify"):
        r = np.array(ref[k])
        if k not in ("fista", "admm"):  # supports and kept sets exactly
            assert np.array_equal(got[k] != 0, r != 0), k
        assert np.abs(got[k] - r).max() <= 1e-9 * max(1.0, np.abs(r).max()), k


def test_defaults_follow_the_paper():
    par = json.load(open(os.path.join(HERE, "paper_parameters.json")))
    from paper_2401_14762_gb300 import build, cs
    build.build()
    cs.load_library()
    o = cs.cs_opts_default()
    assert o.eps == par["eps"]["value"] and o.mu == par["mu"]["value"]
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    assert bench.EPS == par["eps"]["value"] and bench.MU == par["mu"]["value"]
    assert bench.G == bench.KAPPA // 5                       # G = floor(kappa / 5)
    assert bench.M == round(par["compression"]["value"] * bench.N)
