"""Writes tests/golden/oracle_small.json: the FP64 oracle's results on small seeded cases
(a 48 x 120 dictionary with 8 pixels, exactly sparse and power-law; a 24-of-64 partial
Fourier dictionary with 4 complex pixels), for the regression test of the oracle.
Calls only oracle/ and the seeded input generator.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle as orc  # noqa: E402
from paper_2401_14762_gb300 import synthetic as sy  # noqa: E402

M, N, SEED = 48, 120, 7


def inputs():
    Phi = sy.gaussian_phi(M, N, SEED)
    A = orc.dictionary(Phi)
    Xs = sy.sparse_coeffs(4, N, 6, SEED, "separated")
    Xp = sy.powerlaw_coeffs(4, N, SEED)
    X = np.vstack([Xs, Xp])
    Y = orc.measure(A, X, sy.noise(8, M, 1e-4, SEED)).astype(np.float32)
    F = (X @ orc.dct2_psi(N).T).astype(np.float32)
    return A, Y, F


def results():
    A, Y, F = inputs()
    L = orc.lipschitz(A)
    out = {"lipschitz": L}
    out["fista"] = orc.fista(A, Y, L, 1e-3, 0.0, 200)[0]
    out["admm"] = orc.admm(A, Y, 1.0, 1e-3, 0.0, 200)[0]
    for name, call in (("gomp", lambda: orc.gomp(A, Y, 8, 2)),
                       ("biht", lambda: orc.biht(A, Y, 8, 0.1)),
                       ("cosamp", lambda: orc.cosamp(A, Y, 8))):
        X, it, _ = call()
        out[name] = X
        out[name + "_iters"] = it
    Xs, k = orc.sparsify(F, 0.1)
    out["sparsify"] = Xs
    out["sparsify_kappa"] = k
    # the complex partial-Fourier setup: 24 of 64 samples, 4 complex 3-sparse pixels
    g = np.random.default_rng(SEED)
    Ac = orc.partial_fourier(24, 64, np.sort(g.choice(64, 24, replace=False)).astype(np.int32))
    Xc = np.zeros((4, 64), dtype=complex)
    for p in range(4):
        Xc[p, g.choice(64, 3, replace=False)] = np.exp(2j * np.pi * g.random(3))
    Yc = Xc @ Ac.T + 0.01 * (g.standard_normal((4, 24)) + 1j * g.standard_normal((4, 24)))
    out["cfista"] = orc.cfista(Ac, Yc, 1.0, 0.02, 0.0, 200)[0]
    out["cadmm"] = orc.cadmm(Ac, Yc, 1.0, 0.02, 0.0, 200)[0]
    for name, call in (("cgomp", lambda: orc.cgomp(Ac, Yc, 3, 1)),
                       ("cbiht", lambda: orc.cbiht(Ac, Yc, 3, 1.0)),
                       ("ccosamp", lambda: orc.ccosamp(Ac, Yc, 3))):
        X, it = call()
        out[name] = X
        out[name + "_iters"] = it
    return out


def main():
    res = {}
    for k, v in results().items():
        if isinstance(v, np.ndarray) and np.iscomplexobj(v):
            res[k] = {"re": v.real.tolist(), "im": v.imag.tolist()}
        else:
            res[k] = v.tolist() if isinstance(v, np.ndarray) else v
    res["_source"] = ("written by tests/golden/make_golden.py from the FP64 oracle: M = 48, "
                      "N = 120, seed 7, 4 exactly 6-sparse and 4 power-law pixels; complex: "
                      "24 of 64 DFT samples, 4 complex 3-sparse pixels")
    with open(os.path.join(HERE, "oracle_small.json"), "w") as f:
        json.dump(res, f, separators=(",", ":"))


if __name__ == "__main__":
    main()
