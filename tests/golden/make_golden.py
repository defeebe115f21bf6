"""Writes tests/golden/oracle_small.json: the FP64 oracle's results on a small seeded case
(48 x 120 dictionary, 8 pixels: exactly sparse and power-law), for the regression test
of the oracle.  Calls only oracle/ and the seeded input generator.

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
    return out


def main():
    res = {k: (v.tolist() if isinstance(v, np.ndarray) else v) for k, v in results().items()}
    res["_source"] = ("written by tests/golden/make_golden.py from the FP64 oracle: M = 48, "
                      "N = 120, seed 7, 4 exactly 6-sparse and 4 power-law pixels")
    with open(os.path.join(HERE, "oracle_small.json"), "w") as f:
        json.dump(res, f, separators=(",", ":"))


if __name__ == "__main__":
    main()
