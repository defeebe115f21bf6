"""Shared helpers of the GPU parity tests: problem generation (oracle-made inputs) and
runners that call the CUDA library through its C ABI."""
from __future__ import annotations

import numpy as np
import pytest

import oracle as orc
from paper_2401_14762_gb300 import synthetic as sy

# Tolerances.  FP32 path: relative L2 <= 1e-5 against the FP64 oracle.  Supports of
# greedy methods must be identical on pixels whose oracle selection margin (relative
# gap between the k-th and (k+1)-th magnitude at every selection) exceeds 1e-3, the
# FP32 resolution with headroom.
REL_L2_FP32 = 1e-5
MARGIN_FP32 = 1e-3
U32 = 2.0 ** -24  # FP32 unit roundoff


def support(X, rel=1e-6):
    """Support of each row: {j : |x_j| > rel max|x|} (entries at rounding level excluded)."""
    X = np.abs(np.asarray(X, np.float64))
    return X > rel * X.max(axis=1, keepdims=True)


def iterate_conditioning(run, Y, rel=1e-7, seed=0):
    """Relative change of the oracle's output per unit relative perturbation of y."""
    Y = np.asarray(Y, np.float64)
    Yp = Y * (1.0 + rel * np.random.default_rng(seed).standard_normal(Y.shape))
    X0, X1 = run(Y), run(Yp)
    return np.linalg.norm(X1 - X0) / np.linalg.norm(X0) / rel


TOL_CAP = 1e-3  # no parity test accepts a FISTA/ADMM iterate further than this


def fixed_iteration_tolerance(cond, iters):
    """FP32 tolerance for an iterate after `iters` unconverged iterations: each iteration
    adds O(u32) relative rounding, propagated with the measured conditioning; K
    independent injections add up like sqrt(K).  Never below the FP32 path's 1e-5 and
    never above 1e-3 (the metric's bar): a case whose conditioning would allow more must
    still meet 1e-3.  Prints the tolerance it returns."""
    tol = min(TOL_CAP, max(REL_L2_FP32, 4.0 * np.sqrt(iters) * cond * U32))
    print(f"fixed-iteration tolerance {tol:.2e} (measured conditioning {cond:.0f}, "
          f"{iters} iterations)")
    return tol


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def library():
    torch_cuda()
    from paper_2401_14762_gb300 import build, cs
    build.build()
    return cs


class Problem:
    def __init__(self, M, N, P, kind="sparse", seed=1, S=8, noise_var=0.0, amplitude="normal"):
        self.M, self.N, self.P = M, N, P
        self.Phi = sy.gaussian_phi(M, N, seed)
        self.A = orc.dictionary(self.Phi)
        if kind == "sparse":
            self.Xt = sy.sparse_coeffs(P, N, S, seed, amplitude)
        else:
            self.Xt = sy.powerlaw_coeffs(P, N, seed)
        self.E = sy.noise(P, M, noise_var, seed)
        # the measurements both sides recover from: oracle FP64 measurement, stored FP32
        self.Y = orc.measure(self.A, self.Xt, self.E).astype(np.float32)
        self.L = orc.lipschitz(self.A)


def rel_l2(X, ref):
    d = np.linalg.norm(ref)
    return float(np.linalg.norm(np.asarray(X, np.float64) - ref) / (d if d > 0 else 1.0))


def gpu_run(call, ctx, Y, N, *args, eps=1e-8, max_iters=100, prec=0, mu=0.1, kappa_pp=None,
            cycle_skip=True):
    """Runs one recovery call on device copies of Y; returns (X, iters, converged) on host."""
    torch = torch_cuda()
    from paper_2401_14762_gb300 import cs
    P = Y.shape[0]
    Yd = torch.from_numpy(np.ascontiguousarray(Y)).cuda()
    Xd = torch.full((P, N), float("nan"), device="cuda", dtype=torch.float32)
    it = torch.full((P,), -1, device="cuda", dtype=torch.int32)
    cv = torch.full((P,), 255, device="cuda", dtype=torch.uint8)
    kp = None if kappa_pp is None else torch.from_numpy(kappa_pp.astype(np.int16)).cuda()
    opts = cs.make_opts(eps=eps, max_iters=max_iters, prec=prec, mu=mu, iters_out=it,
                        converged_out=cv, kappa_per_pixel=kp, cycle_skip=cycle_skip)
    call(ctx, Yd, Xd, *args, opts=opts)
    cs.cs_sync(ctx)
    return Xd.cpu().numpy(), it.cpu().numpy(), cv.cpu().numpy()


def exact_check(Xg, it, Xo, ito, kappa):
    """Greedy parity on every pixel: the GPU certifies each top-k choice against FP64,
    so supports and iteration counts equal the oracle's and the values agree to FP32
    output rounding (cube rel-L2 <= 1e-5), near-tied or not."""
    assert np.all((Xg != 0).sum(1) <= kappa)
    same = np.all(support(Xg) == support(Xo), axis=1)
    assert same.all(), f"{(~same).sum()} of {len(same)} pixels differ in support"
    assert np.array_equal(it, ito), f"{(it != ito).sum()} pixels differ in iterations"
    assert rel_l2(Xg, Xo) <= REL_L2_FP32


def support_check(Xg, Xo, margins, kappa, margin_min=MARGIN_FP32):
    """Greedy parity: every output kappa-sparse; identical supports and values within the
    FP32 tolerance on well-separated pixels.  Returns the well-separated mask."""
    assert np.all((Xg != 0).sum(1) <= kappa)
    sep = margins > margin_min
    assert sep.sum() >= min(20, len(sep)), f"too few well-separated pixels ({sep.sum()})"
    same = np.all(support(Xg[sep]) == support(Xo[sep]), axis=1)
    assert same.all(), f"{(~same).sum()} well-separated pixels differ in support"
    assert rel_l2(Xg[sep], Xo[sep]) <= REL_L2_FP32
    return sep
