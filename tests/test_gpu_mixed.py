"""Mixed-precision (tensor-core) path against the FP64 oracle.

prec = CS_BF16 runs FISTA's two products on the tcgen05 tensor cores with split-BF16
operands (hi*hi + lo*hi + hi*lo, FP32 accumulation).  The bar is relative L2 <= 1e-3
against the FP64 oracle; at fixed, unconverged iteration counts on the ill-conditioned
sparse case the FP32-path tolerance derived from the oracle's conditioning applies when
it is looser.
"""
import numpy as np
import pytest

import oracle as orc
from gpu_common import (Problem, fixed_iteration_tolerance, gpu_run, iterate_conditioning,
                        library, rel_l2, support)

pytestmark = pytest.mark.gpu
REL_L2_MIXED = 1e-3


@pytest.fixture(scope="module")
def cs():
    return library()


@pytest.mark.parametrize("shape,kind,iters,P", [((80, 200), "powerlaw", 300, 32 * 20 + 7),
                                                ((48, 120), "powerlaw", 300, 300),
                                                ((90, 224), "powerlaw", 300, 200)])
def test_fista_bf16_powerlaw(cs, shape, kind, iters, P):
    M, N = shape
    pr = Problem(M, N, P, kind, seed=3, noise_var=1e-3)
    Xo, _ = orc.fista(pr.A, pr.Y, pr.L, 1e-3, 0.0, iters)
    ctx = cs.cs_create(M, N, Phi=pr.Phi)
    Xb, it, cv = gpu_run(cs.cs_recover_fista, ctx, pr.Y, N, 1e-3, iters, eps=0.0,
                         prec=cs.CS_BF16)
    Xf, _, _ = gpu_run(cs.cs_recover_fista, ctx, pr.Y, N, 1e-3, iters, eps=0.0)
    err, err32 = rel_l2(Xb, Xo), rel_l2(Xf, Xo)
    print(f"bf16 {err:.2e} fp32 {err32:.2e}")
    assert np.all(it == iters) and np.all(cv == 0)
    assert err <= REL_L2_MIXED


def test_fista_bf16_small_sparse(cs):
    pr = Problem(48, 120, 32 * 32 + 7, "sparse", seed=1, S=8)
    run = lambda Y: orc.fista(pr.A, Y, pr.L, 1e-3, 0.0, 500)[0]
    Xo = run(pr.Y)
    tol = max(REL_L2_MIXED, fixed_iteration_tolerance(iterate_conditioning(run, pr.Y[:128]), 500))
    ctx = cs.cs_create(pr.M, pr.N, Phi=pr.Phi)
    Xb, it, _ = gpu_run(cs.cs_recover_fista, ctx, pr.Y, pr.N, 1e-3, 500, eps=0.0,
                        prec=cs.CS_BF16)
    print(f"bf16 {rel_l2(Xb, Xo):.2e} tol {tol:.2e}")
    assert rel_l2(Xb, Xo) <= tol


@pytest.mark.parametrize("lam", [0.05, 0.02])
def test_fista_bf16_converged(cs, lam):
    pr = Problem(48, 120, 200, "sparse", seed=21, S=6, noise_var=1e-4)
    Xo, _ = orc.fista(pr.A, pr.Y, pr.L, lam, 0.0, 20000)
    ctx = cs.cs_create(pr.M, pr.N, Phi=pr.Phi)
    Xb, it, cv = gpu_run(cs.cs_recover_fista, ctx, pr.Y, pr.N, lam, 20000, eps=1e-7,
                         prec=cs.CS_BF16)
    print(f"bf16 converged {rel_l2(Xb, Xo):.2e} iters {it.mean():.0f}")
    assert rel_l2(Xb, Xo) <= REL_L2_MIXED
    # supports at the resolution the mixed path targets (BF16 x 3 keeps ~16 bits)
    assert np.all(support(Xb, 1e-3) == support(Xo, 1e-3))


def test_fista_bf16_stop_rule_and_edges(cs):
    """Delta stopping per pixel, eps > 1, zero iterations, a ragged single pixel."""
    pr = Problem(80, 200, 129, "powerlaw", seed=4, noise_var=1e-3)
    ctx = cs.cs_create(pr.M, pr.N, Phi=pr.Phi)
    Xo, ito = orc.fista(pr.A, pr.Y, pr.L, 0.05, 1e-4, 3000)
    Xb, it, cv = gpu_run(cs.cs_recover_fista, ctx, pr.Y, pr.N, 0.05, 3000, eps=1e-4,
                         prec=cs.CS_BF16)
    assert np.all(cv == 1)
    assert np.abs(it.astype(int) - ito.astype(int)).max() <= max(3, int(0.05 * ito.max()))
    assert rel_l2(Xb, Xo) <= REL_L2_MIXED
    Xb, it, _ = gpu_run(cs.cs_recover_fista, ctx, pr.Y, pr.N, 0.05, 100, eps=2.0,
                        prec=cs.CS_BF16)
    assert np.all(Xb == 0) and np.all(it == 0)
    Xb, it, _ = gpu_run(cs.cs_recover_fista, ctx, pr.Y, pr.N, 0.05, 0, eps=0.0,
                        prec=cs.CS_BF16)
    assert np.all(Xb == 0) and np.all(it == 0)
    Xo1, _ = orc.fista(pr.A, pr.Y[:1], pr.L, 1e-3, 0.0, 50)
    Xb1, _, _ = gpu_run(cs.cs_recover_fista, ctx, pr.Y[:1], pr.N, 1e-3, 50, eps=0.0,
                        prec=cs.CS_BF16)
    assert rel_l2(Xb1, Xo1) <= REL_L2_MIXED
