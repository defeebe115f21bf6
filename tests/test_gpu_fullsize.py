"""The bench's workloads at full size, in the launch configuration bench.py times: the
2048 x 2048 x 256 cube (M = 102) of the headline and the 1024 x 1024 x 224 cube (M = 90)
beside it, measured on the GPU (the sampled measurements checked against the oracle's)
and every pixel recovered by all five algorithms with the bench's options (FISTA and ADMM on the mixed path where a tensor-core tile exists).
384 pixels spread over the cube, plus its first and last, are recovered by the FP64
oracle from the same FP32 measurements: the greedy pixels must follow the oracle's
trajectories exactly, FISTA and ADMM stay within the metric's rel-L2 of 1e-3."""
import os
import sys

import numpy as np
import pytest

import oracle as orc
from gpu_common import exact_check, library, rel_l2, torch_cuda

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402  (the workload's constants)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cs():
    return library()


WORKLOADS = {"2048x2048x256": (bench.M, bench.N, bench.SIDE, bench.KAPPA, bench.G),
             "1024x1024x224": (bench.CTX["M"], bench.CTX["N"], bench.CTX["SIDE"],
                               bench.CTX["KAPPA"], bench.CTX["G"])}


@pytest.mark.parametrize("workload", list(WORKLOADS))
def test_full_cube_sampled_against_oracle(cs, workload):
    torch = torch_cuda()
    from paper_2401_14762_gb300 import synthetic as sy
    M, N, side, KAPPA, G = WORKLOADS[workload]
    P = side * side
    dev = torch.device("cuda", 0)
    Phi = sy.gaussian_phi(M, N, bench.SEED)
    Xt = sy.powerlaw_coeffs_torch(P, N, bench.SEED, dev)
    E = sy.noise_torch(P, M, bench.NOISE_VAR, bench.SEED, dev)
    ctx = cs.cs_create(M, N, Phi=Phi, admm_rho=bench.RHO)
    Y = torch.empty((P, M), device=dev)
    cs.cs_measure(ctx, Xt, Y, E)
    out, its = {}, {}
    for a in ("fista", "admm", "gomp", "biht", "cosamp"):
        X = torch.empty((P, N), device=dev)
        it = torch.full((P,), -1, dtype=torch.int32, device=dev)
        if a == "fista":
            cs.cs_recover_fista(ctx, Y, X, bench.LAM, bench.ITERS,
                                cs.make_opts(eps=bench.EPS, prec=cs.CS_BF16, iters_out=it))
        elif a == "admm":
            cs.cs_recover_admm(ctx, Y, X, bench.RHO, bench.LAM, bench.ITERS,
                               cs.make_opts(eps=bench.EPS, prec=cs.CS_BF16, iters_out=it))
        elif a == "gomp":
            cs.cs_recover_gomp(ctx, Y, X, KAPPA, G,
                               cs.make_opts(eps=bench.EPS, iters_out=it))
        elif a == "biht":
            cs.cs_recover_biht(ctx, Y, X, KAPPA,
                               cs.make_opts(eps=bench.EPS, mu=bench.MU, iters_out=it))
        else:
            cs.cs_recover_cosamp(ctx, Y, X, KAPPA,
                                 cs.make_opts(eps=bench.EPS, iters_out=it))
        out[a], its[a] = X, it
    cs.cs_sync(ctx)
    idx = np.unique(np.concatenate([np.random.default_rng(3).choice(P, 384, replace=False),
                                    [0, P - 1]]))
    sel = torch.from_numpy(idx).to(dev)
    Ys = Y[sel].cpu().numpy()  # the FP32 measurements both sides recover from
    A = orc.dictionary(Phi)
    L = orc.lipschitz(A)
    # the measurement itself (the TMA-fed tiled kernel over the whole cube) at the samples
    Yo = orc.measure(A, Xt[sel].cpu().double().numpy(), E[sel].cpu().double().numpy())
    assert (np.abs(Ys - Yo) / np.linalg.norm(Yo, axis=1, keepdims=True)).max() < 1e-6
    g = {a: out[a][sel].cpu().numpy() for a in out}
    gi = {a: its[a][sel].cpu().numpy() for a in its}
    ef = rel_l2(g["fista"], orc.fista(A, Ys, L, bench.LAM, bench.EPS, bench.ITERS)[0])
    ea = rel_l2(g["admm"], orc.admm(A, Ys, bench.RHO, bench.LAM, bench.EPS, bench.ITERS)[0])
    print(f"{workload}: FISTA rel-L2 {ef:.2e}, ADMM rel-L2 {ea:.2e}")
    assert ef <= 1e-3 and ea <= 1e-3
    Xo, ito, _ = orc.gomp(A, Ys, KAPPA, G, bench.EPS)
    exact_check(g["gomp"], gi["gomp"], Xo, ito, KAPPA)
    Xo, ito, _ = orc.biht(A, Ys, KAPPA, bench.MU, bench.EPS, 100)
    exact_check(g["biht"], gi["biht"], Xo, ito, KAPPA)
    Xo, ito, _ = orc.cosamp(A, Ys, KAPPA, bench.EPS, 100)
    exact_check(g["cosamp"], gi["cosamp"], Xo, ito, KAPPA)
    cs.cs_destroy(ctx)
