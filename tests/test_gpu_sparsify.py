"""cs_sparsify (the sparsification pre-processing of Section II) against the FP64 oracle.

Every keep/zero decision is a floating-point comparison that decides an integer outcome,
so it must be the FP64 oracle's decision exactly: the zero patterns and kappa are
compared bit for bit; the kept values agree to the FP32 transform's error bound."""
import numpy as np
import pytest

import oracle as orc
from gpu_common import exact_check, gpu_run, library, rel_l2, torch_cuda
from paper_2401_14762_gb300 import synthetic as sy

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cs():
    return library()


def spectra(P, N, seed, noise=0.01):
    """Power-law spectra f = Psi x plus white noise (the shape of the paper's cubes)."""
    X = sy.powerlaw_coeffs(P, N, seed)
    E = noise * np.random.default_rng(seed + 1000).standard_normal((P, N))
    return (X @ orc.dct2_psi(N).T + E).astype(np.float32)


def run(cs, ctx, F, T, ddof=1):
    torch = torch_cuda()
    P, N = F.shape
    Fd = torch.from_numpy(np.ascontiguousarray(F)).cuda()
    Xd = torch.full((P, N), float("nan"), device="cuda")
    kd = torch.full((P,), -1, dtype=torch.int16, device="cuda")
    rc = torch.zeros(1, dtype=torch.int64, device="cuda")
    cs.cs_sparsify(ctx, Fd, Xd, T, ddof, kappa_out=kd, recomputed_out=rc)
    cs.cs_sync(ctx)
    return Xd.cpu().numpy(), kd.cpu().numpy().astype(np.int32), int(rc.item())


def check(Xg, kg, Xo, ko, F):
    assert np.array_equal(Xg != 0, Xo != 0), f"{(( Xg != 0) != (Xo != 0)).sum()} decisions differ"
    assert np.array_equal(kg, ko)
    # kept values: within the FP32 transform bound (gamma_N + 2u) ||f|| per coefficient
    N = F.shape[1]
    u = 2.0 ** -24
    bound = (N * u / (1 - N * u) + 2 * u) * np.linalg.norm(F.astype(np.float64), axis=1)
    assert np.all(np.abs(Xg - Xo) <= bound[:, None] + 1e-30)
    assert rel_l2(Xg, Xo) <= 1e-6


@pytest.mark.parametrize("N", [120, 200, 224, 256])
@pytest.mark.parametrize("T,ddof", [(0.1, 1), (0.5, 0), (-0.2, 1)])
def test_sparsify_matches_oracle(cs, N, T, ddof):
    M = (2 * N) // 5
    ctx = cs.cs_create(M, N, Phi=sy.gaussian_phi(M, N, 3))
    F = spectra(1037, N, N + 7)  # several warp passes and a ragged tail
    F[5] = 0.0                   # a zero spectrum: nothing kept, kappa 0
    Xg, kg, _ = run(cs, ctx, F, T, ddof)
    Xo, ko = orc.sparsify(F, T, ddof)
    check(Xg, kg, Xo, ko, F)
    assert kg[5] == 0 and not Xg[5].any()
    assert np.isfinite(Xg).all()


@pytest.mark.parametrize("N,offset", [(50, 0), (120, 1), (129, 3)])
def test_sparsify_odd_shapes_and_unaligned_output(cs, N, offset):
    """N not a multiple of 4, or X starting off a 16-byte boundary: the rows are written
    element by element; N = 129 uses the two-float4-per-lane layout with one column."""
    torch = torch_cuda()
    M = max(1, (2 * N) // 5)
    ctx = cs.cs_create(M, N, Phi=sy.gaussian_phi(M, N, 4))
    F = spectra(333, N, N + 1)
    Fd = torch.from_numpy(F).cuda()
    buf = torch.full((F.size + offset,), float("nan"), device="cuda")
    Xd = buf[offset:].view(F.shape)
    kd = torch.zeros(F.shape[0], dtype=torch.int16, device="cuda")
    cs.cs_sparsify(ctx, Fd, Xd, 0.1, 1, kappa_out=kd)
    cs.cs_sync(ctx)
    Xo, ko = orc.sparsify(F, 0.1)
    check(Xd.cpu().numpy(), kd.cpu().numpy().astype(np.int32), Xo, ko, F)
    assert torch.isnan(buf[:offset]).all()


def test_sparsify_ties_are_decided_in_fp64(cs):
    """With Psi = I the FP32 transform is exact and ties at the threshold are exact:
    those pixels must go through the FP64 path and keep every tied coefficient
    (only |x_i| - mu < T sigma zeroes), as the hand-worked cases of the oracle pins."""
    N = 8
    ctx = cs.cs_create(4, N, Phi=sy.gaussian_phi(4, N, 1), Psi=np.eye(N))
    F = np.array([[3, 1, 2, -2, 2, 2, 1, 3],      # mean |f| = 2: four ties at T = 0
                  [4, -2, 1, 0, 0, 0, 0, 0],
                  [0, 0, 0, 0, 0, 0, 0, 0]], dtype=np.float32)
    Xg, kg, rec = run(cs, ctx, F, 0.0)
    Xo, ko = orc.sparsify(F, 0.0, 1, np.eye(N))
    assert np.array_equal(Xg, Xo.astype(np.float32)) and np.array_equal(kg, ko)
    assert np.array_equal(Xg[0], [3, 0, 2, -2, 2, 2, 0, 3])
    assert rec >= 2  # the tied row and the zero row


def test_sparsify_full_cube_sampled(cs):
    """512 x 512 pixels of N = 200 spectra, T = 0.1: decisions on a sample of pixels spread
    over the cube equal the oracle's, and only a small share of pixels needed FP64."""
    torch = torch_cuda()
    P, N, M = 512 * 512, 200, 80
    ctx = cs.cs_create(M, N, Phi=sy.gaussian_phi(M, N, 1))
    F = spectra(P, N, 11)
    Xg, kg, rec = run(cs, ctx, F, 0.1)
    idx = np.random.default_rng(5).choice(P, 3000, replace=False)
    idx = np.concatenate([idx, [0, P - 1]])
    Xo, ko = orc.sparsify(F[idx], 0.1)
    check(Xg[idx], kg[idx], Xo, ko, F[idx])
    assert rec < P // 20
    del torch


def test_sparsify_then_recover(cs):
    """The pipeline of the paper: sparsify, measure at 2.5x, recover with gOMP using the
    per-pixel kappa that sparsification produced (G = max(1, kappa / 5)): the greedy
    result equals the oracle's gOMP on the same measurements pixel for pixel."""
    torch = torch_cuda()
    P, N, M = 600, 200, 80
    ctx = cs.cs_create(M, N, Phi=sy.gaussian_phi(M, N, 9))
    F = spectra(P, N, 12)
    Xs, ks, _ = run(cs, ctx, F, 0.1)  # about 93% of the coefficients zeroed, kappa 8..20
    Xo, ko = orc.sparsify(F, 0.1)
    check(Xs, ks, Xo, ko, F)
    A = orc.dictionary(sy.gaussian_phi(M, N, 9))
    Y = orc.measure(A, Xs.astype(np.float64)).astype(np.float32)
    kmax = int(ks.max())
    assert 0 < kmax <= 32
    Xg, itg, _ = gpu_run(cs.cs_recover_gomp, ctx, Y, N, kmax, 0, kappa_pp=ks)
    Xr = np.zeros((P, N))
    itr = np.zeros(P, dtype=np.int32)
    for k in np.unique(ks):
        sel = ks == k
        Xr[sel], itr[sel], _ = orc.gomp(A, Y[sel], int(k), max(1, int(k) // 5))
    exact_check(Xg, itg, Xr, itr, kmax)
    del torch


def test_sparsify_argument_errors(cs):
    torch = torch_cuda()
    A = orc.dictionary(sy.gaussian_phi(8, 20, 1))
    ctx_a = cs.cs_create(8, 20, A=A)  # made from A: no Psi
    ctx = cs.cs_create(8, 20, Phi=sy.gaussian_phi(8, 20, 1))
    F = torch.zeros((4, 20), device="cuda")
    X = torch.zeros((4, 20), device="cuda")
    for c, args in ((ctx_a, (F, X, 0.1, 1)), (ctx, (F, X, 0.1, 2)),
                    (ctx, (F, X, float("nan"), 1)), (ctx, (F.cpu().numpy(), X, 0.1, 1))):
        with pytest.raises(cs.CsError) as e:
            cs.cs_sparsify(c, *args)
        assert e.value.status == cs.CS_ERR_ARG
    cs.cs_sparsify(ctx, F[:0], X[:0], 0.1)  # P = 0 is a no-op
    cs.cs_sync(ctx)
