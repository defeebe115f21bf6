"""The paper's complex setup (Section II: Psi the unitary DFT, Phi keeping M spectral
samples) on the GPU: a context from cs_create_complex runs FISTA and ADMM on the real
form of A with thresholds on the moduli, against the FP64 complex oracle."""
import numpy as np
import pytest

import oracle as orc
from gpu_common import library, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cs():
    return library()


def _problem(M, N, P, seed, S=5, noise=0.01):
    g = np.random.default_rng(seed)
    rows = np.sort(g.choice(N, M, replace=False)).astype(np.int32)
    A = orc.partial_fourier(M, N, rows)
    X = np.zeros((P, N), dtype=np.complex128)
    for p in range(P):
        X[p, g.choice(N, S, replace=False)] = (0.5 + g.random(S)) * np.exp(2j * np.pi * g.random(S))
    Y = X @ A.T + noise * (g.standard_normal((P, M)) + 1j * g.standard_normal((P, M)))
    return A, Y.astype(np.complex64)


def rel_l2(X, ref):
    return float(np.linalg.norm(X - ref) / np.linalg.norm(ref))


def _run(cs, call, ctx, Y, N, *args, **kw):
    torch = torch_cuda()
    P = Y.shape[0]
    Yd = torch.from_numpy(np.ascontiguousarray(Y).view(np.float32)).cuda()
    Xd = torch.full((P, 2 * N), float("nan"), device="cuda")
    call(ctx, Yd, Xd, *args, opts=cs.make_opts(**kw))
    cs.cs_sync(ctx)
    return Xd.cpu().numpy().view(np.complex64).astype(np.complex128)


def _tolerance(run, Y, iters, rel=1e-7):
    """FP32 tolerance of an iterate after `iters` iterations: the oracle's own output
    change per unit relative perturbation of y (measured), times K rounding injections
    of 2^-24 adding up like sqrt(K); never below the FP32 path's 1e-5."""
    Yp = Y * (1.0 + rel * np.random.default_rng(0).standard_normal(Y.shape))
    X0, X1 = run(Y), run(Yp)
    cond = np.linalg.norm(X1 - X0) / np.linalg.norm(X0) / rel
    return max(1e-5, 4.0 * np.sqrt(iters) * cond * 2.0 ** -24)


def test_complex_fista_matches_oracle(cs):
    M, N, P = 24, 64, 37 * 3 + 2
    A, Y = _problem(M, N, P, 1)
    ctx = cs.cs_create_complex(M, N, A)
    L = cs.cs_get_lipschitz(ctx)
    assert abs(L - 1.0) < 1e-10  # orthonormal rows
    Yc = Y.astype(np.complex128)
    for iters in (60, 1500):
        Xg = _run(cs, cs.cs_recover_fista, ctx, Y, N, 0.02, iters, eps=0.0)
        run = lambda y: orc.cfista(A, y, L, 0.02, 0.0, iters)[0]  # noqa: E731
        tol = _tolerance(run, Yc[:32], iters)
        assert rel_l2(Xg, run(Yc)) <= tol, (iters, rel_l2(Xg, run(Yc)), tol)


def test_complex_admm_matches_oracle(cs):
    M, N, P = 24, 64, 70
    A, Y = _problem(M, N, P, 2)
    ctx = cs.cs_create_complex(M, N, A, admm_rho=1.0)
    Yc = Y.astype(np.complex128)
    Xg = _run(cs, cs.cs_recover_admm, ctx, Y, N, 1.0, 0.02, 300, eps=0.0)
    run = lambda y: orc.cadmm(A, y, 1.0, 0.02, 0.0, 300)[0]  # noqa: E731
    assert rel_l2(Xg, run(Yc)) <= _tolerance(run, Yc[:32], 300)


def test_complex_full_dft_closed_form(cs):
    """With the full unitary DFT the LASSO solution is modulus-soft(Psi^H y, lambda)."""
    N = 32
    Psi = orc.dft_psi(N)
    g = np.random.default_rng(3)
    Y = (g.standard_normal((40, N)) + 1j * g.standard_normal((40, N))).astype(np.complex64)
    ctx = cs.cs_create_complex(N, N, Psi)
    Xg = _run(cs, cs.cs_recover_fista, ctx, Y, N, 0.3, 20, eps=0.0)
    a = np.fft.ifft(Y.astype(np.complex128), norm="ortho", axis=1)
    ref = np.maximum(np.abs(a) - 0.3, 0.0) * np.exp(1j * np.angle(a))
    assert np.abs(Xg - ref).max() < 1e-5


def test_complex_measure_and_precision_option(cs):
    torch = torch_cuda()
    M, N, P = 24, 64, 50
    A, Y = _problem(M, N, P, 4)
    ctx = cs.cs_create_complex(M, N, A)
    g = np.random.default_rng(5)
    X = (g.standard_normal((P, N)) + 1j * g.standard_normal((P, N))).astype(np.complex64)
    Xd = torch.from_numpy(X.view(np.float32)).cuda()
    Yd = torch.empty((P, 2 * M), device="cuda")
    cs.cs_measure(ctx, Xd, Yd)
    cs.cs_sync(ctx)
    Yg = Yd.cpu().numpy().view(np.complex64)
    ref = X.astype(np.complex128) @ A.T
    assert np.abs(Yg - ref).max() <= 1e-5 * np.abs(ref).max()
    # the tensor-core path is for real contexts: the BF16 option runs the same FP32 path
    a = _run(cs, cs.cs_recover_fista, ctx, Y, N, 0.02, 40, eps=0.0, prec=cs.CS_BF16)
    b = _run(cs, cs.cs_recover_fista, ctx, Y, N, 0.02, 40, eps=0.0)
    assert np.array_equal(a, b)


def test_complex_context_errors(cs):
    torch = torch_cuda()
    M, N = 24, 64
    A, Y = _problem(M, N, 4, 6)
    ctx = cs.cs_create_complex(M, N, A)
    Yd = torch.from_numpy(Y.view(np.float32)).cuda()
    Xd = torch.zeros((4, 2 * N), device="cuda")
    for call, args in ((cs.cs_recover_gomp, (4, 1)), (cs.cs_recover_cosamp, (4,)),
                       (cs.cs_recover_biht, (4,))):
        with pytest.raises(cs.CsError) as e:
            call(ctx, Yd, Xd, *args)
        assert e.value.status == cs.CS_ERR_ARG
    with pytest.raises(cs.CsError) as e:
        cs.cs_sparsify(ctx, Xd, Xd, 0.1)
    assert e.value.status == cs.CS_ERR_ARG
    with pytest.raises(cs.CsError) as e:
        cs.cs_create_complex(65, 128, np.zeros((65, 128), dtype=np.complex128))
    assert e.value.status == cs.CS_ERR_SHAPE
