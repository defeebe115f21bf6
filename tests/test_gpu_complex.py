"""The paper's complex setup (Section II: Psi the unitary DFT, Phi keeping M spectral
samples) on the GPU: a context from cs_create_complex runs FISTA and ADMM on the real
form of A with thresholds on the moduli, and gOMP, BIHT and CoSaMP with each complex atom
a column pair of the real form, selected by modulus, against the FP64 complex oracle."""
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
    with pytest.raises(cs.CsError) as e:
        cs.cs_sparsify(ctx, Xd, Xd, 0.1)
    assert e.value.status == cs.CS_ERR_ARG
    with pytest.raises(cs.CsError) as e:
        cs.cs_create_complex(65, 128, np.zeros((65, 128), dtype=np.complex128))
    assert e.value.status == cs.CS_ERR_SHAPE


def _greedy(cs, ctx, algo, Y, N, kappa, G=2, mu=1.0):
    torch = torch_cuda()
    P = Y.shape[0]
    Yd = torch.from_numpy(np.ascontiguousarray(Y).view(np.float32)).cuda()
    Xd = torch.full((P, 2 * N), float("nan"), device="cuda")
    it = torch.full((P,), -1, device="cuda", dtype=torch.int32)
    opts = cs.make_opts(mu=mu, iters_out=it)
    if algo == "gomp":
        cs.cs_recover_gomp(ctx, Yd, Xd, kappa, G, opts)
    elif algo == "biht":
        cs.cs_recover_biht(ctx, Yd, Xd, kappa, opts)
    else:
        cs.cs_recover_cosamp(ctx, Yd, Xd, kappa, opts)
    cs.cs_sync(ctx)
    X = Xd.cpu().numpy().view(np.complex64).astype(np.complex128)
    return X, it.cpu().numpy()


@pytest.mark.parametrize("algo,noise", [("gomp", 0.01), ("biht", 0.01), ("cosamp", 0.01),
                                        ("gomp", 0.0), ("biht", 0.0)])
def test_complex_greedy_matches_oracle(cs, algo, noise):
    """gOMP, BIHT and CoSaMP on complex data: the real form of A with each complex atom
    the column pair (2j, 2j + 1), selected and pruned by its modulus (certified against
    the FP64 modulus).  Every pixel takes the complex oracle's support and iteration
    count, and the cube is within the FP32 path's rel-L2 of 1e-5; noiseless 4-sparse
    pixels at 2.5x are recovered exactly.  (Noiseless CoSaMP is left out: once its
    residual vanishes the complex oracle's Householder least squares, which has no
    rank-deficient fallback, refuses some of the unions it then forms.)"""
    M, N, P = 24, 64, 37 * 3 + 2
    A, Y = _problem(M, N, P, 11 + int(noise > 0), S=4, noise=noise)
    ctx = cs.cs_create_complex(M, N, A)
    Yc = Y.astype(np.complex128)
    kappa = 6
    if algo == "gomp":
        Xo, ito = orc.cgomp(A, Yc, kappa, 2)
    elif algo == "biht":
        Xo, ito = orc.cbiht(A, Yc, kappa, mu=1.0)
    else:
        Xo, ito = orc.ccosamp(A, Yc, kappa)
    Xg, it = _greedy(cs, ctx, algo, Y, N, kappa)
    sup = lambda X: np.abs(X) > 1e-6 * np.abs(X).max(axis=1, keepdims=True)  # noqa: E731
    same = np.all(sup(Xg) == sup(Xo), axis=1)
    assert same.all(), f"{(~same).sum()} of {P} pixels differ in support"
    assert np.array_equal(it, ito), f"{(it != ito).sum()} pixels differ in iterations"
    assert np.all((np.abs(Xg) > 0).sum(axis=1) <= kappa)
    err = rel_l2(Xg, Xo)
    print(f"complex {algo} noise {noise}: rel-L2 {err:.2e}, iterations {it.min()}..{it.max()}")
    assert err <= 1e-5


def test_complex_greedy_in_streams_and_batches(cs):
    """The complex greedy methods in cs_recover_stream (ragged chunks, pinned host memory)
    and in cs_recover_batch (two complex cubes of different shapes) give the single
    calls' X and iteration counts bit for bit; a batch mixing complex and real contexts,
    and kappa above the complex N, are refused."""
    torch = torch_cuda()
    shapes = [(24, 64, 37), (30, 100, 50)]
    probs = [_problem(M, N, P, 20 + i, S=4) for i, (M, N, P) in enumerate(shapes)]
    ctxs = [cs.cs_create_complex(M, N, A) for (M, N, _), (A, _) in zip(shapes, probs)]
    singles = {}
    for algo, code in (("gomp", cs.CS_ALGO_GOMP), ("biht", cs.CS_ALGO_BIHT),
                       ("cosamp", cs.CS_ALGO_COSAMP)):
        for i, ((M, N, P), (A, Y), ctx) in enumerate(zip(shapes, probs, ctxs)):
            singles[algo, i] = _greedy(cs, ctx, algo, Y, N, 6)
        # stream, first cube
        (M, N, P), (A, Y), ctx = shapes[0], probs[0], ctxs[0]
        Yh = torch.from_numpy(np.ascontiguousarray(Y).view(np.float32)).pin_memory()
        Xh = torch.full((P, 2 * N), float("nan")).pin_memory()
        it = torch.full((P,), -1, device="cuda", dtype=torch.int32)
        cs.cs_recover_stream(ctx, code, Yh, Xh, 16, kappa=6, G=2 if algo == "gomp" else 0,
                             opts=cs.make_opts(mu=1.0, iters_out=it))
        Xs = Xh.numpy().view(np.complex64).astype(np.complex128)
        assert np.array_equal(Xs, singles[algo, 0][0]) and np.array_equal(it.cpu().numpy(),
                                                                           singles[algo, 0][1])
        # batch of both cubes
        items, outs = [], []
        for (M, N, P), (A, Y), ctx in zip(shapes, probs, ctxs):
            Yd = torch.from_numpy(np.ascontiguousarray(Y).view(np.float32)).cuda()
            Xd = torch.full((P, 2 * N), float("nan"), device="cuda")
            itd = torch.full((P,), -1, device="cuda", dtype=torch.int32)
            items.append({"ctx": ctx, "Y": Yd, "X": Xd, "iters_out": itd})
            outs.append((Xd, itd))
        cs.cs_recover_batch(items, code, kappa=6, G=2 if algo == "gomp" else 0,
                            opts=cs.make_opts(mu=1.0))
        cs.cs_sync(ctxs[0])
        for i, (Xd, itd) in enumerate(outs):
            Xb = Xd.cpu().numpy().view(np.complex64).astype(np.complex128)
            assert np.array_equal(Xb, singles[algo, i][0])
            assert np.array_equal(itd.cpu().numpy(), singles[algo, i][1])
    # a real context beside a complex one, and kappa above the complex N
    real = cs.cs_create(48, 128, Phi=np.random.default_rng(0).standard_normal((48, 128)) / 7)
    Yd = torch.zeros((4, 48), device="cuda")
    Yc = torch.zeros((4, 48), device="cuda")
    with pytest.raises(cs.CsError) as e:
        cs.cs_recover_batch([{"ctx": ctxs[0], "Y": Yc, "X": torch.zeros((4, 128), device="cuda")},
                             {"ctx": real, "Y": Yd, "X": torch.zeros((4, 128), device="cuda")}],
                            cs.CS_ALGO_COSAMP, kappa=4)
    assert e.value.status == cs.CS_ERR_ARG
    with pytest.raises(cs.CsError) as e:  # kappa counts complex atoms: at most N
        cs.cs_recover_gomp(ctxs[0], Yc, torch.zeros((4, 128), device="cuda"), 65, 2)
    assert e.value.status == cs.CS_ERR_ARG
