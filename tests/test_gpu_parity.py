"""CUDA path (through the C ABI) against the FP64 oracle on identical seeded inputs.

Sizes span several 32-pixel tiles with a ragged tail; dimensions follow the small
(N=120, M=48) and FP32 (N=200, M=80) cube recipes.  Tolerances: relative L2 <= 1e-5
for the FP32 path; greedy supports identical on well-separated pixels.
"""
import numpy as np
import pytest

import oracle as orc
from gpu_common import (MARGIN_FP32, REL_L2_FP32, Problem, fixed_iteration_tolerance,
                        exact_check, gpu_run, iterate_conditioning, library, rel_l2, support,
                        support_check)
from oracle_pins import rand_orthogonal, soft_np
from paper_2401_14762_gb300 import synthetic as sy

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cs():
    return library()


@pytest.fixture(scope="module")
def small():
    return Problem(48, 120, 32 * 32 + 7, "sparse", seed=1, S=8)


@pytest.fixture(scope="module")
def plaw():
    return Problem(80, 200, 32 * 9 + 5, "powerlaw", seed=2, noise_var=1e-3)


# --------------------------------------------------------------------------- setup
@pytest.mark.parametrize("M,N,seed", [(48, 120, 1), (80, 200, 2), (90, 224, 3), (102, 256, 4),
                                      (5, 7, 5), (64, 64, 6)])
def test_setup_dictionary_lipschitz(cs, M, N, seed):
    Phi = sy.gaussian_phi(M, N, seed)
    A = orc.dictionary(Phi)
    ctx = cs.cs_create(M, N, Phi=Phi)
    assert np.abs(cs.cs_get_dictionary(ctx) - A).max() < 1e-13
    L = orc.lipschitz(A)
    assert abs(cs.cs_get_lipschitz(ctx) - L) <= 1e-12 * L


def test_setup_given_A_and_Psi(cs):
    M, N = 20, 32
    Phi = sy.gaussian_phi(M, N, 7)
    Psi = rand_orthogonal(N, 8)
    ctx = cs.cs_create(M, N, Phi=Phi, Psi=Psi)
    assert np.abs(cs.cs_get_dictionary(ctx) - orc.dictionary(Phi, Psi)).max() < 1e-13
    A = orc.dictionary(Phi)
    ctx2 = cs.cs_create(M, N, A=A)
    assert np.abs(cs.cs_get_dictionary(ctx2) - A).max() == 0.0


# --------------------------------------------------------------------------- measure
@pytest.mark.parametrize("M,N", [(48, 120), (80, 200), (102, 256), (128, 256), (3, 5)])
def test_measure(cs, M, N):
    """Y = X A^T + E per pixel, to FP32 accuracy.  P spans two or three 256-pixel tiles
    per CTA of the persistent tiled kernel (N a multiple of 4) and ends on a ragged tile;
    N = 5 takes the general kernel."""
    torch = pytest.importorskip("torch")
    P = 256 * 152 * 2 + 37
    Phi = sy.gaussian_phi(M, N, 3)
    A = orc.dictionary(Phi)
    X = sy.powerlaw_coeffs(P, N, 3, permute=True).astype(np.float32)
    E = sy.noise(P, M, 1e-3, 3).astype(np.float32)
    ctx = cs.cs_create(M, N, Phi=Phi)
    Yd = torch.zeros((P, M), device="cuda")
    Xd, Ed = torch.from_numpy(X).cuda(), torch.from_numpy(E).cuda()  # alive until the sync
    cs.cs_measure(ctx, Xd, Yd, Ed)
    cs.cs_sync(ctx)
    ref = orc.measure(A, X.astype(np.float64), E.astype(np.float64))
    scale = np.linalg.norm(ref, axis=1, keepdims=True)
    assert (np.abs(Yd.cpu().numpy() - ref) / scale).max() < 1e-6


@pytest.mark.parametrize("M,N,P,offset", [(2, 4, 1, 0), (3, 8, 37, 0), (16, 32, 255, 0),
                                          (20, 60, 257, 0), (5, 28, 600, 0), (48, 120, 1000, 1),
                                          (102, 256, 513, 2)])
def test_measure_edges(cs, M, N, P, offset):
    """The tiled kernel's tensor-map boxes (256 pixels x 32 columns) wider than X (N < 32)
    or taller (P < 256), ending inside a column chunk or a tile, and X starting off a
    16-byte boundary (offset floats into its buffer), which takes the general kernel."""
    torch = pytest.importorskip("torch")
    Phi = sy.gaussian_phi(M, N, 4)
    A = orc.dictionary(Phi)
    X = sy.powerlaw_coeffs(P, N, 4, permute=True).astype(np.float32)
    E = sy.noise(P, M, 1e-3, 4).astype(np.float32)
    ctx = cs.cs_create(M, N, Phi=Phi)
    buf = torch.zeros(P * N + 4, device="cuda")
    Xd = buf[offset:offset + P * N].view(P, N)
    Xd.copy_(torch.from_numpy(X))
    assert (Xd.data_ptr() % 16 == 0) == (offset == 0)
    Yd = torch.full((P, M), float("nan"), device="cuda")
    Ed = torch.from_numpy(E).cuda()
    cs.cs_measure(ctx, Xd, Yd, Ed)
    cs.cs_sync(ctx)
    ref = orc.measure(A, X.astype(np.float64), E.astype(np.float64))
    scale = np.linalg.norm(ref, axis=1, keepdims=True)
    assert (np.abs(Yd.cpu().numpy() - ref) / scale).max() < 1e-6


# --------------------------------------------------------------------------- FISTA
def _fista_fixed(cs, pr, lam, iters):
    """A fixed, unconverged iteration count: the oracle's own output is ill-conditioned
    there (momentum amplifies perturbations in weakly determined directions), so the
    FP32 tolerance follows from its measured conditioning."""
    run = lambda Y: orc.fista(pr.A, Y, pr.L, lam, 0.0, iters)[0]
    Xo = run(pr.Y)
    tol = fixed_iteration_tolerance(iterate_conditioning(run, pr.Y[:128]), iters)
    ctx = cs.cs_create(pr.M, pr.N, Phi=pr.Phi)
    Xg, it, cv = gpu_run(cs.cs_recover_fista, ctx, pr.Y, pr.N, lam, iters, eps=0.0)
    print(f"FISTA FP32 {iters} iterations: rel-L2 {rel_l2(Xg, Xo):.2e}, tolerance {tol:.2e}")
    assert rel_l2(Xg, Xo) <= tol, (rel_l2(Xg, Xo), tol)
    assert np.all(it == iters) and np.all(cv == 0)
    return rel_l2(Xg, Xo)


def test_fista_small(cs, small):
    _fista_fixed(cs, small, 1e-3, 500)


def test_fista_small_long_run_meets_fp32_bar(cs, small):
    """The same small sparse cube after 2000 iterations: the iterate has settled enough
    that its conditioning no longer amplifies FP32 rounding past the FP32 path's 1e-5
    (a numpy model in FP32 gives 7e-7 here, 7e-4 at 500 iterations)."""
    Xo = orc.fista(small.A, small.Y, small.L, 1e-3, 0.0, 2000)[0]
    ctx = cs.cs_create(small.M, small.N, Phi=small.Phi)
    Xg, it, _ = gpu_run(cs.cs_recover_fista, ctx, small.Y, small.N, 1e-3, 2000, eps=0.0)
    print(f"FISTA FP32 2000 iterations: rel-L2 {rel_l2(Xg, Xo):.2e}")
    assert np.all(it == 2000)
    assert rel_l2(Xg, Xo) <= REL_L2_FP32


def test_fista_momentum_table_reused_across_run_lengths(cs, small):
    """A context computes the momentum sequence once for its longest run: a short run, a
    longer run that outgrows the table, and the short run again give the bits that fresh
    contexts give for the same lengths."""
    def run(ctx, iters):
        return gpu_run(cs.cs_recover_fista, ctx, small.Y, small.N, 1e-3, iters, eps=0.0)[0]
    ctx = cs.cs_create(small.M, small.N, Phi=small.Phi)
    short1, long1, short2 = run(ctx, 40), run(ctx, 2500), run(ctx, 40)
    fresh_short = run(cs.cs_create(small.M, small.N, Phi=small.Phi), 40)
    fresh_long = run(cs.cs_create(small.M, small.N, Phi=small.Phi), 2500)
    assert np.array_equal(short1, fresh_short) and np.array_equal(short2, fresh_short)
    assert np.array_equal(long1, fresh_long)


def test_fista_powerlaw(cs, plaw):
    _fista_fixed(cs, plaw, 1e-3, 300)


@pytest.mark.parametrize("lam", [0.05, 0.02])
def test_fista_converged(cs, lam):
    """Run to the LASSO solution (Delta < eps): the map is contractive there and the FP32
    path meets the 1e-5 bound."""
    pr = Problem(48, 120, 200, "sparse", seed=21, S=6, noise_var=1e-4)
    Xo, _ = orc.fista(pr.A, pr.Y, pr.L, lam, 0.0, 20000)
    ctx = cs.cs_create(pr.M, pr.N, Phi=pr.Phi)
    Xg, it, cv = gpu_run(cs.cs_recover_fista, ctx, pr.Y, pr.N, lam, 20000, eps=1e-7)
    assert rel_l2(Xg, Xo) <= REL_L2_FP32
    assert np.all(support(Xg) == support(Xo))


def test_fista_delta_stop(cs):
    """A orthogonal: x^2 = x^1 = soft(A^T y, lambda), so Delta_2 ~ 0 and both sides stop
    after exactly 2 iterations; eps > 1 stops before the first iteration."""
    N = 64
    Q = rand_orthogonal(N, 9)
    Y = sy.noise(70, N, 1.0, 9).astype(np.float32)
    ctx = cs.cs_create(N, N, A=Q)
    Xg, it, cv = gpu_run(cs.cs_recover_fista, ctx, Y, N, 0.3, 100, eps=1e-4)
    Xo, ito = orc.fista(Q, Y, orc.lipschitz(Q), 0.3, 1e-4, 100)
    assert np.all(ito == 2) and np.all(it == 2) and np.all(cv == 1)
    assert rel_l2(Xg, soft_np(Y.astype(np.float64) @ Q, 0.3)) < 1e-5
    Xg, it, cv = gpu_run(cs.cs_recover_fista, ctx, Y, N, 0.3, 100, eps=2.0)
    assert np.all(Xg == 0) and np.all(it == 0)


# --------------------------------------------------------------------------- ADMM
@pytest.mark.parametrize("rho", [1.0, 1.8])
def test_admm_small(cs, small, rho):
    Xo, _ = orc.admm(small.A, small.Y, rho, 1e-3, 0.0, 500)
    ctx = cs.cs_create(small.M, small.N, Phi=small.Phi, admm_rho=1.0)
    Xg, it, cv = gpu_run(cs.cs_recover_admm, ctx, small.Y, small.N, rho, 1e-3, 500, eps=0.0)
    assert rel_l2(Xg, Xo) <= REL_L2_FP32
    assert np.all(it == 500)


def test_admm_powerlaw(cs, plaw):
    Xo, _ = orc.admm(plaw.A, plaw.Y, 1.0, 1e-3, 0.0, 300)
    ctx = cs.cs_create(plaw.M, plaw.N, Phi=plaw.Phi, admm_rho=1.0)
    Xg, _, _ = gpu_run(cs.cs_recover_admm, ctx, plaw.Y, plaw.N, 1.0, 1e-3, 300, eps=0.0)
    assert rel_l2(Xg, Xo) <= REL_L2_FP32


def test_admm_orthonormal_fixed_point(cs):
    N = 64
    Q = rand_orthogonal(N, 10)
    Y = sy.noise(40, N, 1.0, 10).astype(np.float32)
    ctx = cs.cs_create(N, N, A=Q)
    Xg, _, _ = gpu_run(cs.cs_recover_admm, ctx, Y, N, 1.8, 0.3, 400, eps=0.0)
    assert rel_l2(Xg, soft_np(Y.astype(np.float64) @ Q, 0.3)) < 1e-5


# --------------------------------------------------------------------------- greedy
def test_gomp_small(cs, small):
    Xo, ito, mg = orc.gomp(small.A, small.Y, 8, 2)
    ctx = cs.cs_create(small.M, small.N, Phi=small.Phi)
    Xg, it, cv = gpu_run(cs.cs_recover_gomp, ctx, small.Y, small.N, 8, 2)
    support_check(Xg, Xo, mg, 8)
    exact_check(Xg, it, Xo, ito, 8)


def test_gomp_powerlaw(cs, plaw):
    Xo, ito, mg = orc.gomp(plaw.A, plaw.Y, 20, 4)
    ctx = cs.cs_create(plaw.M, plaw.N, Phi=plaw.Phi)
    Xg, it, cv = gpu_run(cs.cs_recover_gomp, ctx, plaw.Y, plaw.N, 20, 4)
    exact_check(Xg, it, Xo, ito, 20)


def test_gomp_support_outgrows_shared_factor(cs, plaw):
    """gOMP keeps at most 64 rows of its FP32 factor in shared memory (fewer if that seats
    16 warps per SM, never fewer than 2 kappa): 59 rows at M = 80, N = 200, kappa = G = 9.
    Supports of 63 and 72 atoms (7 and 8 iterations) outgrow it, and those solves move to
    the FP64 factorisation in the warp's global slot: every pixel still follows the
    oracle's trajectory."""
    Xo, ito, _ = orc.gomp(plaw.A, plaw.Y, 9, 9)
    assert (9 * ito > 59).sum() >= 5  # pixels that overflow
    ctx = cs.cs_create(plaw.M, plaw.N, Phi=plaw.Phi)
    Xg, it, _ = gpu_run(cs.cs_recover_gomp, ctx, plaw.Y, plaw.N, 9, 9)
    exact_check(Xg, it, Xo, ito, 9)


def test_gomp_is_omp_exact(cs):
    """gOMP with G = 1 on [I | H/8]: OMP recovers every 4-sparse x exactly."""
    import scipy.linalg
    M = 64
    A = np.hstack([np.eye(M), scipy.linalg.hadamard(M) / 8.0])
    Xt = sy.sparse_coeffs(100, 2 * M, 4, 11)
    Y = (Xt @ A.T).astype(np.float32)
    ctx = cs.cs_create(M, 2 * M, A=A)
    Xg, _, _ = gpu_run(cs.cs_recover_gomp, ctx, Y, 2 * M, 4, 1)
    assert np.all(support(Xg) == (Xt != 0))
    assert rel_l2(Xg, Xt) < 1e-6


@pytest.mark.parametrize("mu", [0.1, 1.0])
def test_biht_small(cs, small, mu):
    Xo, ito, mg = orc.biht(small.A, small.Y, 8, mu)
    ctx = cs.cs_create(small.M, small.N, Phi=small.Phi)
    Xg, it, cv = gpu_run(cs.cs_recover_biht, ctx, small.Y, small.N, 8, mu=mu)
    support_check(Xg, Xo, mg, 8)
    exact_check(Xg, it, Xo, ito, 8)


def test_biht_powerlaw(cs, plaw):
    Xo, ito, mg = orc.biht(plaw.A, plaw.Y, 20, 0.1)
    ctx = cs.cs_create(plaw.M, plaw.N, Phi=plaw.Phi)
    Xg, it, _ = gpu_run(cs.cs_recover_biht, ctx, plaw.Y, plaw.N, 20, mu=0.1)
    exact_check(Xg, it, Xo, ito, 20)


def test_biht_worked_example(cs):
    A = np.array([[1.0, 0.0, 1.0], [0.0, 1.0, 1.0]])
    Y = np.array([[1.0, 3.0]], dtype=np.float32)
    ctx = cs.cs_create(2, 3, A=A)
    Xg, it, _ = gpu_run(cs.cs_recover_biht, ctx, Y, 3, 1, mu=2.0)
    assert np.abs(Xg[0] - [0.0, 0.0, 3.0]).max() < 1e-6 and it[0] == 3


def test_cosamp_small(cs, small):
    Xo, ito, mg = orc.cosamp(small.A, small.Y, 8)
    ctx = cs.cs_create(small.M, small.N, Phi=small.Phi)
    Xg, it, cv = gpu_run(cs.cs_recover_cosamp, ctx, small.Y, small.N, 8)
    support_check(Xg, Xo, mg, 8)
    exact_check(Xg, it, Xo, ito, 8)


def test_cosamp_powerlaw(cs):
    # the 2 kappa = 40-atom cut of power-law spectra is often near-tied and CoSaMP
    # oscillates up to its cap: any selection that differed from FP64 would show
    plaw = Problem(80, 200, 32 * 40 + 5, "powerlaw", seed=2, noise_var=1e-3)
    Xo, ito, mg = orc.cosamp(plaw.A, plaw.Y, 20)
    ctx = cs.cs_create(plaw.M, plaw.N, Phi=plaw.Phi)
    Xg, it, _ = gpu_run(cs.cs_recover_cosamp, ctx, plaw.Y, plaw.N, 20)
    assert (ito == 100).mean() > 0.3  # many pixels never converge: a long trajectory
    exact_check(Xg, it, Xo, ito, 20)


@pytest.mark.parametrize("algo", ["biht", "cosamp"])
def test_cycle_skip_is_exact(cs, algo):
    """Stopping at a repeated iterate changes nothing: X, iteration counts and flags are
    bit for bit those of running every iteration, with less work done."""
    pr = Problem(80, 200, 32 * 12 + 7, "powerlaw", seed=5, noise_var=1e-3)
    ctx = cs.cs_create(pr.M, pr.N, Phi=pr.Phi)
    call = cs.cs_recover_biht if algo == "biht" else cs.cs_recover_cosamp
    runs = []
    for skip in (True, False):
        runs.append(gpu_run(call, ctx, pr.Y, pr.N, 20, mu=1.0 if algo == "biht" else 0.1,
                            cycle_skip=skip, eps=0.0 if algo == "biht" else 1e-8))
        runs[-1] += (cs.cs_get_work(ctx),)
    (Xs, its, cvs, ws), (Xf, itf, cvf, wf) = runs
    assert np.array_equal(Xs.view(np.uint32), Xf.view(np.uint32))
    assert np.array_equal(its, itf) and np.array_equal(cvs, cvf)
    assert (itf == 100).mean() > 0.3 and ws < 0.8 * wf


def test_min_norm_support(cs):
    """CoSaMP with 3 kappa > M: supports larger than M take the minimum-norm solution."""
    pr = Problem(24, 60, 70, "sparse", seed=12, S=10)
    Xo, ito, mg = orc.cosamp(pr.A, pr.Y, 10, max_iters=5)
    ctx = cs.cs_create(pr.M, pr.N, Phi=pr.Phi)
    Xg, it, _ = gpu_run(cs.cs_recover_cosamp, ctx, pr.Y, pr.N, 10, max_iters=5)
    exact_check(Xg, it, Xo, ito, 10)


def test_kappa_per_pixel(cs):
    """Per-pixel sparsity with G = max(1, floor(kappa/5)) (the paper's G rule)."""
    pr = Problem(48, 120, 200, "sparse", seed=13, S=6, amplitude="separated")
    kp = sy.kappa_per_pixel(pr.P, 4, 12, 13)
    ctx = cs.cs_create(pr.M, pr.N, Phi=pr.Phi)
    Xg, it, _ = gpu_run(cs.cs_recover_gomp, ctx, pr.Y, pr.N, 12, 0, kappa_pp=kp)
    Xo = np.zeros_like(pr.Xt)
    mg = np.zeros(pr.P)
    ito = np.zeros(pr.P, dtype=it.dtype)
    for k in np.unique(kp):
        sel = kp == k
        Xo[sel], ito[sel], mg[sel] = orc.gomp(pr.A, pr.Y[sel], int(k), max(1, int(k) // 5))
    support_check(Xg, Xo, mg, 12)
    exact_check(Xg, it, Xo, ito, 12)


# --------------------------------------------------------------------------- edges
def test_edge_cases(cs, small):
    torch = pytest.importorskip("torch")
    ctx = cs.cs_create(small.M, small.N, Phi=small.Phi)
    Y = small.Y[:40].copy()
    Y[3] = 0.0  # y = 0 -> x = 0 for every method
    for call, args in [(cs.cs_recover_fista, (1e-3, 50)), (cs.cs_recover_admm, (1.0, 1e-3, 50)),
                       (cs.cs_recover_gomp, (8, 2)), (cs.cs_recover_biht, (8,)),
                       (cs.cs_recover_cosamp, (8,))]:
        Xg, it, _ = gpu_run(call, ctx, Y, small.N, *args)
        assert np.all(Xg[3] == 0), call.__name__
        assert np.all(np.isfinite(Xg))
    Xg, it, _ = gpu_run(cs.cs_recover_gomp, ctx, Y, small.N, 0, 2)  # kappa = 0
    assert np.all(Xg == 0) and np.all(it == 0)
    # P = 0 is a no-op
    e = torch.zeros((0, small.M), device="cuda")
    cs.cs_recover_fista(ctx, e, torch.zeros((0, small.N), device="cuda"), 1e-3, 10)
    cs.cs_sync(ctx)
    # a single pixel
    Xg, _, _ = gpu_run(cs.cs_recover_gomp, ctx, small.Y[:1], small.N, 8, 2)
    Xo, _, _ = orc.gomp(small.A, small.Y[:1], 8, 2)
    assert rel_l2(Xg, Xo) < 1e-5


def test_nonfinite_input_is_reported(cs, small):
    torch = pytest.importorskip("torch")
    ctx = cs.cs_create(small.M, small.N, Phi=small.Phi)
    Y = small.Y[:8].copy()
    Y[2, 5] = np.nan
    X = torch.zeros((8, small.N), device="cuda")
    Yd = torch.from_numpy(Y).cuda()  # kept alive until the asynchronous call is synced
    cs.cs_recover_gomp(ctx, Yd, X, 8, 2)
    with pytest.raises(cs.CsError) as e:
        cs.cs_sync(ctx)
    assert e.value.status == cs.CS_ERR_NONFINITE
    cs.cs_sync(ctx)  # the status word was cleared


def test_host_pointer_path_matches_device(cs, small):
    ctx = cs.cs_create(small.M, small.N, Phi=small.Phi)
    Xh = np.zeros((small.P, small.N), dtype=np.float32)
    cs.cs_recover_fista(ctx, small.Y, Xh, 1e-3, 100, opts=cs.make_opts(eps=0.0))
    Xd, _, _ = gpu_run(cs.cs_recover_fista, ctx, small.Y, small.N, 1e-3, 100, eps=0.0)
    assert np.array_equal(Xh, Xd)
    Xh = np.zeros((small.P, small.N), dtype=np.float32)
    cs.cs_recover_gomp(ctx, small.Y, Xh, 8, 2)
    Xd, _, _ = gpu_run(cs.cs_recover_gomp, ctx, small.Y, small.N, 8, 2)
    assert np.array_equal(Xh, Xd)


def test_argument_errors(cs, small):
    torch = pytest.importorskip("torch")
    ctx = cs.cs_create(small.M, small.N, Phi=small.Phi)
    Y = torch.zeros((4, small.M), device="cuda")
    X = torch.zeros((4, small.N), device="cuda")
    bad = [lambda: cs.cs_recover_fista(ctx, Y, X, -1.0, 10),
           lambda: cs.cs_recover_fista(ctx, Y, X, 0.1, -1),
           lambda: cs.cs_recover_admm(ctx, Y, X, 0.0, 0.1, 10),
           lambda: cs.cs_recover_gomp(ctx, Y, X, small.N + 1, 2),
           lambda: cs.cs_recover_gomp(ctx, Y, X, 8, 0),
           lambda: cs.cs_recover_cosamp(ctx, Y, X, small.N // 2 + 1),
           lambda: cs.cs_recover_fista(ctx, Y, X.cpu().numpy(), 0.1, 10),
           lambda: cs.cs_recover_fista(ctx, Y, X, 0.1, 10, opts=cs.make_opts(eps=-1.0))]
    for f in bad:
        with pytest.raises(cs.CsError) as e:
            f()
        assert e.value.status == cs.CS_ERR_ARG


# --------------------------------------------------------------------------- maximum sizes
@pytest.mark.parametrize("algo,kappa,G", [("gomp", 16, 8), ("biht", 60, 0), ("cosamp", 42, 0)])
def test_greedy_maximum_shape(cs, algo, kappa, G):
    """M = 128, N = 256 (the largest dictionary) with supports of up to 120-128 atoms, the
    widest register layout of the greedy kernel: exact against the oracle."""
    pr = Problem(128, 256, 70, "sparse", seed=31, S=12, amplitude="separated")
    ctx = cs.cs_create(128, 256, Phi=pr.Phi)
    if algo == "gomp":
        Xo, ito, _ = orc.gomp(pr.A, pr.Y, kappa, G)
        Xg, it, _ = gpu_run(cs.cs_recover_gomp, ctx, pr.Y, 256, kappa, G)
    elif algo == "biht":
        Xo, ito, _ = orc.biht(pr.A, pr.Y, kappa, 1.0)
        Xg, it, _ = gpu_run(cs.cs_recover_biht, ctx, pr.Y, 256, kappa, mu=1.0)
    else:
        Xo, ito, _ = orc.cosamp(pr.A, pr.Y, kappa)
        Xg, it, _ = gpu_run(cs.cs_recover_cosamp, ctx, pr.Y, 256, kappa)
    exact_check(Xg, it, Xo, ito, kappa)


def test_admm_maximum_shape(cs):
    pr = Problem(128, 256, 70, "powerlaw", seed=32, noise_var=1e-3)
    Xo, _ = orc.admm(pr.A, pr.Y, 1.0, 1e-3, 0.0, 150)
    ctx = cs.cs_create(128, 256, Phi=pr.Phi, admm_rho=1.0)
    Xg, it, _ = gpu_run(cs.cs_recover_admm, ctx, pr.Y, 256, 1.0, 1e-3, 150, eps=0.0)
    assert np.all(it == 150)
    assert rel_l2(Xg, Xo) <= REL_L2_FP32


def test_fista_maximum_shape(cs):
    """FP32 FISTA at M = 128, N = 256 (the BF16 request falls back to it there)."""
    pr = Problem(128, 256, 70, "powerlaw", seed=33, noise_var=1e-3)
    run = lambda Y: orc.fista(pr.A, Y, pr.L, 1e-3, 0.0, 120)[0]
    Xo = run(pr.Y)
    tol = fixed_iteration_tolerance(iterate_conditioning(run, pr.Y), 120)
    ctx = cs.cs_create(128, 256, Phi=pr.Phi)
    for prec in (0, 1):
        Xg, it, _ = gpu_run(cs.cs_recover_fista, ctx, pr.Y, 256, 1e-3, 120, eps=0.0, prec=prec)
        print(f"FISTA M=128 N=256 prec {prec}: rel-L2 {rel_l2(Xg, Xo):.2e}, tolerance {tol:.2e}")
        assert np.all(it == 120)
        assert rel_l2(Xg, Xo) <= tol
