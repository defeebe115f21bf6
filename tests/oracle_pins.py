"""Pins for the FP64 oracle: facts fixed by the paper and by mathematics, not by the
oracle itself.

Each ``pin_*`` function raises AssertionError when the oracle disagrees with a
closed form, an invariant, a special case that reduces to a textbook or library
routine, or a brute-force answer.  ``test_oracle_pins.py`` runs them against the
oracle; ``test_oracle_mutants.py`` runs them against copies of the oracle with
planted mistakes and requires every mistake to be caught.

Algorithm references are to the paper (Justo et al., Section II-A):
Algorithm 1 FISTA, 2 ADMM, 3 gOMP, 4 BIHT, 5 CoSaMP; Eq. 1 the measurement model,
Eq. 2 the LASSO objective.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.fft
import scipy.linalg

import oracle as orc
from paper_2401_14762_gb300 import synthetic as sy


def _rng(seed):
    return np.random.default_rng(seed)


def soft_np(v, t):
    return np.sign(v) * np.maximum(np.abs(v) - t, 0.0)


def rand_orthogonal(n, seed):
    Q, R = np.linalg.qr(_rng(seed).standard_normal((n, n)))
    return Q * np.sign(np.diag(R))


def small_problem(M=20, N=40, S=4, seed=3, noise=0.01):
    A = sy.gaussian_phi(M, N, seed)
    x = sy.sparse_coeffs(1, N, S, seed, "separated")[0]
    y = A @ x + noise * _rng(seed).standard_normal(M)
    return A, x, y


def lasso_objective(A, y, x, lam):
    """H(x) = 1/2 ||Ax - y||^2 + lambda ||x||_1 (Eq. 2)."""
    return 0.5 * np.sum((A @ x - y) ** 2) + lam * np.sum(np.abs(x))


def check_kkt(A, y, x, lam, tol):
    """Optimality of Eq. 2: g = A^T (y - A x) equals lambda sign(x_j) on the support
    and |g_j| <= lambda off it."""
    g = A.T @ (y - A @ x)
    on = np.abs(x) > 1e-12  # ADMM's x iterate keeps ~1e-17 entries off the support
    assert np.all(np.abs(g[on] - lam * np.sign(x[on])) <= tol), np.abs(g[on] - lam * np.sign(x[on])).max()
    assert np.all(np.abs(g[~on]) <= lam + tol)
    return on


def textbook_omp(A, y, k):
    """Orthogonal matching pursuit (Pati et al. 1993) with numpy least squares."""
    r, support = y.copy(), []
    x = np.zeros(A.shape[1])
    for _ in range(k):
        corr = np.abs(A.T @ r)
        corr[support] = -1.0
        support.append(int(np.argmax(corr)))
        s, *_ = np.linalg.lstsq(A[:, support], y, rcond=None)
        x = np.zeros(A.shape[1])
        x[support] = s
        r = y - A @ x
    return x


def topk_np(v, k):
    """Largest |v| first, lower index on ties (the oracle's argmax_k reading)."""
    order = np.lexsort((np.arange(len(v)), -np.abs(v)))
    return order[:k]


# --------------------------------------------------------------------------
# Eq. 1: transform, dictionary, measurement
# --------------------------------------------------------------------------
def pin_psi():
    for N in (8, 120, 200, 256):
        Psi = orc.dct2_psi(N)
        assert np.abs(Psi.T @ Psi - np.eye(N)).max() < 1e-13
        x = _rng(N).standard_normal(N)
        # Psi x is the orthonormal inverse DCT-II (DCT-III) of x: library special case
        assert np.abs(Psi @ x - scipy.fft.idct(x, norm="ortho")).max() < 1e-12
        # Parseval: the MSE is the same in the band and coefficient domains
        assert abs(np.sum((Psi @ x) ** 2) - np.sum(x ** 2)) < 1e-11


def pin_dictionary_measure():
    M, N, P = 12, 30, 7
    Phi = sy.gaussian_phi(M, N, 5)
    A = orc.dictionary(Phi)
    Psi_ref = scipy.fft.idct(np.eye(N), norm="ortho", axis=0)
    assert np.abs(A - Phi @ Psi_ref).max() < 1e-12
    X = _rng(1).standard_normal((P, N))
    E = _rng(2).standard_normal((P, M))
    assert np.abs(orc.measure(A, X, E) - (X @ A.T + E)).max() < 1e-12
    assert np.abs(orc.measure(A, X) - X @ A.T).max() < 1e-12


def pin_lipschitz():
    for (M, N, seed) in [(5, 9, 1), (48, 120, 2), (80, 200, 3), (102, 256, 4)]:
        A = sy.gaussian_phi(M, N, seed)
        ref = np.linalg.eigvalsh(A.T @ A).max()
        assert abs(orc.lipschitz(A) - ref) <= 1e-12 * ref
        assert abs(orc.lipschitz(A) - np.linalg.svd(A, compute_uv=False)[0] ** 2) <= 1e-12 * ref
    # orthonormal rows: A A^T = I, so L = 1
    Q = rand_orthogonal(16, 7)[:6]
    assert abs(orc.lipschitz(Q) - 1.0) < 1e-13
    # a diagonal case: eigenvalues are the squared diagonal
    D = np.zeros((3, 5))
    D[0, 0], D[1, 1], D[2, 2] = 1.0, -3.0, 2.0
    assert abs(orc.lipschitz(D) - 9.0) < 1e-13


def pin_argmax_k():
    v = np.array([1.0, -3.0, 3.0, 2.0, 0.0, 0.0])
    idx, gap = orc.argmax_k(v, 3)
    assert list(idx) == [1, 2, 3]
    assert abs(gap - (2.0 - 1.0) / 2.0) < 1e-15
    idx, _ = orc.argmax_k(v, 6)
    assert list(idx) == [1, 2, 3, 0, 4, 5]
    for seed in range(20):
        w = np.round(_rng(seed).standard_normal(37), 1)  # rounding creates ties
        for k in (1, 5, 17):
            idx, _ = orc.argmax_k(w, k)
            assert list(idx) == list(topk_np(w, k))


def pin_lstsq():
    rng = _rng(11)
    A = rng.standard_normal((10, 30))
    A[:, 7] = A[:, 3]  # a repeated atom makes some supports rank deficient
    y = rng.standard_normal(10)
    for c in ([0, 5, 9], list(range(10)), [2, 4, 6, 8, 10, 12, 14, 16, 18, 20, 22, 24, 26],
              [3, 7, 1], [3, 7, 1, 2, 5, 11, 12, 13, 14, 15, 16, 17]):
        s = orc.support_lstsq(A, c, y)
        ref = np.linalg.pinv(A[:, c]) @ y
        assert np.abs(s - ref).max() < 1e-9 * max(1.0, np.abs(ref).max()), c


# --------------------------------------------------------------------------
# Algorithm 1: FISTA
# --------------------------------------------------------------------------
def pin_fista_orthonormal():
    """A orthogonal and L = 1: every iterate is soft(A^T y, lambda), the LASSO solution."""
    N = 16
    Q = rand_orthogonal(N, 2)
    Y = _rng(3).standard_normal((3, N))
    for iters in (1, 2, 7):
        X, it = orc.fista(Q, Y, 1.0, 0.3, 0.0, iters)
        assert np.abs(X - soft_np(Y @ Q, 0.3)).max() < 1e-12
        assert np.all(it == iters)


def pin_fista_first_iterate():
    """z^0 = 0 gives x^1 = soft(A^T y / L, lambda / L)."""
    A, _, y = small_problem()
    L = orc.lipschitz(A)
    X, _ = orc.fista(A, y[None], L, 0.05, 0.0, 1)
    assert np.abs(X[0] - soft_np(A.T @ y / L, 0.05 / L)).max() < 1e-13


def pin_fista_zero():
    """lambda >= ||A^T y||_inf makes x = 0 the solution and a fixed point."""
    A, _, y = small_problem()
    lam = np.abs(A.T @ y).max() * 1.0001
    X, _ = orc.fista(A, y[None], orc.lipschitz(A), lam, 0.0, 50)
    assert np.all(X == 0.0)


def _lasso_reference(A, y, lam):
    X, _ = orc.fista(A, y[None], orc.lipschitz(A), lam, 0.0, 20000)
    return X[0]


def pin_fista_lasso():
    """Converged FISTA satisfies the LASSO KKT conditions (Eq. 2) to 1e-9, and on its
    support it solves A_S^T A_S x_S = A_S^T y - lambda sign(x_S)."""
    A, _, y = small_problem()
    lam = 0.05
    x = _lasso_reference(A, y, lam)
    on = check_kkt(A, y, x, lam, 1e-9)
    xs = np.linalg.solve(A[:, on].T @ A[:, on], A[:, on].T @ y - lam * np.sign(x[on]))
    assert np.abs(xs - x[on]).max() < 1e-9


def pin_fista_rate():
    """Beck-Teboulle bound: H(x^k) - H* <= 2 L ||x^0 - x*||^2 / (k+1)^2, and the gap
    closes (momentum makes FISTA beat the ISTA bound L||x*||^2/(2k) by k = 40)."""
    A, _, y = small_problem(seed=8)
    lam = 0.05
    L = orc.lipschitz(A)
    xs = _lasso_reference(A, y, lam)
    Hs = lasso_objective(A, y, xs, lam)
    R2 = np.sum(xs ** 2)
    gaps = []
    for k in range(1, 41):
        X, _ = orc.fista(A, y[None], L, lam, 0.0, k)
        gap = lasso_objective(A, y, X[0], lam) - Hs
        assert gap <= 2 * L * R2 / (k + 1) ** 2 + 1e-12, k
        gaps.append(gap)
    assert gaps[-1] < 0.25 * L * R2 / (2 * 40)


def pin_fista_momentum():
    """Scalar quadratic (A = I, lambda = 0, L = 100 > lambda_max = 1): the error e_k = x^k - y
    obeys e^{k+1} = q (e^k + beta_k (e^k - e^{k-1})), q = 1 - 1/L, so the momentum
    weights beta_k can be read off the iterates.  t^0 = 1 gives beta_1 = 0 (the second
    iterate is a plain proximal-gradient step), and the t-sequence of Algorithm 1 makes
    beta_k approach Nesterov's (k-1)/(k+2) within 0.3/k for 5 <= k <= 40."""
    A = np.eye(1)
    Y = np.ones((1, 1))
    q = 1.0 - 1.0 / 100.0
    e = [-1.0]  # x^0 = 0
    for k in range(1, 43):
        X, _ = orc.fista(A, Y, 100.0, 0.0, 0.0, k)
        e.append(X[0, 0] - 1.0)
    beta = {k: (e[k + 1] / q - e[k]) / (e[k] - e[k - 1]) for k in range(1, 41)}
    assert abs(beta[1]) < 1e-12
    for k in range(5, 41):
        assert abs(beta[k] - (k - 1) / (k + 2)) <= 0.3 / k, (k, beta[k])


def pin_fista_stop_rule():
    """The loop stops at the first i with ||r^i - r^{i-1}|| < eps, r^0 = y."""
    A, _, y = small_problem(seed=9)
    L, lam, eps = orc.lipschitz(A), 0.05, 1e-3
    X, it = orc.fista(A, y[None], L, lam, eps, 10000)
    n = int(it[0])
    prev_r = y
    first = None
    for k in range(1, n + 1):
        Xk, _ = orc.fista(A, y[None], L, lam, 0.0, k)
        r = y - A @ Xk[0]
        if first is None and np.linalg.norm(r - prev_r) < eps:
            first = k
        prev_r = r
    assert first == n
    assert np.abs(X[0] - Xk[0]).max() == 0.0
    X0, it0 = orc.fista(A, y[None], L, lam, 2.0, 100)  # Delta starts at 1 < eps
    assert it0[0] == 0 and np.all(X0 == 0)


# --------------------------------------------------------------------------
# Algorithm 2: ADMM
# --------------------------------------------------------------------------
def pin_admm_first_iterate():
    """z^0 = w^0 = 0 gives x^1 = (A^T A + alpha I)^{-1} A^T y: ridge regression, i.e.
    least squares on the stacked system [A; sqrt(alpha) I] x = [y; 0]."""
    A, _, y = small_problem()
    alpha = 1.8
    X, _ = orc.admm(A, y[None], alpha, 0.05, 0.0, 1)
    N = A.shape[1]
    ref, *_ = np.linalg.lstsq(np.vstack([A, np.sqrt(alpha) * np.eye(N)]),
                              np.concatenate([y, np.zeros(N)]), rcond=None)
    assert np.abs(X[0] - ref).max() < 1e-12


def pin_admm_orthonormal():
    """A orthogonal: ADMM converges to soft(A^T y, lambda) for alpha != 1, which pins
    the lambda/alpha threshold reading (lambda*alpha would give soft(., lambda*alpha^2))."""
    N = 16
    Q = rand_orthogonal(N, 4)
    Y = _rng(5).standard_normal((3, N))
    X, _ = orc.admm(Q, Y, 1.8, 0.3, 0.0, 400)
    assert np.abs(X - soft_np(Y @ Q, 0.3)).max() < 1e-10


def pin_admm_lasso():
    """Converged ADMM (alpha = 1.8) meets the LASSO KKT conditions and equals FISTA's
    converged point."""
    A, _, y = small_problem()
    lam = 0.05
    X, _ = orc.admm(A, y[None], 1.8, lam, 0.0, 20000)
    check_kkt(A, y, X[0], lam, 1e-9)
    assert np.abs(X[0] - _lasso_reference(A, y, lam)).max() < 1e-9


# --------------------------------------------------------------------------
# Algorithms 3-5: greedy
# --------------------------------------------------------------------------
def pin_gomp_is_omp():
    """gOMP with G = 1 is OMP: one atom per iteration, LS refit, and (|c| <= kappa) no pruning."""
    M, N = 30, 70
    A = sy.gaussian_phi(M, N, 12)
    Y = sy.powerlaw_coeffs(6, N, 12, permute=True) @ A.T + 0.01 * _rng(1).standard_normal((6, M))
    X, it, _ = orc.gomp(A, Y, 9, 1, 0.0)
    for p in range(6):
        ref = textbook_omp(A, Y[p], 9)
        assert set(np.flatnonzero(X[p])) == set(np.flatnonzero(ref))
        assert np.abs(X[p] - ref).max() < 1e-10
    assert np.all(it == 9)


def pin_first_iterates():
    """One iteration of each greedy method from r^0 = y, x^0 = 0, c^0 = {} has a closed form."""
    A, _, y = small_problem(M=24, N=60, S=5, seed=13)
    corr = A.T @ y
    kappa = 5
    # gOMP (G = 3 <= kappa): c = top-3 |A^T y|, no pruning, x = LS on c
    X, _, _ = orc.gomp(A, y[None], kappa, 3, 0.0, 1)
    c = topk_np(corr, 3)
    ref = np.zeros(60)
    ref[c] = np.linalg.lstsq(A[:, c], y, rcond=None)[0]
    assert np.abs(X[0] - ref).max() < 1e-11
    # BIHT: u = mu A^T y, c = top-kappa |u|, x = LS on c
    X, _, _ = orc.biht(A, y[None], kappa, 0.1, 0.0, 1)
    c = topk_np(corr, kappa)
    ref = np.zeros(60)
    ref[c] = np.linalg.lstsq(A[:, c], y, rcond=None)[0]
    assert np.abs(X[0] - ref).max() < 1e-11
    # CoSaMP: c = top-2kappa |A^T y|, s = LS on c, keep the kappa largest |s| unrefit
    X, _, _ = orc.cosamp(A, y[None], kappa, 0.0, 1)
    c = topk_np(corr, 2 * kappa)
    s = np.linalg.lstsq(A[:, c], y, rcond=None)[0]
    keep = topk_np(s, kappa)
    ref = np.zeros(60)
    ref[c[keep]] = s[keep]
    assert np.abs(X[0] - ref).max() < 1e-11


def pin_biht_small_step():
    """With mu -> 0, u = x_a + mu A^T(y - A x_a) ranks like x_a itself, so from the second
    iteration on Theta = supp(x_a), c does not grow, r repeats and Delta = 0: BIHT stops
    after 2 iterations at the first iterate (LS on the top-kappa of |A^T y|)."""
    A, _, y = small_problem(M=24, N=60, S=5, seed=13)
    X, it, _ = orc.biht(A, y[None], 5, 1e-9, 1e-8, 100)
    c = topk_np(A.T @ y, 5)
    ref = np.zeros(60)
    ref[c] = np.linalg.lstsq(A[:, c], y, rcond=None)[0]
    assert it[0] == 2
    assert np.abs(X[0] - ref).max() < 1e-11


def pin_biht_orthogonal_large_step():
    """A orthogonal: every support LS is A^T y restricted to the support, so after the first
    iterate (the kappa largest |A^T y|) a large step mu = 3 may propose new atoms, but the
    union-then-prune of Algorithm 4 keeps the same kappa atoms, r repeats and Delta = 0:
    the result is the hard threshold H_kappa(A^T y) after 2 iterations."""
    Q = rand_orthogonal(16, 4)
    Y = _rng(5).standard_normal((4, 16))
    X, it, _ = orc.biht(Q, Y, 4, 3.0, 1e-8, 100)
    B = Y @ Q
    for p in range(4):
        ref = np.zeros(16)
        keep = topk_np(B[p], 4)
        ref[keep] = B[p, keep]
        assert np.abs(X[p] - ref).max() < 1e-12
    assert np.all(it == 2)


def pin_biht_worked_example():
    """Worked by hand: A = [e1 e2 (1,1)^T], y = (1, 3), kappa = 1, mu = 2.
    Iter 1: u = 2 A^T y = (2, 6, 8) -> c = {3}, s = 2, x = 2 e3, r = (-1, 1).
    Iter 2: g = A^T r = (-1, 1, 0), u = x + 2g = (-2, 2, 2): a three-way tie, the lowest
      index wins -> c = {3} U {1}; the 2x2 fit gives s3 = 3, s1 = -2; keep the larger:
      x = 3 e3, r = (-2, 0).
    Iter 3: g = (-2, 0, -2), u = (-4, 0, -1) -> c = {3, 1} again, x = 3 e3, Delta = 0.
    So x = (0, 0, 3) after 3 iterations (a wrong step sign would give u = (4, 0, 7) in
    iteration 3 and x = 2 e3; the other tie-break would stop at 2 e3)."""
    A = np.array([[1.0, 0.0, 1.0], [0.0, 1.0, 1.0]])
    X, it, _ = orc.biht(A, np.array([[1.0, 3.0]]), 1, 2.0, 1e-8, 100)
    assert np.abs(X[0] - np.array([0.0, 0.0, 3.0])).max() < 1e-12
    assert it[0] == 3


def pin_gomp_cap():
    """With eps = 0 gOMP runs exactly min(kappa, floor(M/G)) iterations."""
    A = sy.gaussian_phi(20, 50, 14)
    Y = sy.powerlaw_coeffs(2, 50, 14, permute=True) @ A.T
    for kappa, G in [(8, 3), (15, 2), (4, 7)]:
        _, it, _ = orc.gomp(A, Y, kappa, G, 0.0, 100)
        assert np.all(it == min(kappa, 20 // G))


def pin_greedy_invariants():
    """Outputs are kappa-sparse; gOMP's final x is the LS fit on its own support
    (A_q^T (y - A x) = 0)."""
    M, N, kappa = 40, 100, 8
    A = sy.gaussian_phi(M, N, 15)
    Y = sy.powerlaw_coeffs(5, N, 15, permute=True) @ A.T + 0.03 * _rng(2).standard_normal((5, M))
    Xg, _, _ = orc.gomp(A, Y, kappa, 2)
    Xb, _, _ = orc.biht(A, Y, kappa)
    Xc, _, _ = orc.cosamp(A, Y, kappa)
    for X in (Xg, Xb, Xc):
        assert np.all((X != 0).sum(1) <= kappa)
    for p in range(5):
        q = np.flatnonzero(Xg[p])
        assert np.abs(A[:, q].T @ (Y[p] - A @ Xg[p])).max() < 1e-10


def pin_exact_recovery():
    """Noiseless S-sparse pixels with well-separated amplitudes and M = 48 >= 2S are
    recovered exactly by all three greedy methods (kappa = S).  BIHT takes the unit
    gradient step mu = 1 here (see pin_biht_small_step for mu -> 0)."""
    M, N, S, P = 48, 120, 4, 24
    A = sy.gaussian_phi(M, N, 16)
    Xt = sy.sparse_coeffs(P, N, S, 16, "separated")
    Y = Xt @ A.T
    Xg, _, _ = orc.gomp(A, Y, S, 2)
    Xc, _, _ = orc.cosamp(A, Y, S)
    Xb, _, _ = orc.biht(A, Y, S, 1.0)
    for X in (Xg, Xc, Xb):
        assert np.abs(X - Xt).max() < 1e-9


def pin_coherence_guarantee():
    """A = [I | H/sqrt(M)] (M = 64) has coherence 1/8, so OMP (gOMP with G = 1) recovers
    every S-sparse x with S < (1 + 8)/2 exactly (Tropp 2004, exact recovery condition)."""
    M = 64
    A = np.hstack([np.eye(M), scipy.linalg.hadamard(M) / np.sqrt(M)])
    for S in (1, 2, 3, 4):
        Xt = sy.sparse_coeffs(20, 2 * M, S, 100 + S, "normal")
        X, _, _ = orc.gomp(A, Xt @ A.T, S, 1)
        assert np.abs(X - Xt).max() < 1e-10, S


def pin_brute_force():
    """Tiny problems (N = 12, M = 6, S = 2): exhaustive search over all C(12, 2) supports
    finds exactly one zero-residual support, the true one; whenever a greedy method
    reaches a zero residual its answer is that unique solution."""
    M, N, S = 6, 12, 2
    agree = 0
    for seed in range(12):
        A = sy.gaussian_phi(M, N, 200 + seed)
        xt = sy.sparse_coeffs(1, N, S, 200 + seed, "separated")[0]
        y = A @ xt
        zero = []
        for c in itertools.combinations(range(N), S):
            s = np.linalg.lstsq(A[:, c], y, rcond=None)[0]
            if np.linalg.norm(y - A[:, c] @ s) < 1e-10:
                zero.append(c)
        assert zero == [tuple(np.flatnonzero(xt))]
        for X in (orc.gomp(A, y[None], S, 1)[0], orc.cosamp(A, y[None], S)[0],
                  orc.biht(A, y[None], S, 1.0)[0]):
            if np.linalg.norm(y - A @ X[0]) < 1e-9:
                assert np.abs(X[0] - xt).max() < 1e-9
                agree += 1
    assert agree >= 18


def pin_degenerate():
    """y = 0 gives x = 0 for every method; an empty cube gives an empty result."""
    A = sy.gaussian_phi(10, 25, 17)
    Y = np.zeros((2, 10))
    L = orc.lipschitz(A)
    assert np.all(orc.fista(A, Y, L, 0.1, 0.0, 20)[0] == 0)
    assert np.all(orc.admm(A, Y, 1.0, 0.1, 0.0, 20)[0] == 0)
    assert np.all(orc.gomp(A, Y, 4, 2)[0] == 0)
    assert np.all(orc.biht(A, Y, 4)[0] == 0)
    assert np.all(orc.cosamp(A, Y, 4)[0] == 0)
    assert orc.gomp(A, np.zeros((0, 10)), 4, 2)[0].shape == (0, 25)


# --------------------------------------------------------------------------
# Sparsification pre-processing (Section II): x = Psi^T f, zero x_i where
# |x_i| - mean|x| < T std|x|
# --------------------------------------------------------------------------
def pin_sparsify_worked_example():
    """Hand-worked cases with Psi = I (so x = f exactly).  f = (4, -2, 1, 0): mean |x|
    = 7/4, squared deviations sum to 8.75, sample std sqrt(8.75/3) = 1.7078, population
    std sqrt(8.75/4) = 1.4790.  Centred magnitudes (2.25, 0.25, -0.75, -1.75).
    T = 0.15: sample threshold 0.2562 keeps index 0; population 0.2219 keeps 0 and 1.
    T = 0 keeps 0 and 1; T = -1.1 (sample, -1.8786) keeps everything.
    f = (3, 1, 2, -2), T = 0: mean 2, centred (1, -1, 0, 0): the entries equal to the
    mean are kept (only |x_i| - mu < T sigma zeroes), with their signs."""
    I4 = np.eye(4)
    F = np.array([[4.0, -2.0, 1.0, 0.0], [3.0, 1.0, 2.0, -2.0]])
    X, k = orc.sparsify(F, 0.15, 1, I4)
    assert np.array_equal(X[0], [4, 0, 0, 0]) and np.array_equal(X[1], [3, 0, 0, 0])
    assert list(k) == [1, 1]
    X, k = orc.sparsify(F, 0.15, 0, I4)
    assert np.array_equal(X[0], [4, -2, 0, 0]) and list(k)[0] == 2
    X, k = orc.sparsify(F, 0.0, 1, I4)
    assert np.array_equal(X[0], [4, -2, 0, 0])
    assert np.array_equal(X[1], [3, 0, 2, -2]) and list(k) == [2, 3]
    X, k = orc.sparsify(F[:1], -1.1, 1, I4)
    assert np.array_equal(X[0], F[0]) and list(k) == [3]  # the kept 0 is not counted


def pin_sparsify_transform():
    """With every coefficient kept (T very negative) the output is the analysis
    transform x = Psi^T f: for the DCT-II that is the orthonormal DCT-II of f (library
    routine), and for a random orthogonal Psi it is Psi^T f."""
    F = _rng(21).standard_normal((5, 200))
    X, k = orc.sparsify(F, -1e9)
    assert np.abs(X - scipy.fft.dct(F, type=2, norm="ortho", axis=1)).max() < 1e-12
    assert list(k) == [200] * 5
    Q = rand_orthogonal(40, 22)
    F = _rng(23).standard_normal((3, 40))
    X, _ = orc.sparsify(F, -1e9, 1, Q)
    assert np.abs(X - F @ Q).max() < 1e-12


def pin_sparsify_monotone_and_scale_free():
    """Section II: a larger T keeps fewer coefficients (the kept sets are nested), and
    scaling a spectrum scales mean and std alike, so the kept set does not change."""
    F = sy.powerlaw_coeffs(40, 120, 24) @ orc.dct2_psi(120).T + \
        0.01 * _rng(25).standard_normal((40, 120))
    prev = None
    for T in (-0.5, 0.0, 0.1, 0.5, 1.0, 2.0):
        X, k = orc.sparsify(F, T)
        keep = X != 0
        if prev is not None:
            assert np.all(keep <= prev)  # nested
        prev = keep
        Xs, ks = orc.sparsify(4.0 * F, T)
        assert np.array_equal(Xs != 0, keep) and np.array_equal(ks, k)
        assert np.abs(Xs - 4.0 * X).max() < 1e-12
    # at T = 0 a coefficient survives exactly when its magnitude reaches the mean
    X0, _ = orc.sparsify(F, 0.0)
    x = scipy.fft.dct(F, type=2, norm="ortho", axis=1)
    a = np.abs(x)
    far = np.abs(a - a.mean(axis=1, keepdims=True)) > 1e-9
    assert np.array_equal((X0 != 0)[far], (a >= a.mean(axis=1, keepdims=True))[far])


# --------------------------------------------------------------------------
# The paper's complex setup (Section II): unitary DFT Psi, Phi keeping M rows
# --------------------------------------------------------------------------
def _rows(M, N, seed):
    return np.sort(_rng(seed).choice(N, M, replace=False)).astype(np.int32)


def _crandn(shape, seed):
    g = _rng(seed)
    return g.standard_normal(shape) + 1j * g.standard_normal(shape)


def pin_dft_partial_fourier():
    """Psi is numpy's orthonormal FFT matrix (library routine); the partial-Fourier A has
    orthonormal rows; A x is the FFT of x at the kept samples."""
    for N in (8, 120, 200):
        Psi = orc.dft_psi(N)
        assert np.abs(Psi - np.fft.fft(np.eye(N), norm="ortho", axis=0)).max() < 1e-12
        M = (2 * N) // 5
        rows = _rows(M, N, N)
        A = orc.partial_fourier(M, N, rows)
        assert np.abs(A @ A.conj().T - np.eye(M)).max() < 1e-12
        x = _crandn(N, N + 1)
        assert np.abs(A @ x - np.fft.fft(x, norm="ortho")[rows]).max() < 1e-12


def _csoft_np(a, t):
    return np.maximum(np.abs(a) - t, 0.0) * np.exp(1j * np.angle(a))


def pin_cfista_closed_forms():
    """First iterate from zero: x1 = modulus-soft(A^H y / L, lambda / L) (the proximal map
    of the complex l1 norm).  With the full unitary DFT (M = N, L = 1) the LASSO solution
    is modulus-soft(Psi^H y, lambda), reached at once."""
    N, M = 64, 26
    A = orc.partial_fourier(M, N, _rows(M, N, 5))
    Y = _crandn((3, M), 6)
    lam, L = 0.05, 1.0
    X1, _ = orc.cfista(A, Y, L, lam, 0.0, 1)
    assert np.abs(X1 - _csoft_np(Y @ A.conj() / L, lam / L)).max() < 1e-12
    Psi = orc.dft_psi(N)
    Yf = _crandn((3, N), 7)
    Xf, _ = orc.cfista(Psi, Yf, 1.0, lam, 0.0, 40)
    assert np.abs(Xf - _csoft_np(np.fft.ifft(Yf, norm="ortho", axis=1), lam)).max() < 1e-12


def pin_cfista_kkt():
    """At convergence the complex LASSO optimality conditions hold: g = A^H (y - A x)
    equals lambda x_k / |x_k| on the support and has modulus <= lambda off it."""
    N, M = 64, 26
    A = orc.partial_fourier(M, N, _rows(M, N, 8))
    xt = np.zeros((2, N), dtype=complex)
    xt[:, [3, 17, 40]] = _crandn((2, 3), 9)
    Y = xt @ A.T + 0.01 * _crandn((2, M), 10)
    lam = 0.02
    X, _ = orc.cfista(A, Y, 1.0, lam, 0.0, 5000)
    for x, y in zip(X, Y):
        g = A.conj().T @ (y - A @ x)
        on = np.abs(x) > 1e-9
        assert on.sum() >= 2
        assert np.abs(g[on] - lam * x[on] / np.abs(x[on])).max() < 1e-7
        assert np.abs(g[~on]).max() <= lam * (1 + 1e-7)


def pin_cadmm_closed_forms():
    """First iterate from zero: x1 = (A^H A + rho I)^{-1} A^H y = A^H y / (1 + rho) for a
    partial Fourier A (orthonormal rows, Woodbury).  With the full unitary DFT the
    fixed point is the LASSO solution modulus-soft(Psi^H y, lambda) (threshold
    lambda / rho in the z-step, reading R1), here with rho = 2."""
    N, M = 64, 26
    A = orc.partial_fourier(M, N, _rows(M, N, 16))
    Y = _crandn((3, M), 17)
    X1, _ = orc.cadmm(A, Y, 2.0, 0.05, 0.0, 1)
    assert np.abs(X1 - (Y @ A.conj()) / 3.0).max() < 1e-12
    Psi = orc.dft_psi(N)
    Yf = _crandn((3, N), 18)
    Xf, _ = orc.cadmm(Psi, Yf, 2.0, 0.05, 0.0, 400)
    assert np.abs(Xf - _csoft_np(np.fft.ifft(Yf, norm="ortho", axis=1), 0.05)).max() < 1e-10


def pin_complex_reduces_to_real():
    """On real data the complex routines take every step the real ones take: equal
    results and iteration counts to those of the (independently pinned) real oracle."""
    A = sy.gaussian_phi(20, 40, 11)
    Y = sy.sparse_coeffs(5, 40, 4, 11, "separated") @ A.T + 0.01 * _rng(11).standard_normal(
        (5, 20))
    L = orc.lipschitz(A)
    Xr = orc.fista(A, Y, L, 1e-2, 0.0, 150)[0]
    Xc, _ = orc.cfista(A, Y, L, 1e-2, 0.0, 150)
    assert np.abs(Xc - Xr).max() < 1e-10 and np.abs(Xc.imag).max() == 0.0
    Xr, itr, _ = orc.gomp(A, Y, 6, 2)
    Xc, itc = orc.cgomp(A, Y, 6, 2)
    assert np.array_equal(itr, itc) and np.abs(Xc - Xr).max() < 1e-10
    Xr, itr, _ = orc.cosamp(A, Y, 5)
    Xc, itc = orc.ccosamp(A, Y, 5)
    assert np.array_equal(itr, itc) and np.abs(Xc - Xr).max() < 1e-10
    Xr = orc.admm(A, Y, 1.5, 1e-2, 0.0, 120)[0]
    Xc, _ = orc.cadmm(A, Y, 1.5, 1e-2, 0.0, 120)
    assert np.abs(Xc - Xr).max() < 1e-10
    for mu in (0.1, 1.0):
        Xr, itr, _ = orc.biht(A, Y, 5, mu)
        Xc, itc = orc.cbiht(A, Y, 5, mu)
        assert np.array_equal(itr, itc) and np.abs(Xc - Xr).max() < 1e-10


def pin_cgomp_is_complex_omp():
    """gOMP with G = 1 is orthogonal matching pursuit: a textbook complex OMP with numpy's
    least squares gives the same iterates."""
    N, M, k = 64, 26, 5
    A = orc.partial_fourier(M, N, _rows(M, N, 12))
    Y = _crandn((4, M), 13)
    X, _ = orc.cgomp(A, Y, k, 1, eps=0.0)
    for x, y in zip(X, Y):
        r, sup = y.copy(), []
        for _ in range(k):
            corr = np.abs(A.conj().T @ r)
            corr[sup] = -1.0
            sup.append(int(np.argmax(corr)))
            s, *_ = np.linalg.lstsq(A[:, sup], y, rcond=None)
            ref = np.zeros(N, dtype=complex)
            ref[sup] = s
            r = y - A @ ref
        assert np.abs(x - ref).max() < 1e-10


def pin_complex_exact_recovery():
    """Noiseless S-sparse complex pixels measured at 2.5x by a partial Fourier matrix
    are recovered exactly by gOMP, CoSaMP and BIHT with mu = 1."""
    N, M, S = 120, 48, 4
    A = orc.partial_fourier(M, N, _rows(M, N, 14))
    Xt = np.zeros((6, N), dtype=complex)
    g = _rng(15)
    for i in range(6):
        Xt[i, g.choice(N, S, replace=False)] = (1.0 + g.random(S)) * np.exp(
            2j * np.pi * g.random(S))
    Y = Xt @ A.T
    Xg, _ = orc.cgomp(A, Y, S, 1)
    assert np.abs(Xg - Xt).max() < 1e-10
    Xc, _ = orc.ccosamp(A, Y, S)
    assert np.abs(Xc - Xt).max() < 1e-10
    Xb, _ = orc.cbiht(A, Y, S, 1.0)
    assert np.abs(Xb - Xt).max() < 1e-10


ALL_PINS = [v for k, v in sorted(globals().items()) if k.startswith("pin_")]
