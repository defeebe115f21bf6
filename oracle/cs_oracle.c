/*
 * cs_oracle.c -- plain, slow, FP64 CPU oracle for per-pixel sparse recovery of a
 * compressively sensed hyperspectral cube (Justo et al., "A Comparative Study of
 * Compressive Sensing Algorithms for Hyperspectral Imaging Reconstruction").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this file.  The GPU library never links,
 * calls or includes it, and it shares no code with the GPU library.
 *
 * Every routine follows the paper's statement directly, pixel by pixel, in
 * double precision, with no blocking, fusion or reordering:
 *   - signal model y = Phi f = Phi Psi x = A x          (Section II, Eq. 1)
 *   - LASSO objective 1/2||Ax-y||^2 + lambda||x||_1     (Section II-A, Eq. 2)
 *   - Lipschitz constant L = lambda_max(A^T A)          (Section II-A, after Eq. 2)
 *   - FISTA  (Algorithm 1), ADMM (Algorithm 2), gOMP (Algorithm 3),
 *     BIHT (Algorithm 4, backtracking IHT), CoSaMP (Algorithm 5)
 *   - stopping rule Delta = ||r^i - r^{i-1}||_2 < eps   (Section II-A)
 *
 * Readings where the paper is silent or ambiguous (all listed in the design notes):
 *   R1  ADMM soft threshold uses lambda/alpha (Boyd's scaled form), so the fixed
 *       point is the Eq. 2 LASSO solution; Algorithm 2 prints lambda*alpha.
 *   R2  Psi is the orthonormal DCT-II synthesis matrix (real), Psi = C^T with
 *       C[k][n] = a_k cos(pi (2n+1) k / 2N), a_0 = sqrt(1/N), a_k = sqrt(2/N).
 *   R3  argmax_k orders by |v| descending, ties to the lower index.
 *   R4  gOMP stops after min(max_iters, kappa, floor(M/G)) iterations at most.
 *   R5  q = argmax_kappa(|x|) ranges over the current support only; if the
 *       support holds <= kappa atoms, q is the whole support.
 *   R6  B^+ y is the minimum-norm least-squares solution (pinv semantics):
 *       Householder QR when B has full column rank, one-sided Jacobi SVD otherwise.
 *   R7  sign(0) = 0 in the soft threshold.
 *   R8  The loop runs while Delta >= eps and fewer than max_iters iterations ran;
 *       eps = 0 gives a fixed iteration count.  The time cap t_conv is not used.
 *   R9  ADMM returns the x iterate of Algorithm 2 (the variable its residual uses).
 *   R11 The paper's own transform (Section II): Psi is the unitary DFT, Psi[n][k] =
 *       exp(-2 pi i n k / N) / sqrt(N) (f in the DFT domain, x = Psi^H f in the IDFT
 *       domain), Phi keeps M of the N spectral samples (rows), so A = Psi(rows, :) and
 *       y, x, f are complex.  FISTA thresholds the modulus (x_k scaled by
 *       max(|a_k| - t, 0) / |a_k|, 0 at a_k = 0), and so does ADMM's z-step; the greedy
 *       selections rank |A^H r|, |u| and |s|; least squares by complex Householder QR
 *       (full column rank required); A^* is the conjugate transpose.
 *   R10 Sparsification (Section II): x = Psi^T f (Psi orthonormal, so Psi^T = Psi^{-1});
 *       mu and sigma are the mean and the standard deviation of |x| over the N
 *       coefficients, sigma normalised by N - ddof (ddof = 1: sample form, the default;
 *       0: population form); x_i is zeroed when |x_i| - mu < T sigma and kept otherwise;
 *       kappa = ||x_s||_0.
 *
 * Layout: all matrices row-major. A is M x N, X is P x N, Y is P x M.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_ERR_ARG -1
#define OR_ERR_NOMEM -2

/* ------------------------------------------------------------------------- */
/* small dense helpers                                                        */
/* ------------------------------------------------------------------------- */

static double dot(int n, const double *a, const double *b) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

/* out[m] = sum_n A[m][n] v[n]  (A x) */
static void mat_vec(int M, int N, const double *A, const double *v, double *out) {
  for (int m = 0; m < M; ++m) out[m] = dot(N, A + (size_t)m * N, v);
}

/* out[n] = sum_m A[m][n] v[m]  (A^T v; A is real so A^* = A^T) */
static void mat_t_vec(int M, int N, const double *A, const double *v, double *out) {
  for (int n = 0; n < N; ++n) {
    double s = 0.0;
    for (int m = 0; m < M; ++m) s += A[(size_t)m * N + n] * v[m];
    out[n] = s;
  }
}

/* soft threshold, Algorithm 1 step 2 / Algorithm 2 step 2; sign(0) = 0 (R7) */
static double soft(double a, double thr) {
  double mag = fabs(a) - thr;
  if (mag <= 0.0) return 0.0;
  return a > 0.0 ? mag : (a < 0.0 ? -mag : 0.0);
}

/* ------------------------------------------------------------------------- */
/* Section II, Eq. 1: transform and dictionary                                */
/* ------------------------------------------------------------------------- */

/* Psi[n][k] = a_k cos(pi (2n+1) k / (2N)) -- column k is the k-th cosine atom (R2) */
void or_dct2_psi(int N, double *Psi) {
  const double pi = 3.14159265358979323846;
  for (int n = 0; n < N; ++n)
    for (int k = 0; k < N; ++k) {
      double a = (k == 0) ? sqrt(1.0 / N) : sqrt(2.0 / N);
      Psi[(size_t)n * N + k] = a * cos(pi * (2.0 * n + 1.0) * k / (2.0 * N));
    }
}

/* A = Phi Psi (Eq. 1): A[m][k] = sum_n Phi[m][n] Psi[n][k] */
void or_dictionary(int M, int N, const double *Phi, const double *Psi, double *A) {
  for (int m = 0; m < M; ++m)
    for (int k = 0; k < N; ++k) {
      double s = 0.0;
      for (int n = 0; n < N; ++n) s += Phi[(size_t)m * N + n] * Psi[(size_t)n * N + k];
      A[(size_t)m * N + k] = s;
    }
}

/* y = A x (+ e) for every pixel (Eq. 1).  E may be NULL. */
void or_measure(int M, int N, const double *A, int64_t P, const double *X, const double *E,
                double *Y) {
  for (int64_t p = 0; p < P; ++p) {
    mat_vec(M, N, A, X + p * N, Y + p * M);
    if (E)
      for (int m = 0; m < M; ++m) Y[p * M + m] += E[p * M + m];
  }
}

/* ------------------------------------------------------------------------- */
/* Sparsification pre-processing (Section II, reading R10), pixel by pixel:   */
/* x = Psi^T f; mu = mean |x|; sigma = std |x| (N - ddof); x_i = 0 where      */
/* |x_i| - mu < T sigma.  kappa (may be NULL) = number of nonzero kept x_i.   */
/* ------------------------------------------------------------------------- */
int or_sparsify(int N, const double *Psi, int64_t P, const double *F, double T, int ddof,
                double *X, int32_t *kappa) {
  if (N <= 0 || P < 0 || (ddof != 0 && ddof != 1)) return OR_ERR_ARG;
  double *a = (double *)malloc(sizeof(double) * N);
  if (!a) return OR_ERR_NOMEM;
  for (int64_t p = 0; p < P; ++p) {
    const double *f = F + p * N;
    double *x = X + p * N;
    for (int i = 0; i < N; ++i) { /* x_i = sum_n Psi[n][i] f_n */
      double s = 0.0;
      for (int n = 0; n < N; ++n) s += Psi[(size_t)n * N + i] * f[n];
      x[i] = s;
      a[i] = fabs(s);
    }
    double mu = 0.0;
    for (int i = 0; i < N; ++i) mu += a[i];
    mu /= N;
    double ss = 0.0;
    for (int i = 0; i < N; ++i) ss += (a[i] - mu) * (a[i] - mu);
    double sigma = N - ddof > 0 ? sqrt(ss / (N - ddof)) : 0.0;
    int32_t nz = 0;
    for (int i = 0; i < N; ++i) {
      if (a[i] - mu < T * sigma) x[i] = 0.0;
      if (x[i] != 0.0) ++nz;
    }
    if (kappa) kappa[p] = nz;
  }
  free(a);
  return OR_OK;
}

/* ------------------------------------------------------------------------- */
/* Lipschitz constant L = lambda_max(A^* A)  (Section II-A)                   */
/* Cyclic Jacobi eigenvalue iteration on the M x M matrix A A^T, whose        */
/* nonzero eigenvalues are those of A^T A.                                    */
/* ------------------------------------------------------------------------- */
double or_lipschitz(int M, int N, const double *A) {
  double *S = (double *)malloc(sizeof(double) * M * M);
  if (!S) return -1.0;
  for (int i = 0; i < M; ++i)
    for (int j = 0; j < M; ++j) S[i * M + j] = dot(N, A + (size_t)i * N, A + (size_t)j * N);
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < M; ++i)
      for (int j = 0; j < M; ++j) {
        tot += S[i * M + j] * S[i * M + j];
        if (i != j) off += S[i * M + j] * S[i * M + j];
      }
    if (off <= 1e-30 * tot) break;
    for (int p = 0; p < M; ++p)
      for (int q = p + 1; q < M; ++q) {
        double apq = S[p * M + q];
        if (apq == 0.0) continue;
        double app = S[p * M + p], aqq = S[q * M + q];
        double theta = (aqq - app) / (2.0 * apq);
        double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < M; ++k) { /* rotate columns p, q */
          double skp = S[k * M + p], skq = S[k * M + q];
          S[k * M + p] = c * skp - s * skq;
          S[k * M + q] = s * skp + c * skq;
        }
        for (int k = 0; k < M; ++k) { /* rotate rows p, q */
          double spk = S[p * M + k], sqk = S[q * M + k];
          S[p * M + k] = c * spk - s * sqk;
          S[q * M + k] = s * spk + c * sqk;
        }
      }
  }
  double lmax = S[0];
  for (int i = 1; i < M; ++i)
    if (S[i * M + i] > lmax) lmax = S[i * M + i];
  free(S);
  return lmax;
}

/* ------------------------------------------------------------------------- */
/* argmax_k(|v|) over a candidate index list (R3): repeatedly take the        */
/* remaining candidate with the largest |v|, the lower index winning ties.    */
/* Writes k indices to out; returns the relative gap between the k-th and     */
/* (k+1)-th largest |v| (1.0 if there is no (k+1)-th candidate).              */
/* ------------------------------------------------------------------------- */
static double argmax_k(const double *v, const int *cand, int ncand, int k, int *out,
                       unsigned char *taken) {
  for (int i = 0; i < ncand; ++i) taken[i] = 0;
  double kth = 0.0;
  for (int j = 0; j < k; ++j) {
    int best = -1;
    for (int i = 0; i < ncand; ++i) {
      if (taken[i]) continue;
      if (best < 0) { best = i; continue; }
      double a = fabs(v[cand[i]]), b = fabs(v[cand[best]]);
      if (a > b || (a == b && cand[i] < cand[best])) best = i;
    }
    taken[best] = 1;
    out[j] = cand[best];
    kth = fabs(v[cand[best]]);
  }
  double next = -1.0;
  for (int i = 0; i < ncand; ++i)
    if (!taken[i] && fabs(v[cand[i]]) > next) next = fabs(v[cand[i]]);
  if (next < 0.0) return 1.0;
  if (kth == 0.0) return 0.0;
  return (kth - next) / kth;
}

/* ------------------------------------------------------------------------- */
/* s = B^+ y with B = A(:, c): minimum-norm least squares (R6).               */
/* ------------------------------------------------------------------------- */

/* One-sided Jacobi SVD of W (m x n, m >= n, row-major, overwritten by U*Sigma),
 * V (n x n) accumulates the right rotations.  sig receives the column norms. */
static void jacobi_svd(int m, int n, double *W, double *V, double *sig) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) V[i * n + j] = (i == j) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 80; ++sweep) {
    int rotated = 0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        double alpha = 0.0, beta = 0.0, gamma = 0.0;
        for (int i = 0; i < m; ++i) {
          double wp = W[i * n + p], wq = W[i * n + q];
          alpha += wp * wp;
          beta += wq * wq;
          gamma += wp * wq;
        }
        if (fabs(gamma) <= 1e-15 * sqrt(alpha * beta) || gamma == 0.0) continue;
        rotated = 1;
        double zeta = (beta - alpha) / (2.0 * gamma);
        double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
        for (int i = 0; i < m; ++i) {
          double wp = W[i * n + p], wq = W[i * n + q];
          W[i * n + p] = c * wp - s * wq;
          W[i * n + q] = s * wp + c * wq;
        }
        for (int i = 0; i < n; ++i) {
          double vp = V[i * n + p], vq = V[i * n + q];
          V[i * n + p] = c * vp - s * vq;
          V[i * n + q] = s * vp + c * vq;
        }
      }
    if (!rotated) break;
  }
  for (int j = 0; j < n; ++j) {
    double s = 0.0;
    for (int i = 0; i < m; ++i) s += W[i * n + j] * W[i * n + j];
    sig[j] = sqrt(s);
  }
}

/* pinv(B) y through the SVD: B = U S V^T  =>  B^+ y = V S^+ U^T y, with the
 * singular-value cutoff max(rows, cols) * eps * sigma_max (MATLAB pinv default). */
static void pinv_svd(int M, int nc, const double *B, const double *y, double *s, double *work) {
  const double eps = 2.220446049250313e-16;
  if (nc <= M) {
    /* B is M x nc with M >= nc: SVD of B directly. */
    double *W = work, *V = W + (size_t)M * nc, *sig = V + (size_t)nc * nc;
    memcpy(W, B, sizeof(double) * M * nc);
    jacobi_svd(M, nc, W, V, sig);
    double smax = 0.0;
    for (int j = 0; j < nc; ++j) smax = fmax(smax, sig[j]);
    double tol = (M > nc ? M : nc) * eps * smax;
    for (int i = 0; i < nc; ++i) s[i] = 0.0;
    for (int j = 0; j < nc; ++j) {
      if (sig[j] <= tol) continue;
      double uty = 0.0; /* u_j = W(:,j)/sig_j */
      for (int i = 0; i < M; ++i) uty += W[i * nc + j] * y[i];
      uty /= sig[j] * sig[j];
      for (int i = 0; i < nc; ++i) s[i] += V[i * nc + j] * uty;
    }
  } else {
    /* nc > M: SVD of B^T (nc x M).  B^T = U S V^T  =>  B^+ = U S^+ V^T. */
    double *W = work, *V = W + (size_t)nc * M, *sig = V + (size_t)M * M;
    for (int i = 0; i < nc; ++i)
      for (int j = 0; j < M; ++j) W[i * M + j] = B[j * nc + i];
    jacobi_svd(nc, M, W, V, sig);
    double smax = 0.0;
    for (int j = 0; j < M; ++j) smax = fmax(smax, sig[j]);
    double tol = nc * eps * smax;
    for (int i = 0; i < nc; ++i) s[i] = 0.0;
    for (int j = 0; j < M; ++j) {
      if (sig[j] <= tol) continue;
      double vty = 0.0;
      for (int i = 0; i < M; ++i) vty += V[i * M + j] * y[i];
      vty /= sig[j] * sig[j];
      for (int i = 0; i < nc; ++i) s[i] += W[i * M + j] * vty; /* u_j sig_j = W(:,j) */
    }
  }
}

/* Householder QR least squares for B (M x nc, nc <= M).  Returns 0 on success,
 * 1 if B is numerically rank deficient (caller falls back to the SVD). */
static int qr_lstsq(int M, int nc, const double *B, const double *y, double *s, double *work) {
  const double eps = 2.220446049250313e-16;
  double *R = work, *b = R + (size_t)M * nc, *v = b + M;
  memcpy(R, B, sizeof(double) * M * nc);
  memcpy(b, y, sizeof(double) * M);
  for (int j = 0; j < nc; ++j) {
    double norm = 0.0;
    for (int i = j; i < M; ++i) norm += R[i * nc + j] * R[i * nc + j];
    norm = sqrt(norm);
    if (norm == 0.0) return 1;
    double alpha = R[j * nc + j] > 0 ? -norm : norm;
    for (int i = j; i < M; ++i) v[i] = R[i * nc + j];
    v[j] -= alpha;
    double vv = 0.0;
    for (int i = j; i < M; ++i) vv += v[i] * v[i];
    if (vv > 0.0) {
      for (int k = j; k < nc; ++k) { /* R(:,k) -= 2 v (v^T R(:,k)) / (v^T v) */
        double d = 0.0;
        for (int i = j; i < M; ++i) d += v[i] * R[i * nc + k];
        d = 2.0 * d / vv;
        for (int i = j; i < M; ++i) R[i * nc + k] -= d * v[i];
      }
      double d = 0.0;
      for (int i = j; i < M; ++i) d += v[i] * b[i];
      d = 2.0 * d / vv;
      for (int i = j; i < M; ++i) b[i] -= d * v[i];
    }
  }
  double rmax = 0.0;
  for (int j = 0; j < nc; ++j) rmax = fmax(rmax, fabs(R[j * nc + j]));
  for (int j = 0; j < nc; ++j)
    if (fabs(R[j * nc + j]) <= (M > nc ? M : nc) * eps * rmax) return 1;
  for (int j = nc - 1; j >= 0; --j) { /* back substitution R s = Q^T y */
    double acc = b[j];
    for (int k = j + 1; k < nc; ++k) acc -= R[j * nc + k] * s[k];
    s[j] = acc / R[j * nc + j];
  }
  return 0;
}

/* s = A(:, c)^+ y.  work must hold at least 2*M*(N+1) + (2N+2)*(N+1) doubles. */
static void support_lstsq(int M, int N, const double *A, const int *c, int nc, const double *y,
                          double *s, double *work) {
  if (nc == 0) return;
  double *B = work, *w2 = B + (size_t)M * nc;
  for (int i = 0; i < M; ++i)
    for (int j = 0; j < nc; ++j) B[i * nc + j] = A[(size_t)i * N + c[j]];
  if (nc <= M && qr_lstsq(M, nc, B, y, s, w2) == 0) return;
  pinv_svd(M, nc, B, y, s, w2);
}

/* exported for tests: s = A(:, c)^+ y */
int or_support_lstsq(int M, int N, const double *A, const int *c, int nc, const double *y,
                     double *s) {
  if (M <= 0 || N <= 0 || nc < 0 || nc > N) return OR_ERR_ARG;
  size_t wsz = (size_t)2 * M * (N + 1) + (size_t)(2 * N + 2) * (N + 1) + 64;
  double *work = (double *)malloc(sizeof(double) * wsz);
  if (!work) return OR_ERR_NOMEM;
  support_lstsq(M, N, A, c, nc, y, s, work);
  free(work);
  return OR_OK;
}

/* exported for tests: argmax_k(|v|) over all N indices */
double or_argmax_k(int N, const double *v, int k, int *out) {
  int *cand = (int *)malloc(sizeof(int) * N);
  unsigned char *taken = (unsigned char *)malloc(N);
  for (int i = 0; i < N; ++i) cand[i] = i;
  double gap = argmax_k(v, cand, N, k, out, taken);
  free(cand);
  free(taken);
  return gap;
}

/* residual r = y - A x and Delta = ||r - r_prev||_2 (common step of Alg. 1-5) */
static double residual_delta(int M, int N, const double *A, const double *y, const double *x,
                             double *r, double *r_prev, double *tmp) {
  mat_vec(M, N, A, x, tmp);
  for (int m = 0; m < M; ++m) r[m] = y[m] - tmp[m];
  double d = 0.0;
  for (int m = 0; m < M; ++m) d += (r[m] - r_prev[m]) * (r[m] - r_prev[m]);
  memcpy(r_prev, r, sizeof(double) * M);
  return sqrt(d);
}

static void set_threads(int n_threads) {
#ifdef _OPENMP
  if (n_threads > 0) omp_set_num_threads(n_threads);
#else
  (void)n_threads;
#endif
}

/* ------------------------------------------------------------------------- */
/* Algorithm 1: FISTA                                                         */
/* ------------------------------------------------------------------------- */
int or_fista(int M, int N, const double *A, int64_t P, const double *Y, double *X, double L,
             double lambda, double eps, int max_iters, int32_t *iters_out, int n_threads) {
  if (M <= 0 || N <= 0 || P < 0 || !(L > 0.0) || lambda < 0.0 || max_iters < 0)
    return OR_ERR_ARG;
  set_threads(n_threads);
#pragma omp parallel
  {
    double *buf = (double *)malloc(sizeof(double) * (5 * N + 4 * M));
    double *x = buf, *x_prev = x + N, *z = x_prev + N, *aux = z + N, *g = aux + N;
    double *v = g + N, *r = v + M, *r_prev = r + M, *tmp = r_prev + M;
#pragma omp for schedule(dynamic, 16)
    for (int64_t p = 0; p < P; ++p) {
      const double *y = Y + p * M;
      for (int n = 0; n < N; ++n) x[n] = z[n] = 0.0; /* x^0 = 0, z^0 = x^0 */
      memcpy(r_prev, y, sizeof(double) * M);          /* r^0 = y */
      double t = 1.0, delta = 1.0;                    /* t^0 = 1, Delta = 1 */
      int it = 0;
      while (delta >= eps && it < max_iters) {
        /* 1. aux = z - (1/L) A^*(A z - y) */
        mat_vec(M, N, A, z, v);
        for (int m = 0; m < M; ++m) v[m] -= y[m];
        mat_t_vec(M, N, A, v, g);
        for (int n = 0; n < N; ++n) aux[n] = z[n] - g[n] / L;
        /* 2. x = sign(aux) .* max(|aux| - lambda/L, 0) */
        memcpy(x_prev, x, sizeof(double) * N);
        for (int n = 0; n < N; ++n) x[n] = soft(aux[n], lambda / L);
        /* 3. t^i = (1 + sqrt(1 + 4 t^2)) / 2 */
        double t_new = (1.0 + sqrt(1.0 + 4.0 * t * t)) / 2.0;
        /* 4. z = x + ((t^{i-1} - 1) / t^i) (x - x_prev) */
        for (int n = 0; n < N; ++n) z[n] = x[n] + ((t - 1.0) / t_new) * (x[n] - x_prev[n]);
        t = t_new;
        /* 5. r = y - A x, Delta = ||r - r_prev|| */
        delta = residual_delta(M, N, A, y, x, r, r_prev, tmp);
        ++it;
      }
      memcpy(X + p * N, x, sizeof(double) * N);
      if (iters_out) iters_out[p] = it;
    }
    free(buf);
  }
  return OR_OK;
}

/* ------------------------------------------------------------------------- */
/* Algorithm 2: ADMM.  The x-step solves (A^T A + alpha I) x = A^T y +         */
/* alpha (z - w) through a Cholesky factor computed once.                     */
/* ------------------------------------------------------------------------- */

/* In-place Cholesky K = L L^T (lower), n x n.  Returns nonzero if not SPD. */
static int cholesky(int n, double *K) {
  for (int j = 0; j < n; ++j) {
    double d = K[j * n + j];
    for (int k = 0; k < j; ++k) d -= K[j * n + k] * K[j * n + k];
    if (!(d > 0.0)) return 1;
    d = sqrt(d);
    K[j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double s = K[i * n + j];
      for (int k = 0; k < j; ++k) s -= K[i * n + k] * K[j * n + k];
      K[i * n + j] = s / d;
    }
  }
  return 0;
}

/* Solve L L^T x = b in place (b overwritten by x). */
static void cholesky_solve(int n, const double *Lf, double *b) {
  for (int i = 0; i < n; ++i) {
    double s = b[i];
    for (int k = 0; k < i; ++k) s -= Lf[i * n + k] * b[k];
    b[i] = s / Lf[i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = b[i];
    for (int k = i + 1; k < n; ++k) s -= Lf[k * n + i] * b[k];
    b[i] = s / Lf[i * n + i];
  }
}

int or_admm(int M, int N, const double *A, int64_t P, const double *Y, double *X, double alpha,
            double lambda, double eps, int max_iters, int32_t *iters_out, int n_threads) {
  if (M <= 0 || N <= 0 || P < 0 || !(alpha > 0.0) || lambda < 0.0 || max_iters < 0)
    return OR_ERR_ARG;
  double *K = (double *)malloc(sizeof(double) * N * N);
  if (!K) return OR_ERR_NOMEM;
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) {
      double s = 0.0;
      for (int m = 0; m < M; ++m) s += A[(size_t)m * N + i] * A[(size_t)m * N + j];
      K[i * N + j] = s + (i == j ? alpha : 0.0);
    }
  if (cholesky(N, K)) {
    free(K);
    return OR_ERR_ARG;
  }
  set_threads(n_threads);
#pragma omp parallel
  {
    double *buf = (double *)malloc(sizeof(double) * (5 * N + 3 * M));
    double *x = buf, *z = x + N, *w = z + N, *aty = w + N, *rhs = aty + N;
    double *r = rhs + N, *r_prev = r + M, *tmp = r_prev + M;
#pragma omp for schedule(dynamic, 16)
    for (int64_t p = 0; p < P; ++p) {
      const double *y = Y + p * M;
      for (int n = 0; n < N; ++n) x[n] = z[n] = w[n] = 0.0; /* x^0 = z^0 = w^0 = 0 */
      memcpy(r_prev, y, sizeof(double) * M);                 /* r^0 = y */
      mat_t_vec(M, N, A, y, aty);
      double delta = 1.0;
      int it = 0;
      while (delta >= eps && it < max_iters) {
        /* 1. x = (A^T A + alpha I)^{-1} (A^T y + alpha (z - w)) */
        for (int n = 0; n < N; ++n) rhs[n] = aty[n] + alpha * (z[n] - w[n]);
        cholesky_solve(N, K, rhs);
        memcpy(x, rhs, sizeof(double) * N);
        /* 2. z = sign(x + w) .* max(|x + w| - lambda/alpha, 0)   (R1) */
        for (int n = 0; n < N; ++n) z[n] = soft(x[n] + w[n], lambda / alpha);
        /* 3. w = w + x - z */
        for (int n = 0; n < N; ++n) w[n] = w[n] + x[n] - z[n];
        /* 4. r = y - A x, Delta */
        delta = residual_delta(M, N, A, y, x, r, r_prev, tmp);
        ++it;
      }
      memcpy(X + p * N, x, sizeof(double) * N);
      if (iters_out) iters_out[p] = it;
    }
    free(buf);
  }
  free(K);
  return OR_OK;
}

/* ------------------------------------------------------------------------- */
/* Greedy workspace                                                           */
/* ------------------------------------------------------------------------- */
typedef struct {
  double *x, *p, *s, *r, *r_prev, *tmp, *lsw;
  int *c, *theta, *q, *cand, *merged;
  unsigned char *taken, *in_c;
} greedy_ws;

static int ws_alloc(greedy_ws *w, int M, int N) {
  size_t lsw = (size_t)2 * M * (N + 1) + (size_t)(2 * N + 2) * (N + 1) + 64;
  w->x = (double *)malloc(sizeof(double) * (3 * N + 3 * M + lsw));
  w->c = (int *)malloc(sizeof(int) * 5 * N);
  w->taken = (unsigned char *)malloc(2 * N);
  if (!w->x || !w->c || !w->taken) return 1;
  w->p = w->x + N;
  w->s = w->p + N;
  w->r = w->s + N;
  w->r_prev = w->r + M;
  w->tmp = w->r_prev + M;
  w->lsw = w->tmp + M;
  w->theta = w->c + N;
  w->q = w->theta + N;
  w->cand = w->q + N;
  w->merged = w->cand + N;
  w->in_c = w->taken + N;
  return 0;
}

static void ws_free(greedy_ws *w) {
  free(w->x);
  free(w->c);
  free(w->taken);
}

/* c <- Theta U c, keeping c as a list (no repeated atoms).  Returns |c|. */
static int support_union(int N, int *c, int nc, const int *theta, int nt, unsigned char *in_c) {
  for (int i = 0; i < N; ++i) in_c[i] = 0;
  for (int i = 0; i < nc; ++i) in_c[c[i]] = 1;
  for (int j = 0; j < nt; ++j)
    if (!in_c[theta[j]]) {
      in_c[theta[j]] = 1;
      c[nc++] = theta[j];
    }
  return nc;
}

/* ------------------------------------------------------------------------- */
/* Algorithm 3: gOMP                                                          */
/* ------------------------------------------------------------------------- */
int or_gomp(int M, int N, const double *A, int64_t P, const double *Y, double *X, int kappa, int G,
            double eps, int max_iters, int32_t *iters_out, double *margin_out, int n_threads) {
  if (M <= 0 || N <= 0 || P < 0 || kappa < 0 || kappa > N || G < 1 || G > N || max_iters < 0)
    return OR_ERR_ARG;
  int cap = max_iters; /* R4 */
  if (kappa < cap) cap = kappa;
  if (M / G < cap) cap = M / G;
  set_threads(n_threads);
#pragma omp parallel
  {
    greedy_ws w;
    int bad = ws_alloc(&w, M, N);
#pragma omp for schedule(dynamic, 4)
    for (int64_t p = 0; p < P; ++p) {
      if (bad) continue;
      const double *y = Y + p * M;
      double margin = 1.0;
      for (int n = 0; n < N; ++n) w.x[n] = 0.0;
      memcpy(w.r_prev, y, sizeof(double) * M); /* r^0 = y */
      int nc = 0;                              /* c^0 = empty */
      for (int n = 0; n < N; ++n) w.cand[n] = n;
      double delta = 1.0;
      int it = 0;
      while (delta >= eps && it < cap) {
        /* 1. p = A^* r, Theta = argmax_G |p|, c = Theta U c */
        mat_t_vec(M, N, A, w.r_prev, w.p);
        margin = fmin(margin, argmax_k(w.p, w.cand, N, G, w.theta, w.taken));
        nc = support_union(N, w.c, nc, w.theta, G, w.in_c);
        /* 2. B = A(:, c), s = B^+ y */
        support_lstsq(M, N, A, w.c, nc, y, w.s, w.lsw);
        /* 3. x = 0, x(c) = s, q = argmax_kappa |x| (over c, R5) */
        for (int n = 0; n < N; ++n) w.x[n] = 0.0;
        for (int j = 0; j < nc; ++j) w.x[w.c[j]] = w.s[j];
        int nq = nc < kappa ? nc : kappa;
        if (nc > kappa) margin = fmin(margin, argmax_k(w.x, w.c, nc, kappa, w.q, w.taken));
        else
          for (int j = 0; j < nc; ++j) w.q[j] = w.c[j];
        /*    B = A(:, q), s = B^+ y, x = 0, x(q) = s */
        support_lstsq(M, N, A, w.q, nq, y, w.s, w.lsw);
        for (int n = 0; n < N; ++n) w.x[n] = 0.0;
        for (int j = 0; j < nq; ++j) w.x[w.q[j]] = w.s[j];
        /* 4. r = y - A x, Delta */
        delta = residual_delta(M, N, A, y, w.x, w.r, w.r_prev, w.tmp);
        ++it;
      }
      memcpy(X + p * N, w.x, sizeof(double) * N);
      if (iters_out) iters_out[p] = it;
      if (margin_out) margin_out[p] = margin;
    }
    if (!bad) ws_free(&w);
  }
  return OR_OK;
}

/* ------------------------------------------------------------------------- */
/* Algorithm 4: BIHT (backtracking iterative hard thresholding)               */
/* ------------------------------------------------------------------------- */
int or_biht(int M, int N, const double *A, int64_t P, const double *Y, double *X, int kappa,
            double mu, double eps, int max_iters, int32_t *iters_out, double *margin_out,
            int n_threads) {
  if (M <= 0 || N <= 0 || P < 0 || kappa < 0 || kappa > N || max_iters < 0) return OR_ERR_ARG;
  set_threads(n_threads);
#pragma omp parallel
  {
    greedy_ws w;
    int bad = ws_alloc(&w, M, N);
#pragma omp for schedule(dynamic, 4)
    for (int64_t p = 0; p < P; ++p) {
      if (bad) continue;
      const double *y = Y + p * M;
      double margin = 1.0;
      double *xa = w.x; /* x_a and x coincide after step 3 (x_a(c) = s, x(c) = s) */
      for (int n = 0; n < N; ++n) xa[n] = 0.0; /* x_a^0 = 0 */
      memcpy(w.r_prev, y, sizeof(double) * M); /* r^0 = y */
      for (int n = 0; n < N; ++n) w.cand[n] = n;
      double delta = 1.0;
      int it = 0;
      while (delta >= eps && it < max_iters) {
        /* 1. u = x_a + mu A^*(y - A x_a) */
        mat_vec(M, N, A, xa, w.tmp);
        for (int m = 0; m < M; ++m) w.tmp[m] = y[m] - w.tmp[m];
        mat_t_vec(M, N, A, w.tmp, w.p);
        for (int n = 0; n < N; ++n) w.p[n] = xa[n] + mu * w.p[n];
        /*    Theta = argmax_kappa |u|, c = supp(x_a), c = Theta U c */
        margin = fmin(margin, argmax_k(w.p, w.cand, N, kappa, w.theta, w.taken));
        int nc = 0;
        for (int n = 0; n < N; ++n)
          if (xa[n] != 0.0) w.c[nc++] = n;
        nc = support_union(N, w.c, nc, w.theta, kappa, w.in_c);
        /* 2. B = A(:, c), s = B^+ y */
        support_lstsq(M, N, A, w.c, nc, y, w.s, w.lsw);
        /* 3. h = argmax_kappa |s|, s outside h = 0, x_a(c) = s, x = 0, x(c) = s */
        double *sfull = w.p; /* scatter s over N to rank it with argmax_k over c */
        for (int n = 0; n < N; ++n) sfull[n] = 0.0;
        for (int j = 0; j < nc; ++j) sfull[w.c[j]] = w.s[j];
        int nh = nc < kappa ? nc : kappa;
        if (nc > kappa) margin = fmin(margin, argmax_k(sfull, w.c, nc, kappa, w.q, w.taken));
        else
          for (int j = 0; j < nc; ++j) w.q[j] = w.c[j];
        for (int n = 0; n < N; ++n) xa[n] = 0.0;
        for (int j = 0; j < nh; ++j) xa[w.q[j]] = sfull[w.q[j]];
        /* 4. r = y - A x, Delta */
        delta = residual_delta(M, N, A, y, xa, w.r, w.r_prev, w.tmp);
        ++it;
      }
      memcpy(X + p * N, xa, sizeof(double) * N);
      if (iters_out) iters_out[p] = it;
      if (margin_out) margin_out[p] = margin;
    }
    if (!bad) ws_free(&w);
  }
  return OR_OK;
}

/* ------------------------------------------------------------------------- */
/* Algorithm 5: CoSaMP                                                        */
/* ------------------------------------------------------------------------- */
int or_cosamp(int M, int N, const double *A, int64_t P, const double *Y, double *X, int kappa,
              double eps, int max_iters, int32_t *iters_out, double *margin_out, int n_threads) {
  if (M <= 0 || N <= 0 || P < 0 || kappa < 0 || 2 * kappa > N || max_iters < 0)
    return OR_ERR_ARG;
  set_threads(n_threads);
#pragma omp parallel
  {
    greedy_ws w;
    int bad = ws_alloc(&w, M, N);
#pragma omp for schedule(dynamic, 4)
    for (int64_t p = 0; p < P; ++p) {
      if (bad) continue;
      const double *y = Y + p * M;
      double margin = 1.0;
      for (int n = 0; n < N; ++n) w.x[n] = 0.0;
      memcpy(w.r_prev, y, sizeof(double) * M); /* r^0 = y */
      int nc = 0;                              /* c^0 = empty */
      for (int n = 0; n < N; ++n) w.cand[n] = n;
      double delta = 1.0;
      int it = 0;
      while (delta >= eps && it < max_iters) {
        /* 1. p = A^* r, Theta = argmax_2kappa |p|, c = Theta U c */
        mat_t_vec(M, N, A, w.r_prev, w.p);
        margin = fmin(margin, argmax_k(w.p, w.cand, N, 2 * kappa, w.theta, w.taken));
        nc = support_union(N, w.c, nc, w.theta, 2 * kappa, w.in_c);
        /* 2. B = A(:, c), s = B^+ y */
        support_lstsq(M, N, A, w.c, nc, y, w.s, w.lsw);
        /* 3. q = argmax_kappa |s|, s = s(q), c = c(q), x = 0, x(c) = s */
        for (int n = 0; n < N; ++n) w.x[n] = 0.0;
        for (int j = 0; j < nc; ++j) w.x[w.c[j]] = w.s[j];
        int nq = nc < kappa ? nc : kappa;
        if (nc > kappa) margin = fmin(margin, argmax_k(w.x, w.c, nc, kappa, w.q, w.taken));
        else
          for (int j = 0; j < nc; ++j) w.q[j] = w.c[j];
        for (int j = 0; j < nq; ++j) w.merged[j] = w.q[j];
        for (int j = 0; j < nq; ++j) w.p[j] = w.x[w.q[j]]; /* s(q), read before x is rebuilt */
        for (int n = 0; n < N; ++n) w.x[n] = 0.0;
        for (int j = 0; j < nq; ++j) w.x[w.merged[j]] = w.p[j];
        nc = nq;
        for (int j = 0; j < nq; ++j) w.c[j] = w.merged[j];
        /* 4. r = y - A x, Delta */
        delta = residual_delta(M, N, A, y, w.x, w.r, w.r_prev, w.tmp);
        ++it;
      }
      memcpy(X + p * N, w.x, sizeof(double) * N);
      if (iters_out) iters_out[p] = it;
      if (margin_out) margin_out[p] = margin;
    }
    if (!bad) ws_free(&w);
  }
  return OR_OK;
}

/* ------------------------------------------------------------------------- */
/* The paper's complex setup (Section II, reading R11): unitary DFT Psi,      */
/* Phi keeping M rows.  Complex arrays are interleaved (re, im) doubles.      */
/* ------------------------------------------------------------------------- */
typedef double complex cplx;

/* Psi[n][k] = exp(-2 pi i n k / N) / sqrt(N) */
void or_dft_psi(int N, cplx *Psi) {
  const double pi = 3.14159265358979323846;
  for (int n = 0; n < N; ++n)
    for (int k = 0; k < N; ++k) {
      /* n k mod N keeps the angle exact for large products */
      const double ang = -2.0 * pi * (double)(((long long)n * k) % N) / N;
      Psi[(size_t)n * N + k] = (cos(ang) + sin(ang) * _Complex_I) / sqrt((double)N);
    }
}

/* A = Phi Psi with Phi keeping the rows rows[0..M): A[m][k] = Psi[rows[m]][k] */
int or_partial_fourier(int M, int N, const int *rows, cplx *A) {
  if (M <= 0 || N <= 0 || M > N) return OR_ERR_ARG;
  cplx *Psi = (cplx *)malloc(sizeof(cplx) * N * N);
  if (!Psi) return OR_ERR_NOMEM;
  or_dft_psi(N, Psi);
  for (int m = 0; m < M; ++m) {
    if (rows[m] < 0 || rows[m] >= N) {
      free(Psi);
      return OR_ERR_ARG;
    }
    for (int k = 0; k < N; ++k) A[(size_t)m * N + k] = Psi[(size_t)rows[m] * N + k];
  }
  free(Psi);
  return OR_OK;
}

/* out = A v */
static void cmat_vec(int M, int N, const cplx *A, const cplx *v, cplx *out) {
  for (int m = 0; m < M; ++m) {
    cplx s = 0.0;
    for (int n = 0; n < N; ++n) s += A[(size_t)m * N + n] * v[n];
    out[m] = s;
  }
}

/* out = A^H v (conjugate transpose) */
static void cmat_h_vec(int M, int N, const cplx *A, const cplx *v, cplx *out) {
  for (int n = 0; n < N; ++n) {
    cplx s = 0.0;
    for (int m = 0; m < M; ++m) s += conj(A[(size_t)m * N + n]) * v[m];
    out[n] = s;
  }
}

/* complex soft threshold: a scaled by max(|a| - t, 0) / |a| (0 at a = 0) */
static cplx csoft(cplx a, double t) {
  const double mag = cabs(a);
  if (!(mag > t)) return 0.0;
  return a * ((mag - t) / mag);
}

/* r = y - A x, returns ||r - r_prev|| and moves r into r_prev */
static double cresidual_delta(int M, int N, const cplx *A, const cplx *y, const cplx *x, cplx *r,
                              cplx *r_prev) {
  cmat_vec(M, N, A, x, r);
  double d = 0.0;
  for (int m = 0; m < M; ++m) {
    r[m] = y[m] - r[m];
    const cplx e = r[m] - r_prev[m];
    d += creal(e) * creal(e) + cimag(e) * cimag(e);
    r_prev[m] = r[m];
  }
  return sqrt(d);
}

/* FISTA (Algorithm 1) on complex data: the steps of or_fista with A^H and csoft. */
int or_cfista(int M, int N, const cplx *A, int64_t P, const cplx *Y, cplx *X, double L,
              double lambda, double eps, int max_iters, int32_t *iters_out, int n_threads) {
  if (M <= 0 || N <= 0 || P < 0 || !(L > 0.0) || lambda < 0.0 || max_iters < 0)
    return OR_ERR_ARG;
  set_threads(n_threads);
#pragma omp parallel
  {
    cplx *buf = (cplx *)malloc(sizeof(cplx) * (5 * N + 3 * M));
    cplx *x = buf, *x_prev = x + N, *z = x_prev + N, *aux = z + N, *g = aux + N;
    cplx *v = g + N, *r = v + M, *r_prev = r + M;
#pragma omp for schedule(dynamic, 16)
    for (int64_t p = 0; p < P; ++p) {
      const cplx *y = Y + p * M;
      for (int n = 0; n < N; ++n) x[n] = z[n] = 0.0;
      memcpy(r_prev, y, sizeof(cplx) * M);
      double t = 1.0, delta = 1.0;
      int it = 0;
      while (delta >= eps && it < max_iters) {
        /* 1. aux = z - (1/L) A^H (A z - y) */
        cmat_vec(M, N, A, z, v);
        for (int m = 0; m < M; ++m) v[m] -= y[m];
        cmat_h_vec(M, N, A, v, g);
        for (int n = 0; n < N; ++n) aux[n] = z[n] - (g[n] / L);
        /* 2. x = modulus soft threshold of aux at lambda / L */
        memcpy(x_prev, x, sizeof(cplx) * N);
        const double thr = lambda / L;
        for (int n = 0; n < N; ++n) x[n] = csoft(aux[n], thr);
        /* 3-4. momentum */
        const double tn = (1.0 + sqrt(4.0 * t * t + 1.0)) / 2.0;
        for (int n = 0; n < N; ++n) z[n] = x[n] + ((t - 1.0) / tn) * (x[n] - x_prev[n]);
        t = tn;
        /* 5. r = y - A x, Delta */
        delta = cresidual_delta(M, N, A, y, x, r, r_prev);
        ++it;
      }
      memcpy(X + p * N, x, sizeof(cplx) * N);
      if (iters_out) iters_out[p] = it;
    }
    free(buf);
  }
  return OR_OK;
}

/* s = B^+ y for B = A(:, c) of full column rank (nc <= M), by complex Householder QR:
 * column j is reflected onto alpha e_j with alpha = -e^{i arg(x_0)} ||x||.  Returns 1 if
 * a column is (numerically) dependent on the earlier ones. */
static int cqr_lstsq(int M, int N, const cplx *A, const int *c, int nc, const cplx *y, cplx *s,
                     cplx *work) {
  if (nc > M) return 1;
  cplx *B = work, *b = B + (size_t)M * nc, *v = b + M;
  for (int m = 0; m < M; ++m) {
    for (int j = 0; j < nc; ++j) B[(size_t)m * nc + j] = A[(size_t)m * N + c[j]];
    b[m] = y[m];
  }
  double scale = 0.0;
  for (int m = 0; m < M; ++m)
    for (int j = 0; j < nc; ++j) scale = fmax(scale, cabs(B[(size_t)m * nc + j]));
  for (int j = 0; j < nc; ++j) {
    double nrm2 = 0.0;
    for (int m = j; m < M; ++m) nrm2 += creal(B[(size_t)m * nc + j] * conj(B[(size_t)m * nc + j]));
    const double nrm = sqrt(nrm2);
    if (!(nrm > 1e-13 * scale * sqrt((double)M))) return 1;
    const cplx x0 = B[(size_t)j * nc + j];
    const cplx phase = cabs(x0) > 0.0 ? x0 / cabs(x0) : 1.0;
    const cplx alpha = -phase * nrm;
    double vn2 = 0.0;
    for (int m = j; m < M; ++m) {
      v[m] = B[(size_t)m * nc + j] - (m == j ? alpha : 0.0);
      vn2 += creal(v[m] * conj(v[m]));
    }
    /* H = I - 2 v v^H / (v^H v) applied to the remaining columns and to b */
    for (int k = j; k < nc; ++k) {
      cplx d = 0.0;
      for (int m = j; m < M; ++m) d += conj(v[m]) * B[(size_t)m * nc + k];
      d = 2.0 * d / vn2;
      for (int m = j; m < M; ++m) B[(size_t)m * nc + k] -= d * v[m];
    }
    cplx d = 0.0;
    for (int m = j; m < M; ++m) d += conj(v[m]) * b[m];
    d = 2.0 * d / vn2;
    for (int m = j; m < M; ++m) b[m] -= d * v[m];
  }
  /* R s = (Q^H y)[0..nc) */
  for (int j = nc - 1; j >= 0; --j) {
    cplx acc = b[j];
    for (int k = j + 1; k < nc; ++k) acc -= B[(size_t)j * nc + k] * s[k];
    s[j] = acc / B[(size_t)j * nc + j];
  }
  return 0;
}

typedef struct {
  cplx *x, *p, *s, *r, *r_prev, *lsw;
  double *mag;
  int *c, *theta, *q, *cand;
  unsigned char *taken, *in_c;
} cgreedy_ws;

static int cws_alloc(cgreedy_ws *w, int M, int N) {
  const size_t lsw = (size_t)M * N + 2 * (size_t)M + 16;
  w->x = (cplx *)malloc(sizeof(cplx) * (3 * (size_t)N + 2 * (size_t)M + lsw));
  w->mag = (double *)malloc(sizeof(double) * N);
  w->c = (int *)malloc(sizeof(int) * 4 * N);
  w->taken = (unsigned char *)malloc(2 * N);
  if (!w->x || !w->mag || !w->c || !w->taken) return 1;
  w->p = w->x + N;
  w->s = w->p + N;
  w->r = w->s + N;
  w->r_prev = w->r + M;
  w->lsw = w->r_prev + M;
  w->theta = w->c + N;
  w->q = w->theta + N;
  w->cand = w->q + N;
  w->in_c = w->taken + N;
  return 0;
}

static void cws_free(cgreedy_ws *w) {
  free(w->x);
  free(w->mag);
  free(w->c);
  free(w->taken);
}

/* gOMP (Algorithm 3) on complex data: Theta = the G largest |A^H r|, c = Theta U c,
 * s = B^+ y, q = the kappa largest |s| over c, refit on q, r = y - A x, Delta (R4, R5). */
int or_cgomp(int M, int N, const cplx *A, int64_t P, const cplx *Y, cplx *X, int kappa, int G,
             double eps, int max_iters, int32_t *iters_out, int n_threads) {
  if (M <= 0 || N <= 0 || P < 0 || kappa < 0 || kappa > N || G < 1 || G > N || max_iters < 0)
    return OR_ERR_ARG;
  int cap = max_iters;
  if (kappa < cap) cap = kappa;
  if (cap > M / G) cap = M / G;
  int fail = 0;
  set_threads(n_threads);
#pragma omp parallel reduction(| : fail)
  {
    cgreedy_ws cw;
    int bad = cws_alloc(&cw, M, N);
    fail |= bad;
#pragma omp for schedule(dynamic, 4)
    for (int64_t p = 0; p < P; ++p) {
      if (bad) continue;
      const cplx *y = Y + p * M;
      for (int n = 0; n < N; ++n) cw.x[n] = 0.0;
      memcpy(cw.r_prev, y, sizeof(cplx) * M);
      int nc = 0;
      for (int n = 0; n < N; ++n) cw.cand[n] = n;
      double delta = 1.0;
      int it = 0;
      while (delta >= eps && it < cap) {
        cmat_h_vec(M, N, A, cw.r_prev, cw.p);
        for (int n = 0; n < N; ++n) cw.mag[n] = cabs(cw.p[n]);
        argmax_k(cw.mag, cw.cand, N, G, cw.theta, cw.taken);
        nc = support_union(N, cw.c, nc, cw.theta, G, cw.in_c);
        fail |= cqr_lstsq(M, N, A, cw.c, nc, y, cw.s, cw.lsw);
        for (int n = 0; n < N; ++n) cw.mag[n] = 0.0;
        for (int j = 0; j < nc; ++j) cw.mag[cw.c[j]] = cabs(cw.s[j]);
        const int nq = nc < kappa ? nc : kappa;
        if (nc > kappa) argmax_k(cw.mag, cw.c, nc, kappa, cw.q, cw.taken);
        else
          for (int j = 0; j < nc; ++j) cw.q[j] = cw.c[j];
        fail |= cqr_lstsq(M, N, A, cw.q, nq, y, cw.s, cw.lsw);
        for (int n = 0; n < N; ++n) cw.x[n] = 0.0;
        for (int j = 0; j < nq; ++j) cw.x[cw.q[j]] = cw.s[j];
        delta = cresidual_delta(M, N, A, y, cw.x, cw.r, cw.r_prev);
        ++it;
      }
      memcpy(X + p * N, cw.x, sizeof(cplx) * N);
      if (iters_out) iters_out[p] = it;
    }
    if (!bad) cws_free(&cw);
  }
  return fail ? OR_ERR_ARG : OR_OK;
}

/* CoSaMP (Algorithm 5) on complex data: Theta = the 2 kappa largest |A^H r|, c = Theta U c,
 * s = B^+ y, keep the kappa largest |s| (c = c(q), x(c) = s(q)), r = y - A x, Delta. */
int or_ccosamp(int M, int N, const cplx *A, int64_t P, const cplx *Y, cplx *X, int kappa,
               double eps, int max_iters, int32_t *iters_out, int n_threads) {
  if (M <= 0 || N <= 0 || P < 0 || kappa < 0 || 2 * kappa > N || max_iters < 0)
    return OR_ERR_ARG;
  int fail = 0;
  set_threads(n_threads);
#pragma omp parallel reduction(| : fail)
  {
    cgreedy_ws cw;
    int bad = cws_alloc(&cw, M, N);
    fail |= bad;
#pragma omp for schedule(dynamic, 4)
    for (int64_t p = 0; p < P; ++p) {
      if (bad) continue;
      const cplx *y = Y + p * M;
      for (int n = 0; n < N; ++n) cw.x[n] = 0.0;
      memcpy(cw.r_prev, y, sizeof(cplx) * M);
      int nc = 0;
      for (int n = 0; n < N; ++n) cw.cand[n] = n;
      double delta = 1.0;
      int it = 0;
      while (delta >= eps && it < max_iters) {
        cmat_h_vec(M, N, A, cw.r_prev, cw.p);
        for (int n = 0; n < N; ++n) cw.mag[n] = cabs(cw.p[n]);
        argmax_k(cw.mag, cw.cand, N, 2 * kappa, cw.theta, cw.taken);
        nc = support_union(N, cw.c, nc, cw.theta, 2 * kappa, cw.in_c);
        fail |= cqr_lstsq(M, N, A, cw.c, nc, y, cw.s, cw.lsw);
        for (int n = 0; n < N; ++n) cw.mag[n] = 0.0;
        for (int j = 0; j < nc; ++j) cw.mag[cw.c[j]] = cabs(cw.s[j]);
        const int nq = nc < kappa ? nc : kappa;
        if (nc > kappa) argmax_k(cw.mag, cw.c, nc, kappa, cw.q, cw.taken);
        else
          for (int j = 0; j < nc; ++j) cw.q[j] = cw.c[j];
        /* x(q) = s(q), c = q (s is indexed by position in c) */
        for (int n = 0; n < N; ++n) cw.x[n] = 0.0;
        for (int j = 0; j < nc; ++j) cw.p[cw.c[j]] = cw.s[j];
        for (int j = 0; j < nq; ++j) cw.x[cw.q[j]] = cw.p[cw.q[j]];
        for (int j = 0; j < nq; ++j) cw.c[j] = cw.q[j];
        nc = nq;
        delta = cresidual_delta(M, N, A, y, cw.x, cw.r, cw.r_prev);
        ++it;
      }
      memcpy(X + p * N, cw.x, sizeof(cplx) * N);
      if (iters_out) iters_out[p] = it;
    }
    if (!bad) cws_free(&cw);
  }
  return fail ? OR_ERR_ARG : OR_OK;
}

/* In-place Hermitian Cholesky K = L L^H (lower, n x n).  Returns nonzero if K is not
 * (numerically) positive definite. */
static int ccholesky(int n, cplx *K) {
  for (int j = 0; j < n; ++j) {
    double dj = creal(K[(size_t)j * n + j]);
    for (int k = 0; k < j; ++k) {
      const cplx l = K[(size_t)j * n + k];
      dj -= creal(l) * creal(l) + cimag(l) * cimag(l);
    }
    if (!(dj > 0.0)) return 1;
    dj = sqrt(dj);
    K[(size_t)j * n + j] = dj;
    for (int i = j + 1; i < n; ++i) {
      cplx acc = K[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) acc -= K[(size_t)i * n + k] * conj(K[(size_t)j * n + k]);
      K[(size_t)i * n + j] = acc / dj;
    }
  }
  return 0;
}

/* Solve L L^H v = b in place. */
static void ccholesky_solve(int n, const cplx *Lf, cplx *b) {
  for (int i = 0; i < n; ++i) {
    cplx acc = b[i];
    for (int k = 0; k < i; ++k) acc -= Lf[(size_t)i * n + k] * b[k];
    b[i] = acc / Lf[(size_t)i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    cplx acc = b[i];
    for (int k = i + 1; k < n; ++k) acc -= conj(Lf[(size_t)k * n + i]) * b[k];
    b[i] = acc / Lf[(size_t)i * n + i];
  }
}

/* ADMM (Algorithm 2, reading R1) on complex data: x = (A^H A + alpha I)^{-1}
 * (A^H y + alpha (z - w)), z = modulus-soft(x + w, lambda / alpha), w += x - z. */
int or_cadmm(int M, int N, const cplx *A, int64_t P, const cplx *Y, cplx *X, double alpha,
             double lambda, double eps, int max_iters, int32_t *iters_out, int n_threads) {
  if (M <= 0 || N <= 0 || P < 0 || !(alpha > 0.0) || lambda < 0.0 || max_iters < 0)
    return OR_ERR_ARG;
  cplx *Kc = (cplx *)malloc(sizeof(cplx) * N * N);
  if (!Kc) return OR_ERR_NOMEM;
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) {
      cplx g = 0.0;
      for (int m = 0; m < M; ++m) g += conj(A[(size_t)m * N + i]) * A[(size_t)m * N + j];
      if (i == j) g += alpha;
      Kc[(size_t)i * N + j] = g;
    }
  if (ccholesky(N, Kc)) {
    free(Kc);
    return OR_ERR_ARG;
  }
  const double zthr = lambda / alpha;
  set_threads(n_threads);
#pragma omp parallel
  {
    cplx *buf = (cplx *)malloc(sizeof(cplx) * (5 * N + 2 * M));
    cplx *x = buf, *z = x + N, *wv = z + N, *ahy = wv + N, *rhs = ahy + N;
    cplx *r = rhs + N, *r_prev = r + M;
#pragma omp for schedule(dynamic, 16)
    for (int64_t p = 0; p < P; ++p) {
      const cplx *y = Y + p * M;
      for (int n = 0; n < N; ++n) x[n] = z[n] = wv[n] = 0.0;
      memcpy(r_prev, y, sizeof(cplx) * M);
      cmat_h_vec(M, N, A, y, ahy);
      double delta = 1.0;
      int it = 0;
      while (delta >= eps && it < max_iters) {
        for (int n = 0; n < N; ++n) rhs[n] = ahy[n] + alpha * (z[n] - wv[n]);
        ccholesky_solve(N, Kc, rhs);
        memcpy(x, rhs, sizeof(cplx) * N);
        for (int n = 0; n < N; ++n) z[n] = csoft(x[n] + wv[n], zthr);
        for (int n = 0; n < N; ++n) wv[n] += x[n] - z[n];
        delta = cresidual_delta(M, N, A, y, x, r, r_prev);
        ++it;
      }
      memcpy(X + p * N, x, sizeof(cplx) * N);
      if (iters_out) iters_out[p] = it;
    }
    free(buf);
  }
  free(Kc);
  return OR_OK;
}

/* BIHT (Algorithm 4, backtracking IHT) on complex data: u = x_a + mu A^H (y - A x_a),
 * Theta = the kappa largest |u|, c = supp(x_a) U Theta, s = B^+ y, keep the kappa
 * largest |s|, r = y - A x, Delta. */
int or_cbiht(int M, int N, const cplx *A, int64_t P, const cplx *Y, cplx *X, int kappa,
             double mu, double eps, int max_iters, int32_t *iters_out, int n_threads) {
  if (M <= 0 || N <= 0 || P < 0 || kappa < 0 || kappa > N || max_iters < 0) return OR_ERR_ARG;
  int fail = 0;
  set_threads(n_threads);
#pragma omp parallel reduction(| : fail)
  {
    cgreedy_ws cw;
    int bad = cws_alloc(&cw, M, N);
    fail |= bad;
#pragma omp for schedule(dynamic, 4)
    for (int64_t p = 0; p < P; ++p) {
      if (bad) continue;
      const cplx *y = Y + p * M;
      cplx *xa = cw.x;
      for (int n = 0; n < N; ++n) xa[n] = 0.0;
      memcpy(cw.r_prev, y, sizeof(cplx) * M);
      for (int n = 0; n < N; ++n) cw.cand[n] = n;
      double delta = 1.0;
      int it = 0;
      while (delta >= eps && it < max_iters) {
        /* u = x_a + mu A^H (y - A x_a) */
        cmat_vec(M, N, A, xa, cw.r);
        for (int m = 0; m < M; ++m) cw.r[m] = y[m] - cw.r[m];
        cmat_h_vec(M, N, A, cw.r, cw.p);
        for (int n = 0; n < N; ++n) cw.mag[n] = cabs(xa[n] + mu * cw.p[n]);
        argmax_k(cw.mag, cw.cand, N, kappa, cw.theta, cw.taken);
        int nc = 0;
        for (int n = 0; n < N; ++n)
          if (cabs(xa[n]) != 0.0) cw.c[nc++] = n;
        nc = support_union(N, cw.c, nc, cw.theta, kappa, cw.in_c);
        fail |= cqr_lstsq(M, N, A, cw.c, nc, y, cw.s, cw.lsw);
        for (int n = 0; n < N; ++n) cw.mag[n] = 0.0;
        for (int j = 0; j < nc; ++j) cw.mag[cw.c[j]] = cabs(cw.s[j]);
        const int nh = nc < kappa ? nc : kappa;
        if (nc > kappa) argmax_k(cw.mag, cw.c, nc, kappa, cw.q, cw.taken);
        else
          for (int j = 0; j < nc; ++j) cw.q[j] = cw.c[j];
        for (int j = 0; j < nc; ++j) cw.p[cw.c[j]] = cw.s[j];
        for (int n = 0; n < N; ++n) xa[n] = 0.0;
        for (int j = 0; j < nh; ++j) xa[cw.q[j]] = cw.p[cw.q[j]];
        delta = cresidual_delta(M, N, A, y, xa, cw.r, cw.r_prev);
        ++it;
      }
      memcpy(X + p * N, xa, sizeof(cplx) * N);
      if (iters_out) iters_out[p] = it;
    }
    if (!bad) cws_free(&cw);
  }
  return fail ? OR_ERR_ARG : OR_OK;
}

int or_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
