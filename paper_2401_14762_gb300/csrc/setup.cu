// One-off FP64 setup of a context on the device (Section II, Eq. 1 and Section II-A):
// the DCT-II basis, the dictionary A = Phi Psi, its Gram matrix A^T A, the Lipschitz
// constant L = lambda_max(A^T A) and the ADMM factor (A A^T + rho I)^{-1}.
// These kernels run once per context on at most 256 x 256 matrices, so they are plain
// one-thread-per-output or single-CTA kernels; none of them is on the per-pixel path.
#include <cuda_runtime.h>

#include "cs_internal.cuh"

namespace cs {
namespace {

// Psi[n][k] = a_k cos(pi (2n+1) k / 2N): column k is the k-th orthonormal DCT-II atom,
// so f = Psi x synthesises a spectrum from its DCT coefficients.
__global__ void k_dct_psi(int N, double* Psi) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N * N) return;
  int n = i / N, k = i % N;
  double a = (k == 0) ? sqrt(1.0 / N) : sqrt(2.0 / N);
  Psi[i] = a * cospi((2.0 * n + 1.0) * k / (2.0 * N));
}

// C[i][j] = sum_k A(i,k) B(k,j) with A(i,k) = A[i*ar + k*ac], B(k,j) = B[k*br + j*bc].
__global__ void k_gemm_f64(int m, int n, int kdim, const double* A, int ar, int ac,
                           const double* B, int br, int bc, double* C) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m * n) return;
  int r = i / n, col = i % n;
  double s = 0.0;
  for (int k = 0; k < kdim; ++k) s += A[r * ar + k * ac] * B[k * br + col * bc];
  C[i] = s;
}

__global__ void k_cast_f32(int n, const double* src, float* dst) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = (float)src[i];
}

__global__ void k_transpose_f64(int rows, int cols, const double* src, double* dst) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * cols) return;
  int r = i / cols, c = i % cols;
  dst[c * rows + r] = src[i];
}

// ---- block-wide reductions for single-CTA kernels (blockDim = 1024) ----
__device__ double block_max_abs(double v, double* red) {
  v = fabs(v);
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    v = (l < (int)(blockDim.x >> 5)) ? red[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (l == 0) red[32] = v;
  }
  __syncthreads();
  return red[32];
}

__device__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    v = (l < (int)(blockDim.x >> 5)) ? red[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (l == 0) red[32] = v;
  }
  __syncthreads();
  return red[32];
}

// lambda_max of the symmetric positive semi-definite M x M matrix S (= A A^T, whose
// nonzero spectrum equals that of A^T A).  Twelve normalised squarings B <- B^2 / max|B^2|
// turn B into (a multiple of) S^4096, whose columns lie along the top eigenvector for any
// eigen-gap above ~1e-3; the column of largest norm, polished by power steps, gives the
// Rayleigh quotient v^T S v / v^T v.  One CTA of 1024 threads; B0, B1 are M*M scratch.
__global__ void __launch_bounds__(1024) k_lambda_max(int M, const double* S, double* B0,
                                                     double* B1, double* v, double* out) {
  __shared__ double red[33];
  const int tid = threadIdx.x, nt = blockDim.x;
  double mx = 0.0;
  for (int i = tid; i < M * M; i += nt) mx = fmax(mx, fabs(S[i]));
  mx = block_max_abs(mx, red);
  if (mx == 0.0) {
    if (tid == 0) *out = 0.0;
    return;
  }
  for (int i = tid; i < M * M; i += nt) B0[i] = S[i] / mx;
  __syncthreads();
  for (int sq = 0; sq < 12; ++sq) {
    double lm = 0.0;
    for (int i = tid; i < M * M; i += nt) {
      int r = i / M, c = i % M;
      double s = 0.0;
      for (int k = 0; k < M; ++k) s += B0[r * M + k] * B0[k * M + c];
      B1[i] = s;
      lm = fmax(lm, fabs(s));
    }
    lm = block_max_abs(lm, red);
    for (int i = tid; i < M * M; i += nt) B0[i] = B1[i] / lm;
    __syncthreads();
  }
  // column of largest norm
  __shared__ double colnorm[kMaxM];
  for (int c = tid; c < M; c += nt) {
    double s = 0.0;
    for (int r = 0; r < M; ++r) s += B0[r * M + c] * B0[r * M + c];
    colnorm[c] = s;
  }
  __syncthreads();
  __shared__ int best;
  if (tid == 0) {
    int b = 0;
    for (int c = 1; c < M; ++c)
      if (colnorm[c] > colnorm[b]) b = c;
    best = b;
  }
  __syncthreads();
  for (int r = tid; r < M; r += nt) v[r] = B0[r * M + best];
  __syncthreads();
  double lam = 0.0;
  for (int it = 0; it < 32; ++it) {
    double nv = 0.0;
    for (int r = tid; r < M; r += nt) nv += v[r] * v[r];
    nv = block_sum(nv, red);
    double sv = 0.0;  // v^T S v and w = S v
    for (int r = tid; r < M; r += nt) {
      double s = 0.0;
      for (int k = 0; k < M; ++k) s += S[r * M + k] * v[k];
      B1[r] = s;
      sv += v[r] * s;
    }
    sv = block_sum(sv, red);
    lam = sv / nv;
    double nw = 0.0;
    for (int r = tid; r < M; r += nt) nw += B1[r] * B1[r];
    nw = block_sum(nw, red);
    double inv = 1.0 / sqrt(nw);
    for (int r = tid; r < M; r += nt) v[r] = B1[r] * inv;
    __syncthreads();
  }
  if (tid == 0) *out = lam;
}

// W = K^{-1} for the symmetric positive definite n x n matrix K (n <= 128), via the
// Cholesky factor K = L L^T computed in place in `work`.  One CTA of 1024 threads.
__global__ void __launch_bounds__(1024) k_spd_inverse(int n, const double* K, double* work,
                                                      float* W, double* W64, int* status) {
  const int tid = threadIdx.x, nt = blockDim.x;
  __shared__ int bad;
  if (tid == 0) bad = 0;
  for (int i = tid; i < n * n; i += nt) work[i] = K[i];
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    if (tid == 0) {
      double d = work[j * n + j];
      if (!(d > 0.0)) bad = 1;
      work[j * n + j] = sqrt(fmax(d, 1e-300));
    }
    __syncthreads();
    double d = work[j * n + j];
    for (int i = j + 1 + tid; i < n; i += nt) work[i * n + j] /= d;
    __syncthreads();
    int rem = n - j - 1;
    for (int e = tid; e < rem * rem; e += nt) {
      int i = j + 1 + e / rem, k = j + 1 + e % rem;
      if (k <= i) work[i * n + k] -= work[i * n + j] * work[k * n + j];
    }
    __syncthreads();
  }
  if (bad) {
    if (tid == 0) atomicOr(status, kStNotSpd);
    return;
  }
  // column c of K^{-1}: solve L y = e_c, then L^T w = y (thread c owns column c)
  for (int c = tid; c < n; c += nt) {
    double y[kMaxM];
    for (int i = 0; i < n; ++i) {
      double s = (i == c) ? 1.0 : 0.0;
      for (int k = 0; k < i; ++k) s -= work[i * n + k] * y[k];
      y[i] = s / work[i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
      double s = y[i];
      for (int k = i + 1; k < n; ++k) s -= work[k * n + i] * y[k];
      y[i] = s / work[i * n + i];
    }
    for (int i = 0; i < n; ++i) {
      W[i * n + c] = (float)y[i];
      W64[i * n + c] = y[i];
    }
  }
}

// dst (rows x ld) = src (rows x cols) with each row zero padded to ld columns.
__global__ void k_pad_rows(int rows, int cols, int ld, const float* src, float* dst) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < rows * ld) {
    int r = i / ld, c = i - r * ld;
    dst[i] = c < cols ? src[r * cols + c] : 0.f;
  }
}

// dst (rows x ld, FP32) = src (rows x cols, FP64) rounded, each row zero padded to ld
__global__ void k_cast_pad_f32(int rows, int cols, int ld, const double* src, float* dst) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < rows * ld) {
    int r = i / ld, c = i - r * ld;
    dst[i] = c < cols ? (float)src[(size_t)r * cols + c] : 0.f;
  }
}

// cn[i] = ||Psi(:, i)||_2 in FP64, rounded up to FP32 (an upper bound for error bounds)
__global__ void k_col_norms(int N, const double* Psi, float* cn) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) {
    double s = 0.0;
    for (int n = 0; n < N; ++n) s += Psi[(size_t)n * N + i] * Psi[(size_t)n * N + i];
    cn[i] = __double2float_ru(sqrt(s) * (1.0 + 1e-12));
  }
}

__global__ void k_add_diag(int n, double* K, double v) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) K[i * n + i] += v;
}

inline int nblk(int n, int t) { return (n + t - 1) / t; }

}  // namespace

cudaError_t setup_dictionary(Ctx& c, const double* A_host, const double* Phi_host,
                             const double* Psi_host) {
  const int M = c.M, N = c.N;
  cudaStream_t s = c.stream;
  cudaError_t e;
  // scratch: Phi, Psi, A A^T, two M*M buffers, a vector, the result
  double* sc = c.scratch64;
  double *Phi = sc, *Psi = Phi + M * N, *S = Psi + N * N, *B0 = S + M * M, *B1 = B0 + M * M;
  double *v = B1 + M * M, *lam = v + kMaxM;
  if (A_host) {
    e = cudaMemcpyAsync(c.A64, A_host, sizeof(double) * M * N, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
  } else {
    e = cudaMemcpyAsync(Phi, Phi_host, sizeof(double) * M * N, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    if (Psi_host) {
      e = cudaMemcpyAsync(Psi, Psi_host, sizeof(double) * N * N, cudaMemcpyHostToDevice, s);
      if (e != cudaSuccess) return e;
    } else {
      k_dct_psi<<<nblk(N * N, 256), 256, 0, s>>>(N, Psi);
    }
    k_gemm_f64<<<nblk(M * N, 256), 256, 0, s>>>(M, N, N, Phi, N, 1, Psi, N, 1, c.A64);
    if (c.Psi64) {  // kept for the sparsification pre-processing
      e = cudaMemcpyAsync(c.Psi64, Psi, sizeof(double) * N * N, cudaMemcpyDeviceToDevice, s);
      if (e != cudaSuccess) return e;
      const int ldp = 128 * ((N + 127) / 128);
      k_cast_pad_f32<<<nblk(N * ldp, 256), 256, 0, s>>>(N, N, ldp, Psi, c.Psi32);
      k_col_norms<<<nblk(N, 256), 256, 0, s>>>(N, Psi, c.psi_cn);
    }
  }
  k_transpose_f64<<<nblk(M * N, 256), 256, 0, s>>>(M, N, c.A64, c.At64);
  // Gram A^T A (N x N): (A^T)(i,k) = A[k*N + i]
  k_gemm_f64<<<nblk(N * N, 256), 256, 0, s>>>(N, N, M, c.A64, 1, N, c.A64, N, 1, c.G64);
  // A A^T (M x M)
  k_gemm_f64<<<nblk(M * M, 256), 256, 0, s>>>(M, M, N, c.A64, N, 1, c.A64, 1, N, S);
  k_cast_f32<<<nblk(M * N, 256), 256, 0, s>>>(M * N, c.A64, c.A32);
  k_cast_f32<<<nblk(M * N, 256), 256, 0, s>>>(M * N, c.At64, c.At32);
  k_cast_f32<<<nblk(N * N, 256), 256, 0, s>>>(N * N, c.G64, c.G32);
  k_lambda_max<<<1, 1024, 0, s>>>(M, S, B0, B1, v, lam);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(&c.L, lam, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(s);
}

cudaError_t setup_admm_factor(Ctx& c, double rho) {
  const int M = c.M, N = c.N;
  cudaStream_t s = c.stream;
  double* sc = c.scratch64;
  double *K = sc + M * N + N * N, *work = K + M * M;
  k_gemm_f64<<<nblk(M * M, 256), 256, 0, s>>>(M, M, N, c.A64, N, 1, c.A64, 1, N, K);
  k_add_diag<<<nblk(M, 256), 256, 0, s>>>(M, K, rho);
  k_spd_inverse<<<1, 1024, 0, s>>>(M, K, work, c.W32, c.W64, c.status);
  const int ldw = smem_ld(M);
  k_pad_rows<<<nblk(M * ldw, 256), 256, 0, s>>>(M, M, ldw, c.W32, c.Wpad);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  c.rho = rho;
  return cudaSuccess;
}

}  // namespace cs
