// FP32 SIMT path: measurement (Eq. 1), FISTA (Algorithm 1) and ADMM (Algorithm 2).
//
// One CTA of 256 threads owns a tile of 32 pixels for the whole solve; the dictionary A
// (M x N, FP32, rows padded) sits in shared memory and every pixel's iterate lives in
// registers, so the only HBM traffic is Y in and X out.  Warp w owns pixels 4w..4w+3.
//   * "column" mapping: lane l owns columns 4l..4l+3 (and 128+4l..128+4l+3 if N > 128)
//     of the N-long vectors of its 4 pixels -- the A^T r products and the proximal step.
//   * "row" mapping: lane l owns rows l, l+32, ... (< M) of the M-long vectors of its 4
//     pixels -- the A x products, the residual and Delta.
// Each product is a register-blocked outer-product loop over shared memory: per step a
// lane reads one float4 of A per chunk and one broadcast float4 of the 4 pixels' operand.
//
// FISTA keeps u = A x so that A z = u + beta (u - u_prev) needs no extra product and
// Delta = ||r^i - r^{i-1}|| = ||u^i - u^{i-1}|| comes for free: 4MN flops per iteration.
// ADMM uses the Woodbury form of its x-step,
//   (A^T A + rho I)^{-1} v = (v - A^T W A v) / rho,  W = (A A^T + rho I)^{-1},
// which with d = z - w and h = W (y - A d) gives x = d + A^T h and A x = y - rho h, so
// r^i = rho h^i: 4MN + 2M^2 flops per iteration, Delta again for free.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <mutex>

#include "cs_internal.cuh"
#include "tc_ptx.cuh"

namespace cs {
namespace {

constexpr int kThreads = 256;
constexpr int kPPW = 4;   // pixels per warp
constexpr int kT = 32;    // pixels per CTA
constexpr int kLdv = 36;  // row stride of the M x T residual buffer (conflict-free float4)

struct CvParams {
  int M, N, Npad, lda, ldw, Mpad;
  const float* A;  // M x N global
  const float* W;  // M x M global (ADMM)
  const float* Wg; // the same with rows padded to ldw, read from global memory when the
                   // kernel's shared-memory layout has no room for W (else null)
  const float* Y;
  float* X;
  const float* E;  // measurement noise (measure only)
  float* Yout;     // measurement output (measure only)
  int64_t P;
  float c1, c2;    // FISTA: 1/L, lambda/L.  ADMM: rho, lambda/rho
  float eps2;      // eps^2 (0 => fixed iteration count)
  int start_done;  // eps > 1: Delta = 1 < eps before the first iteration
  int pairs;       // complex data as (re, im) pairs: thresholds on the moduli
  int iters;
  int32_t* iters_out;
  uint8_t* conv_out;
  int* status;
  const float* beta;  // FISTA momentum weights beta_i, i = 1..iters
};

__device__ __forceinline__ float soft_thr(float a, float t) {
  float m = fabsf(a) - t;
  return m > 0.f ? copysignf(m, a) : 0.f;
}

// The modulus soft threshold of the complex value a0 + i a1: scaled by
// max(|a| - t, 0) / |a| (0 when |a| <= t).
__device__ __forceinline__ void soft_pair(float a0, float a1, float t, float& x0, float& x1) {
  const float m = sqrtf(fmaf(a0, a0, a1 * a1));
  const float s = m > t ? (m - t) / m : 0.f;
  x0 = a0 * s;
  x1 = a1 * s;
}

__device__ __forceinline__ float f4(const float4& v, int e) {
  return e == 0 ? v.x : (e == 1 ? v.y : (e == 2 ? v.z : v.w));
}

// rows x cols global matrix -> shared, row stride ld, zero padding in [cols, ld)
__device__ void stage_matrix(float* dst, const float* src, int rows, int cols, int ld) {
  for (int i = threadIdx.x; i < rows * ld; i += blockDim.x) {
    int r = i / ld, c = i - r * ld;
    dst[i] = c < cols ? src[r * cols + c] : 0.f;
  }
}

// acc[i][j] += sum_k Ms[row_j][k] * Vs[(pix_i) * ldv_ + k]  (row mapping product)
template <int MR>
__device__ __forceinline__ void rows_product(float (&acc)[kPPW][MR], const float* Ms, int ldm,
                                             const float* Vs, int ldv_, int kpad, int warp,
                                             const int (&row)[MR], const bool (&hr)[MR]) {
#pragma unroll
  for (int i = 0; i < kPPW; ++i)
#pragma unroll
    for (int j = 0; j < MR; ++j) acc[i][j] = 0.f;
  const float* vb = Vs + (warp * kPPW) * ldv_;
#pragma unroll 2
  for (int k = 0; k < kpad; k += 4) {
    float4 xv[kPPW];
#pragma unroll
    for (int i = 0; i < kPPW; ++i) xv[i] = *reinterpret_cast<const float4*>(vb + i * ldv_ + k);
#pragma unroll
    for (int j = 0; j < MR; ++j) {
      if (!hr[j]) continue;
      float4 a = *reinterpret_cast<const float4*>(Ms + row[j] * ldm + k);
#pragma unroll
      for (int i = 0; i < kPPW; ++i)
        acc[i][j] += xv[i].x * a.x + xv[i].y * a.y + xv[i].z * a.z + xv[i].w * a.w;
    }
  }
}

// acc[i][4c+e] = sum_m vs[m][pix_i] * As[m][col_c + e]  (column mapping product, A^T v)
template <int NCH>
__device__ __forceinline__ void cols_product(float (&acc)[kPPW][4 * NCH], const float* As,
                                             int lda, const float* vs, int M, int warp,
                                             const int (&col)[NCH], const bool (&hc)[NCH]) {
#pragma unroll
  for (int i = 0; i < kPPW; ++i)
#pragma unroll
    for (int k = 0; k < 4 * NCH; ++k) acc[i][k] = 0.f;
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 2
  for (int m = 0; m < M; ++m) {
    float4 v = *reinterpret_cast<const float4*>(vs + m * kLdv + warp * kPPW);
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
      float4 a = hc[c] ? *reinterpret_cast<const float4*>(As + m * lda + col[c]) : zero;
#pragma unroll
      for (int i = 0; i < kPPW; ++i) {
        float vi = f4(v, i);
        acc[i][4 * c + 0] += vi * a.x;
        acc[i][4 * c + 1] += vi * a.y;
        acc[i][4 * c + 2] += vi * a.z;
        acc[i][4 * c + 3] += vi * a.w;
      }
    }
  }
}

template <int NCH>
__device__ __forceinline__ void write_x(float* X, int64_t pix, int N, const float (&x)[4 * NCH],
                                        const int (&col)[NCH]) {
#pragma unroll
  for (int c = 0; c < NCH; ++c)
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if (col[c] + e < N) X[pix * N + col[c] + e] = x[4 * c + e];
}

// ---------------------------------------------------------------------------------
// Algorithm 1 (FISTA)
// ---------------------------------------------------------------------------------
template <int MR, int NCH>
__global__ void __launch_bounds__(kThreads, 1) k_fista_f32(CvParams p) {
  extern __shared__ __align__(16) float sm[];
  const int M = p.M, lda = p.lda;
  float* As = sm;
  float* xs = As + M * lda;
  float* vs = xs + kT * lda;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t pix0 = (int64_t)blockIdx.x * kT + warp * kPPW;

  stage_matrix(As, p.A, M, p.N, lda);
  for (int i = tid; i < kT * lda; i += kThreads) xs[i] = 0.f;

  int col[NCH], row[MR];
  bool hc[NCH], hr[MR];
#pragma unroll
  for (int c = 0; c < NCH; ++c) {
    col[c] = 128 * c + 4 * lane;
    hc[c] = col[c] < p.Npad;
  }
#pragma unroll
  for (int j = 0; j < MR; ++j) {
    row[j] = lane + 32 * j;
    hr[j] = row[j] < M;
  }
  float yv[kPPW][MR], u[kPPW][MR], up[kPPW][MR];
  float x[kPPW][4 * NCH], z[kPPW][4 * NCH];
  bool done[kPPW];
  bool bad = false;
#pragma unroll
  for (int i = 0; i < kPPW; ++i) {
    bool valid = pix0 + i < p.P;
    done[i] = !valid || p.start_done;
#pragma unroll
    for (int j = 0; j < MR; ++j) {
      float v = (valid && hr[j]) ? p.Y[(pix0 + i) * M + row[j]] : 0.f;
      bad |= !isfinite(v);
      yv[i][j] = v;
      u[i][j] = up[i][j] = 0.f;
    }
#pragma unroll
    for (int k = 0; k < 4 * NCH; ++k) x[i][k] = z[i][k] = 0.f;
  }
  if (bad) atomicOr(p.status, kStNonFinite);
  __syncthreads();

  float beta_prev = 0.f;
  int it = 0;
  // After A is staged the warps never synchronise: a warp owns its pixels in both
  // mappings, so __syncwarp orders every shared-memory hand-off.
  while (it < p.iters) {
    if (done[0] && done[1] && done[2] && done[3]) break;  // warp-uniform
    // residual of the extrapolated point: A z - y = u + beta (u - u_prev) - y
#pragma unroll
    for (int j = 0; j < MR; ++j) {
      if (!hr[j]) continue;
      float4 v;
      v.x = u[0][j] + beta_prev * (u[0][j] - up[0][j]) - yv[0][j];
      v.y = u[1][j] + beta_prev * (u[1][j] - up[1][j]) - yv[1][j];
      v.z = u[2][j] + beta_prev * (u[2][j] - up[2][j]) - yv[2][j];
      v.w = u[3][j] + beta_prev * (u[3][j] - up[3][j]) - yv[3][j];
      *reinterpret_cast<float4*>(vs + row[j] * kLdv + warp * kPPW) = v;
    }
    __syncwarp();
    // steps 1-4: aux = z - A^T(Az - y)/L, x = soft(aux, lambda/L), t, z
    float acc[kPPW][4 * NCH];
    cols_product<NCH>(acc, As, lda, vs, M, warp, col, hc);
    const float beta = p.beta[it];  // beta_{it+1}
#pragma unroll
    for (int i = 0; i < kPPW; ++i) {
      if (done[i]) continue;
      if (p.pairs) {
        // a lane's columns 4l..4l+3 hold two whole (re, im) pairs
#pragma unroll
        for (int k = 0; k < 4 * NCH; k += 2) {
          float x0, x1;
          soft_pair(z[i][k] - acc[i][k] * p.c1, z[i][k + 1] - acc[i][k + 1] * p.c1, p.c2, x0,
                    x1);
          z[i][k] = x0 + beta * (x0 - x[i][k]);
          z[i][k + 1] = x1 + beta * (x1 - x[i][k + 1]);
          x[i][k] = x0;
          x[i][k + 1] = x1;
        }
      } else {
#pragma unroll
        for (int k = 0; k < 4 * NCH; ++k) {
          float xn = soft_thr(z[i][k] - acc[i][k] * p.c1, p.c2);
          z[i][k] = xn + beta * (xn - x[i][k]);
          x[i][k] = xn;
        }
      }
#pragma unroll
      for (int c = 0; c < NCH; ++c)
        if (hc[c])
          *reinterpret_cast<float4*>(xs + (warp * kPPW + i) * lda + col[c]) =
              make_float4(x[i][4 * c], x[i][4 * c + 1], x[i][4 * c + 2], x[i][4 * c + 3]);
    }
    __syncwarp();
    // step 5: u = A x, Delta = ||u - u_prev||
    float acc1[kPPW][MR];
    rows_product<MR>(acc1, As, lda, xs, lda, p.Npad, warp, row, hr);
    ++it;
#pragma unroll
    for (int i = 0; i < kPPW; ++i) {
      float d2 = 0.f;
#pragma unroll
      for (int j = 0; j < MR; ++j) {
        float df = hr[j] ? acc1[i][j] - u[i][j] : 0.f;
        d2 += df * df;
        up[i][j] = u[i][j];
        u[i][j] = acc1[i][j];
      }
      d2 = warp_sum(d2);
      if (!done[i] && d2 < p.eps2) {
        done[i] = true;
        write_x<NCH>(p.X, pix0 + i, p.N, x[i], col);
        if (lane == 0) {
          if (p.iters_out) p.iters_out[pix0 + i] = it;
          if (p.conv_out) p.conv_out[pix0 + i] = 1;
        }
      }
    }
    beta_prev = beta;
  }
#pragma unroll
  for (int i = 0; i < kPPW; ++i) {
    if (pix0 + i >= p.P) continue;
    if (!done[i] || p.start_done) {
      write_x<NCH>(p.X, pix0 + i, p.N, x[i], col);
      if (lane == 0) {
        if (p.iters_out) p.iters_out[pix0 + i] = it;
        if (p.conv_out) p.conv_out[pix0 + i] = 0;
      }
    }
  }
}

// ---------------------------------------------------------------------------------
// Algorithm 2 (ADMM), Woodbury form
// ---------------------------------------------------------------------------------
template <int MR, int NCH>
__global__ void __launch_bounds__(kThreads, 1) k_admm_f32(CvParams p) {
  extern __shared__ __align__(16) float sm[];
  const int M = p.M, lda = p.lda, ldw = p.ldw;
  const bool w_smem = p.Wg == nullptr;
  float* As = sm;
  float* Ws = As + M * lda;
  float* xs = w_smem ? Ws + M * ldw : Ws;
  const float* Wr = w_smem ? Ws : p.Wg;
  float* es = xs + kT * lda;
  float* vs = es + kT * ldw;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t pix0 = (int64_t)blockIdx.x * kT + warp * kPPW;
  const float rho = p.c1, thr = p.c2;

  stage_matrix(As, p.A, M, p.N, lda);
  if (w_smem) stage_matrix(Ws, p.W, M, M, ldw);
  for (int i = tid; i < kT * lda; i += kThreads) xs[i] = 0.f;
  for (int i = tid; i < kT * ldw; i += kThreads) es[i] = 0.f;

  int col[NCH], row[MR];
  bool hc[NCH], hr[MR];
#pragma unroll
  for (int c = 0; c < NCH; ++c) {
    col[c] = 128 * c + 4 * lane;
    hc[c] = col[c] < p.Npad;
  }
#pragma unroll
  for (int j = 0; j < MR; ++j) {
    row[j] = lane + 32 * j;
    hr[j] = row[j] < M;
  }
  float yv[kPPW][MR], hp[kPPW][MR];
  float z[kPPW][4 * NCH], w[kPPW][4 * NCH];
  bool done[kPPW];
  bool bad = false;
#pragma unroll
  for (int i = 0; i < kPPW; ++i) {
    bool valid = pix0 + i < p.P;
    done[i] = !valid || p.start_done;
#pragma unroll
    for (int j = 0; j < MR; ++j) {
      float v = (valid && hr[j]) ? p.Y[(pix0 + i) * M + row[j]] : 0.f;
      bad |= !isfinite(v);
      yv[i][j] = v;
      hp[i][j] = v / rho;  // r^0 = y = rho h^0
    }
#pragma unroll
    for (int k = 0; k < 4 * NCH; ++k) z[i][k] = w[i][k] = 0.f;
  }
  if (bad) atomicOr(p.status, kStNonFinite);
  __syncthreads();

  int it = 0;
  while (it < p.iters) {
    if (done[0] && done[1] && done[2] && done[3]) break;  // warp-uniform
    // d = z - w
#pragma unroll
    for (int i = 0; i < kPPW; ++i)
#pragma unroll
      for (int c = 0; c < NCH; ++c)
        if (hc[c])
          *reinterpret_cast<float4*>(xs + (warp * kPPW + i) * lda + col[c]) =
              make_float4(z[i][4 * c] - w[i][4 * c], z[i][4 * c + 1] - w[i][4 * c + 1],
                          z[i][4 * c + 2] - w[i][4 * c + 2], z[i][4 * c + 3] - w[i][4 * c + 3]);
    __syncwarp();
    // e = y - A d
    float acc1[kPPW][MR];
    rows_product<MR>(acc1, As, lda, xs, lda, p.Npad, warp, row, hr);
#pragma unroll
    for (int i = 0; i < kPPW; ++i)
#pragma unroll
      for (int j = 0; j < MR; ++j)
        if (hr[j]) es[(warp * kPPW + i) * ldw + row[j]] = yv[i][j] - acc1[i][j];
    __syncwarp();
    // h = W e ; r = rho h ; Delta = rho ||h - h_prev||
    float h[kPPW][MR];
    rows_product<MR>(h, Wr, ldw, es, ldw, p.Mpad, warp, row, hr);
    ++it;
    bool fin[kPPW], conv[kPPW];
#pragma unroll
    for (int i = 0; i < kPPW; ++i) {
      float d2 = 0.f;
#pragma unroll
      for (int j = 0; j < MR; ++j) {
        float df = hr[j] ? rho * (h[i][j] - hp[i][j]) : 0.f;
        d2 += df * df;
        hp[i][j] = h[i][j];
      }
      d2 = warp_sum(d2);
      conv[i] = d2 < p.eps2;
      fin[i] = !done[i] && (conv[i] || it == p.iters);
    }
#pragma unroll
    for (int j = 0; j < MR; ++j)
      if (hr[j])
        *reinterpret_cast<float4*>(vs + row[j] * kLdv + warp * kPPW) =
            make_float4(h[0][j], h[1][j], h[2][j], h[3][j]);
    __syncwarp();
    // x = d + A^T h ; z = soft(x + w, lambda/rho) ; w = w + x - z
    float acc[kPPW][4 * NCH];
    cols_product<NCH>(acc, As, lda, vs, M, warp, col, hc);
#pragma unroll
    for (int i = 0; i < kPPW; ++i) {
      if (done[i]) continue;
      float x[4 * NCH];
      if (p.pairs) {
#pragma unroll
        for (int k = 0; k < 4 * NCH; k += 2) {
          x[k] = (z[i][k] - w[i][k]) + acc[i][k];
          x[k + 1] = (z[i][k + 1] - w[i][k + 1]) + acc[i][k + 1];
          float z0, z1;
          soft_pair(x[k] + w[i][k], x[k + 1] + w[i][k + 1], thr, z0, z1);
          w[i][k] = w[i][k] + x[k] - z0;
          w[i][k + 1] = w[i][k + 1] + x[k + 1] - z1;
          z[i][k] = z0;
          z[i][k + 1] = z1;
        }
      } else {
#pragma unroll
        for (int k = 0; k < 4 * NCH; ++k) {
          x[k] = (z[i][k] - w[i][k]) + acc[i][k];
          float zn = soft_thr(x[k] + w[i][k], thr);
          w[i][k] = w[i][k] + x[k] - zn;
          z[i][k] = zn;
        }
      }
      if (fin[i]) {
        done[i] = true;
        write_x<NCH>(p.X, pix0 + i, p.N, x, col);
        if (lane == 0) {
          if (p.iters_out) p.iters_out[pix0 + i] = it;
          if (p.conv_out) p.conv_out[pix0 + i] = conv[i] ? 1 : 0;
        }
      }
    }
  }
  // zero iterations (iters == 0 or eps > 1): x = x^0 = 0
#pragma unroll
  for (int i = 0; i < kPPW; ++i) {
    if (pix0 + i >= p.P || it > 0) continue;
    float x[4 * NCH];
#pragma unroll
    for (int k = 0; k < 4 * NCH; ++k) x[k] = 0.f;
    write_x<NCH>(p.X, pix0 + i, p.N, x, col);
    if (lane == 0) {
      if (p.iters_out) p.iters_out[pix0 + i] = 0;
      if (p.conv_out) p.conv_out[pix0 + i] = 0;
    }
  }
}

// ---------------------------------------------------------------------------------
// Eq. 1 measurement: Y = X A^T (+ E), persistent over 32-pixel tiles
// ---------------------------------------------------------------------------------
template <int MR>
__global__ void __launch_bounds__(kThreads, 1) k_measure_f32(CvParams p) {
  extern __shared__ __align__(16) float sm[];
  const int M = p.M, N = p.N, lda = p.lda;
  float* As = sm;
  float* xs = As + M * lda;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  stage_matrix(As, p.A, M, N, lda);
  int row[MR];
  bool hr[MR];
#pragma unroll
  for (int j = 0; j < MR; ++j) {
    row[j] = lane + 32 * j;
    hr[j] = row[j] < M;
  }
  const int64_t ntiles = (p.P + kT - 1) / kT;
  __syncthreads();
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t pix0 = tile * kT + warp * kPPW;
    for (int i = 0; i < kPPW; ++i) {
      bool valid = pix0 + i < p.P;
      for (int n = lane; n < lda; n += 32)
        xs[(warp * kPPW + i) * lda + n] = (valid && n < N) ? p.X[(pix0 + i) * N + n] : 0.f;
    }
    __syncwarp();
    float acc[kPPW][MR];
    rows_product<MR>(acc, As, lda, xs, lda, p.Npad, warp, row, hr);
    __syncwarp();  // xs is rewritten by the next tile
#pragma unroll
    for (int i = 0; i < kPPW; ++i) {
      if (pix0 + i >= p.P) continue;
#pragma unroll
      for (int j = 0; j < MR; ++j) {
        if (!hr[j]) continue;
        int64_t o = (pix0 + i) * M + row[j];
        p.Yout[o] = acc[i][j] + (p.E ? p.E[o] : 0.f);
      }
    }
  }
}

// ---------------------------------------------------------------------------------
// Eq. 1 measurement for N a multiple of 4: Y = X A^T (+ E) as a register-tiled SIMT
// product.  Persistent CTAs of 256 threads walk tiles of 256 pixels; A (rows padded to
// 16 RM with zeros, columns to a multiple of 32) stays in shared memory, and the tile's X
// arrives in boxes of 256 pixels x 32 columns that one thread requests from the tensor
// memory accelerator (TMA: cp.async.bulk.tensor with an mbarrier per stage of a 3-stage
// ring), so the next boxes stream from HBM while the current one is multiplied; rows past
// P and columns past N arrive as zeros.  Thread (tp, tm) of the 16 x 16 grid owns pixels
// 16 tp .. 16 tp + 15 and rows tm + 16 r (r < RM): per float4 step of k it reads 16
// float4 of X and RM of A for 64 RM FMAs, so shared memory (one 8-lane wavefront per
// cycle) keeps up with the FMA pipes.  Each output is summed in the order k = 0, 1, ...
// ---------------------------------------------------------------------------------
struct MtParams {
  int M, N, lda;   // lda: row stride of A in shared memory
  const float* A;  // M x N global
  const float* X;  // P x N (read through the tensor map)
  const float* E;  // P x M or null
  float* Y;        // P x M
  int64_t P;
  int* status;     // the context's status word (a TMA box that never arrived)
};

constexpr int kMtP = 256;            // pixels per tile (TMA box rows)
constexpr int kMtPx = kMtP / 16;     // pixels per thread
constexpr int kMtK = 32;             // columns per chunk (TMA box columns: 128 bytes)
constexpr int kMtStages = 3;
constexpr uint64_t kMtWaitNs = 100ull * 1000 * 1000;  // 100 ms for one box
// bytes of A in shared memory, rounded up so that the X ring starts 1024-byte aligned
__host__ __device__ constexpr int mt_abytes(int rm, int lda) {
  return (4 * 16 * rm * lda + 1023) / 1024 * 1024;
}

template <int RM>
__global__ void __launch_bounds__(256, 1)
    k_measure_tiled(MtParams p, const __grid_constant__ CUtensorMap tmap) {
  extern __shared__ __align__(1024) unsigned char msm[];
  __shared__ __align__(8) uint64_t mbx[kMtStages];
  const int M = p.M, N = p.N, lda = p.lda;
  float* As = reinterpret_cast<float*>(msm);                       // 16 RM x lda
  float* Xs = reinterpret_cast<float*>(msm + mt_abytes(RM, lda));  // stages x kMtP x kMtK
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tm = lane & 15, tp = (lane >> 4) + 2 * warp;
  if (tid == 0)
    for (int s = 0; s < kMtStages; ++s) tc::mbar_init(&mbx[s], 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  for (int i = tid; i < 16 * RM * lda; i += 256) {
    const int r = i / lda, c = i - r * lda;
    As[i] = (r < M && c < N) ? p.A[(size_t)r * N + c] : 0.f;
  }
  __syncthreads();
  const int nch = (N + kMtK - 1) / kMtK;
  const int64_t ntiles = (p.P + kMtP - 1) / kMtP;
  const int64_t my_tiles = ntiles > blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t items = my_tiles * nch;  // (tile, chunk) boxes of this CTA, in order
  // box `it` into stage it % kMtStages, by thread 0; the readers of the stage's previous
  // box have passed a barrier since
  auto issue = [&](int64_t it) {
    if (tid != 0 || it >= items) return;
    const int64_t tile = blockIdx.x + (it / nch) * gridDim.x;
    const int s = (int)(it % kMtStages);
    const uint32_t dst = tc::smem_u32(Xs + (size_t)s * kMtP * kMtK);
    const uint32_t mb = tc::smem_u32(&mbx[s]);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb),
                 "r"(kMtP * kMtK * 4)
                 : "memory");
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(&tmap)), "r"((int)(it % nch) * kMtK),
        "r"((int)(tile * kMtP)), "r"(mb)
        : "memory");
  };
#pragma unroll
  for (int s = 0; s < kMtStages - 1; ++s) issue(s);
  float acc[kMtPx][RM];
#pragma unroll
  for (int i = 0; i < kMtPx; ++i)
#pragma unroll
    for (int r = 0; r < RM; ++r) acc[i][r] = 0.f;
  int64_t it = 0;
  for (; it < items; ++it) {
    const bool got = tc::mbar_wait(&mbx[it % kMtStages], (uint32_t)((it / kMtStages) & 1),
                                   kMtWaitNs);
    // box it is in place (or never came); every thread is done with box it - 1
    if (__syncthreads_or(!got)) break;
    issue(it + kMtStages - 1);
    const float* xb = Xs + (size_t)(it % kMtStages) * kMtP * kMtK + (kMtPx * tp) * kMtK;
    const int ch = (int)(it % nch);
    if (p.E && ch == 0) {
      // the tile's E rows into L2 now, so that the epilogue's loads of them hit L2
      const int64_t tile = blockIdx.x + (it / nch) * gridDim.x;
      const int64_t e1 = (tile + 1) * kMtP < p.P ? (tile + 1) * kMtP * M : p.P * M;
      for (int64_t o = tile * kMtP * M + 32 * (int64_t)tid; o < e1; o += 32 * 256)
        asm volatile("prefetch.global.L2 [%0];\n" ::"l"(p.E + o));
    }
    const float* ab = As + tm * lda + ch * kMtK;
#pragma unroll 1
    for (int k4 = 0; k4 < kMtK / 4; ++k4) {
      float4 xv[kMtPx];
#pragma unroll
      for (int i = 0; i < kMtPx; ++i)
        xv[i] = *reinterpret_cast<const float4*>(xb + i * kMtK + 4 * k4);
#pragma unroll
      for (int r = 0; r < RM; ++r) {
        const float4 a = *reinterpret_cast<const float4*>(ab + 16 * r * lda + 4 * k4);
#pragma unroll
        for (int i = 0; i < kMtPx; ++i) {
          float t = fmaf(xv[i].x, a.x, acc[i][r]);
          t = fmaf(xv[i].y, a.y, t);
          t = fmaf(xv[i].z, a.z, t);
          acc[i][r] = fmaf(xv[i].w, a.w, t);
        }
      }
    }
    if (ch == nch - 1) {  // the tile is complete: add E, store, restart the sums
      const int64_t tile = blockIdx.x + (it / nch) * gridDim.x;
      // E through the read-only path, four pixels' rows loaded before any store: plain
      // loads could alias Y's stores and would each wait for the store before them
      constexpr int kG = 4;
#pragma unroll
      for (int i0 = 0; i0 < kMtPx; i0 += kG) {
        float ev[kG][RM];
#pragma unroll
        for (int i = 0; i < kG; ++i) {
          const int64_t pix = tile * kMtP + kMtPx * tp + i0 + i;
#pragma unroll
          for (int r = 0; r < RM; ++r) {
            const int m = tm + 16 * r;
            ev[i][r] = (p.E && pix < p.P && m < M) ? __ldg(p.E + pix * M + m) : 0.f;
          }
        }
#pragma unroll
        for (int i = 0; i < kG; ++i) {
          const int64_t pix = tile * kMtP + kMtPx * tp + i0 + i;
#pragma unroll
          for (int r = 0; r < RM; ++r) {
            const int m = tm + 16 * r;
            if (pix < p.P && m < M) p.Y[pix * M + m] = acc[i0 + i][r] + ev[i][r];
            acc[i0 + i][r] = 0.f;
          }
        }
      }
    }
  }
  if (it < items && tid == 0) {
    // a box never arrived: report it, and give the boxes still in flight (it .. it +
    // stages - 2) one more bounded wait before the CTA's shared memory is released
    atomicOr(p.status, kStTimeout);
    for (int64_t j = it; j < items && j < it + kMtStages - 1; ++j)
      tc::mbar_wait(&mbx[j % kMtStages], (uint32_t)((j / kMtStages) & 1), kMtWaitNs);
  }
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime.
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  });
  return fn;
}

template <int RM>
static cudaError_t measure_tiled(const Ctx& c, MtParams p) {
  const int kpad = (c.N + kMtK - 1) / kMtK * kMtK;
  p.lda = kpad + 4;  // 16-byte rows; 8 consecutive rows fall on distinct 4-bank groups
  const size_t smem = (size_t)mt_abytes(RM, p.lda) + (size_t)kMtStages * kMtP * kMtK * 4;
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  // X as a 2-D tensor of N columns (16-byte row stride: N is a multiple of 4) and P rows,
  // read in boxes of kMtK x kMtP: every box starts at a column that is a multiple of 32
  // (128 bytes) and a row that is a multiple of 256
  PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
  if (!encode) return cudaErrorNotSupported;
  CUtensorMap tmap;
  const cuuint64_t dims[2] = {(cuuint64_t)c.N, (cuuint64_t)p.P};
  const cuuint64_t strides[1] = {(cuuint64_t)c.N * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)kMtK, (cuuint32_t)kMtP};
  const cuuint32_t estr[2] = {1, 1};
  if (encode(&tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(p.X), dims, strides,
             box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_measure_tiled<RM>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t ntiles = (p.P + kMtP - 1) / kMtP;
  const int64_t grid = ntiles < c.num_sms ? ntiles : c.num_sms;
  k_measure_tiled<RM><<<(unsigned)grid, 256, smem, c.stream>>>(p, tmap);
  return cudaGetLastError();
}

// Momentum weights of Algorithm 1 steps 3-4: t_0 = 1, t_i = (1 + sqrt(1 + 4 t_{i-1}^2)) / 2,
// beta_i = (t_{i-1} - 1) / t_i, in FP64 by one thread (the sequence is the same for all
// pixels), stored as FP32 for the iteration kernels.
__global__ void k_momentum(int iters, float* beta) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  double t = 1.0;
  for (int i = 0; i < iters; ++i) {
    double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
    beta[i] = (float)((t - 1.0) / tn);
    t = tn;
  }
}

template <typename K>
void allow_smem(K kernel, size_t bytes) {
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

CvParams base_params(const Ctx& c) {
  CvParams p{};
  p.M = c.M;
  p.N = c.N;
  p.Npad = (c.N + 3) & ~3;
  p.lda = smem_ld(c.N);
  p.Mpad = (c.M + 3) & ~3;
  p.ldw = smem_ld(c.M);
  p.A = c.A32;
  p.W = c.W32;
  p.status = c.status;
  p.pairs = c.complex_pairs ? 1 : 0;
  return p;
}

template <int MR, int NCH>
cudaError_t fista_mr(const Ctx& c, CvParams p, int64_t blocks) {
  size_t smem = sizeof(float) * ((size_t)c.M * p.lda + (size_t)kT * p.lda + (size_t)c.M * kLdv);
  allow_smem(k_fista_f32<MR, NCH>, smem);
  k_fista_f32<MR, NCH><<<(unsigned)blocks, kThreads, smem, c.stream>>>(p);
  return cudaGetLastError();
}

template <int MR, int NCH>
cudaError_t admm_mr(const Ctx& c, CvParams p, int64_t blocks) {
  const size_t tiles = (size_t)kT * p.lda + (size_t)kT * p.ldw + (size_t)c.M * kLdv;
  size_t smem = sizeof(float) * ((size_t)c.M * p.lda + (size_t)c.M * p.ldw + tiles);
  if (smem > 227 * 1024) {
    // no room for W: its padded copy is read through L1/L2 instead (M x M, <= 66 KB)
    p.Wg = c.Wpad;
    smem = sizeof(float) * ((size_t)c.M * p.lda + tiles);
  }
  allow_smem(k_admm_f32<MR, NCH>, smem);
  k_admm_f32<MR, NCH><<<(unsigned)blocks, kThreads, smem, c.stream>>>(p);
  return cudaGetLastError();
}

}  // namespace

#define CS_DISPATCH_MR_NCH(FN, ...)                                  \
  do {                                                               \
    int mr_ = (c.M + 31) / 32, nch_ = (c.N + 127) / 128;             \
    if (nch_ == 1) {                                                 \
      if (mr_ == 1) return FN<1, 1>(__VA_ARGS__);                    \
      if (mr_ == 2) return FN<2, 1>(__VA_ARGS__);                    \
      if (mr_ == 3) return FN<3, 1>(__VA_ARGS__);                    \
      return FN<4, 1>(__VA_ARGS__);                                  \
    } else {                                                         \
      if (mr_ == 1) return FN<1, 2>(__VA_ARGS__);                    \
      if (mr_ == 2) return FN<2, 2>(__VA_ARGS__);                    \
      if (mr_ == 3) return FN<3, 2>(__VA_ARGS__);                    \
      return FN<4, 2>(__VA_ARGS__);                                  \
    }                                                                \
  } while (0)

cudaError_t momentum_table(Ctx& c, int iters) {
  // beta_i does not depend on the run length, so a context computes the sequence once
  // for the longest run it has seen and later calls read its prefix
  if (iters <= c.beta_valid) return cudaSuccess;
  if (c.beta_cap < iters || !c.beta) {
    int cap = iters > 2 * c.beta_cap ? iters : 2 * c.beta_cap;
    if (cap < 1024) cap = 1024;
    float* nb = nullptr;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&nb), sizeof(float) * cap);
    if (e != cudaSuccess) return e;
    if (c.beta) c.beta_retired.push_back(c.beta);
    c.beta = nb;
    c.beta_cap = cap;
    c.beta_valid = 0;
  }
  k_momentum<<<1, 1, 0, c.stream>>>(c.beta_cap, c.beta);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) c.beta_valid = c.beta_cap;
  return e;
}

cudaError_t launch_fista(Ctx& c, const ConvexArgs& a, bool table) {
  if (a.P == 0) return cudaSuccess;
  if (table) {
    cudaError_t e = momentum_table(c, a.iters);
    if (e != cudaSuccess) return e;
  }
  if (a.prec != CS_FP32 && !c.complex_pairs && fista_tc_supported(c.M, c.N)) {
    c.last_prec = CS_BF16;
    return launch_fista_tc(c, a);
  }
  c.last_prec = CS_FP32;
  CvParams p = base_params(c);
  p.beta = c.beta;
  p.Y = a.Y;
  p.X = a.X;
  p.P = a.P;
  p.c1 = (float)(1.0 / c.L);
  p.c2 = (float)(a.lambda / c.L);
  p.eps2 = (float)(a.eps * a.eps);
  p.start_done = a.eps > 1.0;
  p.iters = a.iters;
  p.iters_out = a.iters_out;
  p.conv_out = a.conv_out;
  int64_t blocks = (a.P + kT - 1) / kT;
  if (blocks == 0) return cudaSuccess;
  CS_DISPATCH_MR_NCH(fista_mr, c, p, blocks);
}

cudaError_t launch_admm(Ctx& c, const ConvexArgs& a) {
  if (a.P > 0 && a.prec != CS_FP32 && !c.complex_pairs && admm_tc_supported(c.M, c.N)) {
    c.last_prec = CS_BF16;
    return launch_admm_tc(c, a);
  }
  c.last_prec = CS_FP32;
  CvParams p = base_params(c);
  p.Y = a.Y;
  p.X = a.X;
  p.P = a.P;
  p.c1 = (float)a.rho;
  p.c2 = (float)(a.lambda / a.rho);
  p.eps2 = (float)(a.eps * a.eps);
  p.start_done = a.eps > 1.0;
  p.iters = a.iters;
  p.iters_out = a.iters_out;
  p.conv_out = a.conv_out;
  int64_t blocks = (a.P + kT - 1) / kT;
  if (blocks == 0) return cudaSuccess;
  CS_DISPATCH_MR_NCH(admm_mr, c, p, blocks);
}

template <int MR>
static cudaError_t measure_mr(const Ctx& c, CvParams p) {
  size_t smem = sizeof(float) * ((size_t)c.M * p.lda + (size_t)kT * p.lda);
  allow_smem(k_measure_f32<MR>, smem);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_measure_f32<MR>, kThreads, smem);
  int64_t ntiles = (p.P + kT - 1) / kT;
  int64_t grid = (int64_t)c.num_sms * (per_sm > 0 ? per_sm : 1);
  if (grid > ntiles) grid = ntiles;
  k_measure_f32<MR><<<(unsigned)grid, kThreads, smem, c.stream>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_measure(const Ctx& c, const float* X, float* Y, const float* E, int64_t P) {
  CvParams p = base_params(c);
  p.Yout = Y;
  p.X = const_cast<float*>(X);
  p.E = E;
  p.P = P;
  if (P == 0) return cudaSuccess;
  // the tiled kernel's tensor map addresses rows with 32-bit coordinates
  if (c.N % 4 == 0 && c.M <= 128 && (reinterpret_cast<uintptr_t>(X) & 15) == 0 &&
      P < ((int64_t)1 << 31) - kMtP) {
    MtParams q{c.M, c.N, 0, c.A32, X, E, Y, P, c.status};
    switch ((c.M + 15) / 16) {
      case 1: return measure_tiled<1>(c, q);
      case 2: return measure_tiled<2>(c, q);
      case 3: return measure_tiled<3>(c, q);
      case 4: return measure_tiled<4>(c, q);
      case 5: return measure_tiled<5>(c, q);
      case 6: return measure_tiled<6>(c, q);
      case 7: return measure_tiled<7>(c, q);
      default: return measure_tiled<8>(c, q);
    }
  }
  int mr = (c.M + 31) / 32;
  if (mr == 1) return measure_mr<1>(c, p);
  if (mr == 2) return measure_mr<2>(c, p);
  if (mr == 3) return measure_mr<3>(c, p);
  return measure_mr<4>(c, p);
}

}  // namespace cs
