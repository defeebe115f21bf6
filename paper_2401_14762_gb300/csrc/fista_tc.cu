// FISTA (Algorithm 1) on the tcgen05 tensor cores: the mixed-precision path (CS_BF16).
//
// One CTA of 8 warps owns a tile of 128 pixels (one per TMEM lane) for the whole solve.
// Per iteration the two products of Algorithm 1 step 1 run as BF16 MMAs with FP32
// accumulation in TMEM:
//   GEMM2  C = (A z - y) A       (128 x N, K = M)   -- A^T applied to the residual
//   GEMM1  u = x A^T             (128 x M, K = N)   -- A x, whence A z = u + beta (u - u_prev)
// Every operand is split into BF16 hi + lo parts and each product is the three MMAs
// hi*hi + lo*hi + hi*lo, which keeps about 16 bits of each operand: plain BF16 in either
// product would leave a 2^-9 relative error in A z - y, comparable to the residual the
// method drives to zero.  Shared memory holds A_hi and A_lo once, in a layout that GEMM1
// reads K-major and GEMM2 reads MN-major, plus one operand region that alternates
// between the residual (for GEMM2) and the iterate (for GEMM1).  TMEM holds the product
// (C and u never live at the same time, so they share columns) and the FP32 iterate x;
// z, u_prev and y live in registers, each warp owning 32 pixels and half the columns.
#include <cuda_runtime.h>

#include "cs_internal.cuh"
#include "tc_ptx.cuh"

namespace cs {
namespace {

constexpr int kTcThreads = 256;
constexpr uint64_t kWaitLimitNs = 100ull * 1000 * 1000;  // 100 ms per product

struct FtcParams {
  int M, N, Mp, Np;
  const double* A64;
  const float* Y;
  float* X;
  int64_t P;
  float invL, thr, eps2;
  int start_done, iters;
  int32_t* iters_out;
  uint8_t* conv_out;
  int* status;
  const float* beta;  // momentum weights beta_i, i = 1..iters
  int inject_timeout;  // test hook: the first product is not issued (see launch_fista_tc)
};

using tc::put_operand8;
using tc::soft_thr;

template <int NH, int MH>
__global__ void __launch_bounds__(kTcThreads, 1) k_fista_tc(FtcParams p) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int sub = warp & 3, half = warp >> 2;
  const int r = 32 * sub + lane;  // tile row == TMEM lane
  const int M = p.M, N = p.N, Mp = p.Mp, Np = p.Np;
  const int S = Np * 16;
  unsigned char* sAh = sm;
  unsigned char* sAl = sAh + Mp * Np * 2;
  unsigned char* sO = sAl + Mp * Np * 2;                         // 2 x 128 x Np BF16
  float* red = reinterpret_cast<float*>(sO + 2 * 128 * Np * 2);  // [2][128]

  const int64_t pix = (int64_t)blockIdx.x * 128 + r;
  const bool valid = pix < p.P;

  // A (M x N) split into BF16 hi + lo (from FP64) in the dual layout, zero padded to
  // Mp x Np: GEMM1 reads it K-major (A^T), GEMM2 MN-major
  tc::stage_split(p.A64, M, N, Mp, Np, sAh, sAl);
  if (tid == 0) tc::mbar_init(&mbar, 1);
  if (warp == 0) tc::tmem_alloc(&tmem_slot, 512);
  tc::fence_async_smem();
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_slot;
  const uint32_t tl = tmem + ((uint32_t)(32 * sub) << 16);
  const uint32_t tR = tl;        // product columns [0, 256)
  const uint32_t tX = tl + 256;  // iterate x, columns [256, 256 + Np)
  const int n0 = half * NH, m0 = half * MH;

  float z[NH], up[MH], yv[MH];
  bool bad = false;
#pragma unroll
  for (int j = 0; j < NH; ++j) z[j] = 0.f;
#pragma unroll
  for (int j = 0; j < MH; ++j) {
    int m = m0 + j;
    float v = (valid && m < M) ? p.Y[pix * M + m] : 0.f;
    bad |= !isfinite(v);
    yv[j] = v;
    up[j] = 0.f;
  }
  if (bad) atomicOr(p.status, kStNonFinite);
  {
    const float zero8[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int c = 0; c < NH; c += 8) tc::tmem_st8(tX + n0 + c, zero8);
    tc::tmem_wait_st();
  }

  const uint32_t id2 = tc::idesc_bf16(128, Np, true);   // GEMM2: B = A read MN-major
  const uint32_t id1 = tc::idesc_bf16(128, Mp, false);  // GEMM1: B = A read K-major
  bool done = !valid;
  float beta_prev = 0.f;
  uint32_t phase = 0;
  bool failed = false;

  for (int i = 1;; ++i) {
    // ---- residual of the extrapolated point, A z - y = u + beta (u - u_prev) - y, and
    //      Delta_{i-1} = ||u^{i-1} - u^{i-2}||  (u^0 = 0)
    float d2 = 0.f;
#pragma unroll
    for (int c2 = 0; c2 < MH; c2 += 16) {  // two 8-column chunks per TMEM round trip
      float u[2][8];
      if (i > 1) {
        tc::tmem_ld8(tR + m0 + c2, u[0]);
        if (c2 + 8 < MH) tc::tmem_ld8(tR + m0 + c2 + 8, u[1]);
        tc::tmem_wait_ld();
      } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) u[0][e] = u[1][e] = 0.f;
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int c = c2 + 8 * h;
        if (c < MH) {
          float v[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            float df = u[h][e] - up[c + e];
            d2 += df * df;
            v[e] = u[h][e] + beta_prev * df - yv[c + e];
            up[c + e] = u[h][e];
          }
          put_operand8(sO, Mp, r, m0 + c, v);
        }
      }
    }
    red[half * 128 + r] = d2;
    __syncthreads();
    const float dtot = red[r] + red[128 + r];
    // x^{i-1} is final if Delta_{i-1} < eps, if the cap is reached, or (eps > 1) at once
    const bool conv_now = !done && i > 1 && dtot < p.eps2;
    const bool fin = !done && (conv_now || i - 1 == p.iters || (i == 1 && p.start_done));
    if (__any_sync(0xffffffffu, fin)) {
#pragma unroll
      for (int c = 0; c < NH; c += 8) {
        float xv[8];
        tc::tmem_ld8(tX + n0 + c, xv);
        tc::tmem_wait_ld();
        if (fin) {
#pragma unroll
          for (int e = 0; e < 8; ++e)
            if (n0 + c + e < N) p.X[pix * N + n0 + c + e] = xv[e];
        }
      }
      if (fin && half == 0) {
        if (p.iters_out) p.iters_out[pix] = i - 1;
        if (p.conv_out) p.conv_out[pix] = conv_now ? 1 : 0;
      }
    }
    done = done || fin;
    if (!__syncthreads_or(!done)) break;

    // ---- GEMM2: C = V_hi A_hi + V_lo A_hi + V_hi A_lo   (K = Mp)
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (tid == 0 && !(p.inject_timeout && i == 1)) {
      tc::split_product(tR, tc::smem_u32(sO), tc::smem_u32(sAh), tc::smem_u32(sAl), Mp, S,
                        true, id2);
      tc::mma_commit(&mbar);
    }
    if (__syncthreads_or(!tc::mbar_wait(&mbar, phase, kWaitLimitNs))) {
      failed = true;
      break;
    }
    phase ^= 1u;
    tc::fence_after_sync();

    // ---- steps 1-4: aux = z - C / L, x = soft(aux, lambda / L), t, z
    const float beta = p.beta[i - 1];
    // two 8-column chunks per TMEM round trip
#pragma unroll
    for (int c2 = 0; c2 < NH; c2 += 16) {
      float C[2][8], xp[2][8];
      tc::tmem_ld8(tR + n0 + c2, C[0]);
      tc::tmem_ld8(tX + n0 + c2, xp[0]);
      if (c2 + 8 < NH) {
        tc::tmem_ld8(tR + n0 + c2 + 8, C[1]);
        tc::tmem_ld8(tX + n0 + c2 + 8, xp[1]);
      }
      tc::tmem_wait_ld();
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int c = c2 + 8 * h;
        if (c < NH) {
          float xn[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            float xx = soft_thr(z[c + e] - C[h][e] * p.invL, p.thr);
            if (!done) {
              z[c + e] = xx + beta * (xx - xp[h][e]);
            } else {
              xx = xp[h][e];
            }
            xn[e] = xx;
          }
          tc::tmem_st8(tX + n0 + c, xn);
          put_operand8(sO, Np, r, n0 + c, xn);
        }
      }
    }
    tc::tmem_wait_st();

    // ---- GEMM1: u = X_hi A_hi^T + X_lo A_hi^T + X_hi A_lo^T   (K = Np)
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (tid == 0) {
      tc::split_product(tR, tc::smem_u32(sO), tc::smem_u32(sAh), tc::smem_u32(sAl), Np, S,
                        false, id1);
      tc::mma_commit(&mbar);
    }
    if (__syncthreads_or(!tc::mbar_wait(&mbar, phase, kWaitLimitNs))) {
      failed = true;
      break;
    }
    phase ^= 1u;
    tc::fence_after_sync();
    beta_prev = beta;
  }
  if (failed) {
    // a product never completed: report, give it one more bounded wait, then release TMEM
    if (tid == 0) atomicOr(p.status, kStTimeout);
    tc::mbar_wait(&mbar, phase, kWaitLimitNs);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

template <int NH, int MH>
cudaError_t run(const Ctx& c, const FtcParams& p, size_t smem) {
  auto kern = k_fista_tc<NH, MH>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  unsigned grid = (unsigned)((p.P + 127) / 128);
  kern<<<grid, kTcThreads, smem, c.stream>>>(p);
  return cudaGetLastError();
}

size_t tc_smem(int Mp, int Np) { return (size_t)4 * Mp * Np + (size_t)512 * Np + 256 * 4 + 64; }

}  // namespace

// The tile shapes compiled for the tensor-core FISTA (half-rows of N and M per thread).
bool fista_tc_supported(int M, int N) {
  int Mp = (M + 15) / 16 * 16, Np = (N + 15) / 16 * 16;
  if (tc_smem(Mp, Np) > 227 * 1024) return false;
  int NH = Np / 2, MH = Mp / 2;
  return (NH == 64 && MH == 24) || (NH == 104 && MH == 40) || (NH == 112 && MH == 48);
}

cudaError_t launch_fista_tc(const Ctx& c, const ConvexArgs& a) {
  FtcParams p{};
  p.M = c.M;
  p.N = c.N;
  p.Mp = (c.M + 15) / 16 * 16;
  p.Np = (c.N + 15) / 16 * 16;
  p.A64 = c.A64;
  p.Y = a.Y;
  p.X = a.X;
  p.P = a.P;
  p.invL = (float)(1.0 / c.L);
  p.thr = (float)(a.lambda / c.L);
  p.eps2 = (float)(a.eps * a.eps);
  p.start_done = a.eps > 1.0;
  p.iters = a.iters;
  p.iters_out = a.iters_out;
  p.conv_out = a.conv_out;
  p.status = c.status;
  p.beta = c.beta;
  p.inject_timeout = tc::inject_timeout();
  if (a.P == 0) return cudaSuccess;
  // at least 120 KB so that one CTA (which takes all 512 TMEM columns) runs per SM
  size_t smem = tc_smem(p.Mp, p.Np);
  if (smem < 120 * 1024) smem = 120 * 1024;
  const int NH = p.Np / 2, MH = p.Mp / 2;
  if (NH == 64 && MH == 24) return run<64, 24>(c, p, smem);
  if (NH == 104 && MH == 40) return run<104, 40>(c, p, smem);
  if (NH == 112 && MH == 48) return run<112, 48>(c, p, smem);
  return cudaErrorInvalidValue;
}

}  // namespace cs
