// ADMM (Algorithm 2) on the tcgen05 tensor cores: the mixed-precision path (CS_BF16).
//
// The x-update x = (A^T A + rho I)^{-1} (A^T y + rho d), d = z - w, runs in its Woodbury
// form
//   h = W (y - A d),   x = d + A^T h,   W = (A A^T + rho I)^{-1} (factored once, FP64),
// whence A x = y - rho h: the residual of x is rho h and Delta = rho ||h - h_prev||, with
// h^0 = y / rho (r^0 = y).  One CTA of 8 warps owns a tile of 128 pixels (one per TMEM
// lane) for the whole solve.  Per iteration three products run as BF16 MMAs with FP32
// accumulation in TMEM, each operand split into hi + lo parts (three MMAs per product,
// about 16 bits of each operand; plain BF16 would leave a 2^-9 relative error in
// y - A d, which the method drives toward its noise floor):
//   GEMM1  T = D A^T   (128 x M, K = N)
//   GEMMW  H = E W     (128 x M, K = M),  E = Y - T
//   GEMM2  C = H A     (128 x N, K = M),  x = D + C
// Shared memory holds A and W once, in the dual layout, and one operand region that
// carries D, E and H in turn.  TMEM holds the product (T, H and C share its columns, as
// each is consumed before the next is written), z, and y in the columns past N of each
// half; w and h_prev live in registers, each warp owning 32 pixels and half the columns.
#include <cuda_runtime.h>

#include "cs_internal.cuh"
#include "tc_ptx.cuh"

namespace cs {
namespace {

constexpr int kTcThreads = 256;
constexpr uint64_t kWaitLimitNs = 100ull * 1000 * 1000;  // 100 ms per product

struct AtcParams {
  int M, N, Mp, Np;
  const double* A64;
  const double* W64;
  const float* Y;
  float* X;
  int64_t P;
  float rho, thr, eps2;
  int start_done, iters;
  int32_t* iters_out;
  uint8_t* conv_out;
  int* status;
  int inject_timeout;  // test hook: the first product is not issued (see launch_admm_tc)
};

// Issues one split product (thread 0) after the operand region is complete, and waits
// for it; false if the wait ran out.  issue = false leaves the product out (fault
// injection: the wait then runs out).
__device__ __forceinline__ bool tile_product(uint64_t* mbar, uint32_t& phase, uint32_t d,
                                             uint32_t o, uint32_t bh, uint32_t bl, int K,
                                             int S, bool b_mn, uint32_t idesc,
                                             bool issue = true) {
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (threadIdx.x == 0 && issue) {
    tc::split_product(d, o, bh, bl, K, S, b_mn, idesc);
    tc::mma_commit(mbar);
  }
  const bool late = __syncthreads_or(!tc::mbar_wait(mbar, phase, kWaitLimitNs));
  phase ^= 1u;
  tc::fence_after_sync();
  return !late;
}

template <int NH, int MH>
__global__ void __launch_bounds__(kTcThreads, 1) k_admm_tc(AtcParams p) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int sub = warp & 3, half = warp >> 2;
  const int r = 32 * sub + lane;  // tile row == TMEM lane
  const int M = p.M, N = p.N, Mp = p.Mp, Np = p.Np;
  const int S = Np * 16, SW = Mp * 16;
  const int KO = Np > Mp ? Np : Mp;
  unsigned char* sAh = sm;
  unsigned char* sAl = sAh + Mp * Np * 2;
  unsigned char* sWh = sAl + Mp * Np * 2;
  unsigned char* sWl = sWh + Mp * Mp * 2;
  unsigned char* sO = sWl + Mp * Mp * 2;                         // 2 x 128 x KO BF16
  float* red = reinterpret_cast<float*>(sO + 2 * 128 * KO * 2);  // [2][128]

  const int64_t pix = (int64_t)blockIdx.x * 128 + r;
  const bool valid = pix < p.P;

  // A (M x N) and W (M x M) split into BF16 hi + lo in the dual layout: GEMM1 reads A
  // K-major (A^T), GEMM2 reads A and GEMMW reads W MN-major
  tc::stage_split(p.A64, M, N, Mp, Np, sAh, sAl);
  tc::stage_split(p.W64, M, M, Mp, Mp, sWh, sWl);
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
  const uint32_t tZ = tl + 256;  // z, columns [256, 256 + Np)
  const int n0 = half * NH, m0 = half * MH;
  // this thread's half of y, in columns no product writes: [Np, Np + MH) of its half
  const uint32_t tY = tl + 256 * half + Np;
  const uint32_t uO = tc::smem_u32(sO), uAh = tc::smem_u32(sAh), uAl = tc::smem_u32(sAl);
  const uint32_t uWh = tc::smem_u32(sWh), uWl = tc::smem_u32(sWl);

  float w[NH], hp[MH];
  bool bad = false;
#pragma unroll
  for (int j = 0; j < NH; ++j) w[j] = 0.f;
#pragma unroll
  for (int c = 0; c < MH; c += 8) {
    float y8[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      int m = m0 + c + e;
      float v = (valid && m < M) ? p.Y[pix * M + m] : 0.f;
      bad |= !isfinite(v);
      y8[e] = v;
      hp[c + e] = v / p.rho;  // r^0 = y = rho h^0
    }
    tc::tmem_st8(tY + c, y8);
  }
  if (bad) atomicOr(p.status, kStNonFinite);
  {
    const float zero8[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int c = 0; c < NH; c += 8) tc::tmem_st8(tZ + n0 + c, zero8);
    tc::tmem_wait_st();
  }
  bool done = !valid;
  if (valid && (p.start_done || p.iters == 0)) {
    // no iteration: x = x^0 = 0
    for (int n = n0; n < n0 + NH && n < N; ++n) p.X[pix * N + n] = 0.f;
    if (half == 0) {
      if (p.iters_out) p.iters_out[pix] = 0;
      if (p.conv_out) p.conv_out[pix] = 0;
    }
    done = true;
  }

  const uint32_t id1 = tc::idesc_bf16(128, Mp, false);  // T = D A^T
  const uint32_t idw = tc::idesc_bf16(128, Mp, true);   // H = E W
  const uint32_t id2 = tc::idesc_bf16(128, Np, true);   // C = H A
  uint32_t phase = 0;
  bool failed = false;

  if (__syncthreads_or(!done)) {
    for (int i = 1;; ++i) {
      // ---- D = z - w, the operand of GEMM1 (two 8-column chunks per TMEM round trip)
#pragma unroll
      for (int c2 = 0; c2 < NH; c2 += 16) {
        float zc[2][8];
        tc::tmem_ld8(tZ + n0 + c2, zc[0]);
        if (c2 + 8 < NH) tc::tmem_ld8(tZ + n0 + c2 + 8, zc[1]);
        tc::tmem_wait_ld();
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int c = c2 + 8 * h;
          if (c < NH) {
            float d[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) d[e] = zc[h][e] - w[c + e];
            tc::put_operand8(sO, Np, r, n0 + c, d);
          }
        }
      }
      if (!tile_product(&mbar, phase, tR, uO, uAh, uAl, Np, S, false, id1,
                        !(p.inject_timeout && i == 1))) {
        failed = true;
        break;
      }
      // ---- E = Y - T, the operand of GEMMW
#pragma unroll
      for (int c2 = 0; c2 < MH; c2 += 16) {
        float t[2][8], y8[2][8];
        tc::tmem_ld8(tR + m0 + c2, t[0]);
        tc::tmem_ld8(tY + c2, y8[0]);
        if (c2 + 8 < MH) {
          tc::tmem_ld8(tR + m0 + c2 + 8, t[1]);
          tc::tmem_ld8(tY + c2 + 8, y8[1]);
        }
        tc::tmem_wait_ld();
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int c = c2 + 8 * h;
          if (c < MH) {
            float e8[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) e8[e] = y8[h][e] - t[h][e];
            tc::put_operand8(sO, Mp, r, m0 + c, e8);
          }
        }
      }
      if (!tile_product(&mbar, phase, tR, uO, uWh, uWl, Mp, SW, true, idw)) {
        failed = true;
        break;
      }
      // ---- h: Delta_i = rho ||h - h_prev||, and H, the operand of GEMM2
      float d2 = 0.f;
#pragma unroll
      for (int c2 = 0; c2 < MH; c2 += 16) {
        float hh[2][8];
        tc::tmem_ld8(tR + m0 + c2, hh[0]);
        if (c2 + 8 < MH) tc::tmem_ld8(tR + m0 + c2 + 8, hh[1]);
        tc::tmem_wait_ld();
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int c = c2 + 8 * q;
          if (c < MH) {
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              float df = hh[q][e] - hp[c + e];
              d2 += df * df;
              hp[c + e] = hh[q][e];
            }
            tc::put_operand8(sO, Mp, r, m0 + c, hh[q]);
          }
        }
      }
      red[half * 128 + r] = d2;
      if (!tile_product(&mbar, phase, tR, uO, uAh, uAl, Mp, S, true, id2)) {
        failed = true;
        break;
      }
      const float dtot = p.rho * p.rho * (red[r] + red[128 + r]);
      const bool conv_now = !done && dtot < p.eps2;
      const bool fin = !done && (conv_now || i == p.iters);
      // ---- x = d + A^T h, z = soft(x + w, lambda / rho), w = w + x - z
#pragma unroll
      for (int c2 = 0; c2 < NH; c2 += 16) {
        float C[2][8], zc[2][8];
        tc::tmem_ld8(tR + n0 + c2, C[0]);
        tc::tmem_ld8(tZ + n0 + c2, zc[0]);
        if (c2 + 8 < NH) {
          tc::tmem_ld8(tR + n0 + c2 + 8, C[1]);
          tc::tmem_ld8(tZ + n0 + c2 + 8, zc[1]);
        }
        tc::tmem_wait_ld();
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int c = c2 + 8 * q;
          if (c < NH) {
            float xo[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              const float x = (zc[q][e] - w[c + e]) + C[q][e];
              xo[e] = x;
              if (!done) {
                const float zn = tc::soft_thr(x + w[c + e], p.thr);
                w[c + e] = w[c + e] + x - zn;
                zc[q][e] = zn;
              }
            }
            tc::tmem_st8(tZ + n0 + c, zc[q]);
            if (fin) {
#pragma unroll
              for (int e = 0; e < 8; ++e)
                if (n0 + c + e < N) p.X[pix * N + n0 + c + e] = xo[e];
            }
          }
        }
      }
      tc::tmem_wait_st();
      if (fin && half == 0) {
        if (p.iters_out) p.iters_out[pix] = i;
        if (p.conv_out) p.conv_out[pix] = conv_now ? 1 : 0;
      }
      done = done || fin;
      if (!__syncthreads_or(!done)) break;
    }
  }
  if (failed) {
    // a product never completed: report, give it one more bounded wait (tile_product has
    // already advanced the phase past it), then release TMEM
    if (tid == 0) atomicOr(p.status, kStTimeout);
    tc::mbar_wait(&mbar, phase ^ 1u, kWaitLimitNs);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

size_t admm_tc_smem(int Mp, int Np) {
  const int KO = Np > Mp ? Np : Mp;
  return (size_t)4 * Mp * Np + (size_t)4 * Mp * Mp + (size_t)512 * KO + 256 * 4 + 64;
}

template <int NH, int MH>
cudaError_t run(const Ctx& c, const AtcParams& p, size_t smem) {
  auto kern = k_admm_tc<NH, MH>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  unsigned grid = (unsigned)((p.P + 127) / 128);
  kern<<<grid, kTcThreads, smem, c.stream>>>(p);
  return cudaGetLastError();
}

}  // namespace

// The tile shapes compiled for the tensor-core ADMM (half-rows of N and M per thread)
// whose operands fit in shared memory.
bool admm_tc_supported(int M, int N) {
  int Mp = (M + 15) / 16 * 16, Np = (N + 15) / 16 * 16;
  if (admm_tc_smem(Mp, Np) > 227 * 1024) return false;
  int NH = Np / 2, MH = Mp / 2;
  if (Np + MH > 256) return false;  // y's columns beside the product
  return (NH == 64 && MH == 24) || (NH == 104 && MH == 40);
}

cudaError_t launch_admm_tc(const Ctx& c, const ConvexArgs& a) {
  AtcParams p{};
  p.M = c.M;
  p.N = c.N;
  p.Mp = (c.M + 15) / 16 * 16;
  p.Np = (c.N + 15) / 16 * 16;
  p.A64 = c.A64;
  p.W64 = c.W64;
  p.Y = a.Y;
  p.X = a.X;
  p.P = a.P;
  p.rho = (float)a.rho;
  p.thr = (float)(a.lambda / a.rho);
  p.eps2 = (float)(a.eps * a.eps);
  p.start_done = a.eps > 1.0;
  p.iters = a.iters;
  p.iters_out = a.iters_out;
  p.conv_out = a.conv_out;
  p.status = c.status;
  p.inject_timeout = tc::inject_timeout();
  if (a.P == 0) return cudaSuccess;
  // at least 120 KB so that one CTA (which takes all 512 TMEM columns) runs per SM
  size_t smem = admm_tc_smem(p.Mp, p.Np);
  if (smem < 120 * 1024) smem = 120 * 1024;
  const int NH = p.Np / 2, MH = p.Mp / 2;
  if (NH == 64 && MH == 24) return run<64, 24>(c, p, smem);
  if (NH == 104 && MH == 40) return run<104, 40>(c, p, smem);
  return cudaErrorInvalidValue;
}

}  // namespace cs
