// ADMM (Algorithm 2) on the tcgen05 tensor cores: the mixed-precision path (CS_BF16).
//
// The x-update x = (A^T A + rho I)^{-1} (A^T y + rho d), d = z - w, runs in its Woodbury
// form
//   h = W (y - A d),   x = d + A^T h,   W = (A A^T + rho I)^{-1} (factored once, FP64),
// whence A x = y - rho h: the residual of x is rho h and Delta = rho ||h - h_prev||, with
// h^0 = y / rho (r^0 = y).  One CTA of 8 warps owns a tile of 128 pixels (one per TMEM
// lane) for the whole solve.  Per iteration three products run as BF16 MMAs with FP32
// accumulation in TMEM, each operand split into hi + lo parts (three MMAs per product,
// about 16 bits of each operand):
//   GEMM1  T = D A^T   (128 x M, K = N)
//   GEMMW  H = E W     (128 x M, K = M),  E = Y - T
//   GEMM2  C = H A     (128 x N, K = M),  x = D + C
//
// The iterate lives in TMEM as one vector per pixel, v = z_prev + C = x + w_prev: the
// z- and w-steps give z = soft(v, lambda / rho) and w = w_prev + x - z = v - z, so z, w
// and d = z - w = 2 soft(v) - v all follow from v, and the next v is soft(v) + C (v^0 =
// 0 is z^0 = w^0 = 0).  TMEM holds v (N columns) and one product region that T, H and C
// use in turn; y and h_prev live in registers (warp group g of a tile row owns half of
// every 64-column chunk).  Shared memory holds A and W split into BF16 hi + lo parts in
// the dual layout (read K-major and MN-major) and a ring of two or three operand buffers
// of 64 K-columns: the K-chunks of D stream through it, each chunk's MMAs running while
// the next chunk is written, then E's and H's chunks.
#include <cuda_runtime.h>

#include "cs_internal.cuh"
#include "tc_ptx.cuh"

namespace cs {
namespace {

constexpr int kTcThreads = 256;
constexpr uint64_t kWaitLimitNs = 100ull * 1000 * 1000;  // 100 ms per product
constexpr int kChunk = 64;                                // K-columns per operand buffer
constexpr int kBufBytes = 128 * kChunk * 2 * 2;           // hi + lo, 32 KB
constexpr int kLoOff = 128 * kChunk * 2;                  // lo part after hi

struct AtcParams {
  int M, N;
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
  unsigned long long* counter;  // next pixel to hand out (zeroed before the launch)
  int inject_timeout;  // test hook: the first product is not issued (see launch_admm_tc)
};

// Column plan of a tile shape (N and M padded to 16).
template <int NP, int MP>
struct Shape {
  static constexpr int QN = (NP + kChunk - 1) / kChunk;  // chunks of D (and of C, v)
  static constexpr int QM = (MP + kChunk - 1) / kChunk;  // chunks of E and H
  static constexpr int NH = NP / 2, MH = MP / 2;         // columns per thread
  static constexpr int TCOLS = 2 * NP <= 256 ? 256 : 512;
  static constexpr int A_BYTES = 4 * MP * NP, W_BYTES = 4 * MP * MP;
  static constexpr int NBUF =
      A_BYTES + W_BYTES + 3 * kBufBytes + 2048 <= 227 * 1024 ? 3 : 2;
  static constexpr int SMEM = A_BYTES + W_BYTES + NBUF * kBufBytes + 2 * 128 * 4;
  static_assert(2 * NP <= 512 && MP <= NP, "TMEM columns");
  static_assert(NP % 16 == 0 && MP % 16 == 0, "MMA shapes");
  static_assert(QM <= 2 && QM <= NBUF, "chunk plan");
  // dynamic plus about 1 KB of static shared memory (barriers, lane pixels)
  static_assert(A_BYTES + W_BYTES + 2 * kBufBytes + 1024 + 1024 <= 227 * 1024, "shared memory");
  // chunk q of an L-column operand: start, width
  __host__ __device__ static constexpr int cw(int L, int q) {
    return L - kChunk * q < kChunk ? L - kChunk * q : kChunk;
  }
  // offset of chunk q's columns in a thread's registers (every chunk but the last is full)
  __host__ __device__ static constexpr int ro(int q) { return (kChunk / 2) * q; }
};

using tc::put_operand8;
using tc::soft_thr;

// The finished lanes of a warp (fin) take the next pixels from the counter with one
// atomic: lane by lane in order, -1 once none is left.  All 32 lanes call it.
__device__ __forceinline__ void claim_pixels(bool fin, unsigned long long* counter, int64_t P,
                                             int* s_pix, int r, int lane) {
  const unsigned m = __ballot_sync(0xffffffffu, fin);
  if (!m) return;
  const int leader = __ffs(m) - 1;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(counter, (unsigned long long)__popc(m));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (fin) {
    const unsigned long long nx = base + __popc(m & ((1u << lane) - 1u));
    s_pix[r] = nx < (unsigned long long)P ? (int)nx : -1;
  }
}

// The split MMAs (hi*hi, lo*hi, hi*lo) of `steps` K-steps of 16: the operand at a (hi; lo
// at a + kLoOff, K-major in a 64-column buffer) against the matrix at bh / bl.
__device__ __forceinline__ void issue_steps(uint32_t d, uint32_t a, uint32_t bh, uint32_t bl,
                                            int steps, uint32_t b_step, uint32_t b_lbo,
                                            uint32_t b_sbo, uint32_t idesc, bool first) {
  for (int s = 0; s < steps; ++s) {
    const uint64_t ah = tc::sdesc(a + s * 256, 128, 16 * kChunk);
    const uint64_t al = tc::sdesc(a + kLoOff + s * 256, 128, 16 * kChunk);
    const uint64_t dh = tc::sdesc(bh + s * b_step, b_lbo, b_sbo);
    const uint64_t dl = tc::sdesc(bl + s * b_step, b_lbo, b_sbo);
    tc::mma_bf16(d, ah, dh, idesc, (first && s == 0) ? 0u : 1u);
    tc::mma_bf16(d, al, dh, idesc, 1u);
    tc::mma_bf16(d, ah, dl, idesc, 1u);
  }
}

template <int NP, int MP>
__global__ void __launch_bounds__(kTcThreads, 1) k_admm_tc(AtcParams p) {
  using S = Shape<NP, MP>;
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t mb_buf[3];  // MMAs reading ring buffer b completed
  __shared__ __align__(8) uint64_t mb_done;    // a whole product completed
  __shared__ __align__(8) uint64_t mb_drain;   // every MMA issued so far completed
  __shared__ uint32_t tmem_slot;
  __shared__ int s_fail;
  __shared__ int s_pix[128];  // the pixel each TMEM lane holds (-1: none left; P < 2^31)
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int sub = warp & 3, g = warp >> 2;
  const int r = 32 * sub + lane;  // tile row == TMEM lane
  const int M = p.M, N = p.N;
  constexpr int SA = NP * 16, SW = MP * 16;  // dual-layout row-group strides of A and W
  unsigned char* sAh = sm;
  unsigned char* sAl = sAh + MP * NP * 2;
  unsigned char* sWh = sAl + MP * NP * 2;
  unsigned char* sWl = sWh + MP * MP * 2;
  unsigned char* sB = sWl + MP * MP * 2;  // operand ring
  float* red = reinterpret_cast<float*>(sB + S::NBUF * kBufBytes);  // [2][128]


  // A (M x N) and W (M x M) split into BF16 hi + lo in the dual layout: GEMM1 reads A
  // K-major (A^T), GEMM2 reads A and GEMMW reads W MN-major
  tc::stage_split(p.A64, M, N, MP, NP, sAh, sAl);
  tc::stage_split(p.W64, M, M, MP, MP, sWh, sWl);
  if (tid == 0) {
    for (int k = 0; k < 3; ++k) tc::mbar_init(&mb_buf[k], 1);
    tc::mbar_init(&mb_done, 1);
    tc::mbar_init(&mb_drain, 1);
    s_fail = 0;
    s_pix[0] = (int)min(atomicAdd(p.counter, 128ull), (unsigned long long)p.P);  // this CTA's first 128 pixels
  }
  if (warp == 0) tc::tmem_alloc(&tmem_slot, S::TCOLS);
  tc::fence_async_smem();
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_slot;
  const uint32_t tl = tmem + ((uint32_t)(32 * sub) << 16);
  const uint32_t tR = tl;       // product region: T, H and C in turn
  const uint32_t tV = tl + NP;  // the iterate v, columns [NP, 2 NP)
  const uint32_t uB = tc::smem_u32(sB), uAh = tc::smem_u32(sAh), uAl = tc::smem_u32(sAl);
  const uint32_t uWh = tc::smem_u32(sWh), uWl = tc::smem_u32(sWl);
  // the grid is persistent: every TMEM lane holds one pixel and takes the next one from
  // the counter when its pixel finishes, so converged pixels leave no idle lanes behind
  int64_t pix = (int64_t)s_pix[0] + r;
  __syncthreads();
  if (pix >= p.P) pix = -1;
  bool valid = pix >= 0;

  float yv[S::MH], hp[S::MH];
  // y and h^0 = y / rho (r^0 = y) of the pixel this lane holds
  auto load_y = [&]() {
    const float* yrow = p.Y + (valid ? pix : 0) * M;
    bool bad = false;
#pragma unroll
    for (int k = 0; k < S::QM; ++k) {
      const int c0 = kChunk * k + g * (S::cw(MP, k) / 2);
#pragma unroll
      for (int c = 0; c < S::cw(MP, k) / 2; ++c) {
        const int m = c0 + c;
        const float v = (valid && m < M) ? __ldg(yrow + m) : 0.f;
        bad |= !isfinite(v);
        yv[S::ro(k) + c] = v;
        hp[S::ro(k) + c] = v / p.rho;
      }
    }
    if (bad) atomicOr(p.status, kStNonFinite);
  };
  {
    load_y();
    const float zero8[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int q = 0; q < S::QN; ++q)
#pragma unroll
      for (int c = 0; c < S::cw(NP, q) / 2; c += 8)
        tc::tmem_st8(tV + kChunk * q + g * (S::cw(NP, q) / 2) + c, zero8);
    tc::tmem_wait_st();
  }
  bool done = !valid;
  if (p.start_done || p.iters == 0) {
    // no iteration: x = x^0 = 0 for every pixel, each lane taking pixels until none is
    // left (the barriers are reached by every thread: the loop test is block-wide)
    while (__syncthreads_or(valid)) {
      if (valid) {
        for (int n = g; n < N; n += 2) p.X[pix * N + n] = 0.f;
        if (g == 0) {
          if (p.iters_out) p.iters_out[pix] = 0;
          if (p.conv_out) p.conv_out[pix] = 0;
        }
      }
      if (g == 0) claim_pixels(valid, p.counter, p.P, s_pix, r, lane);
      __syncthreads();
      if (valid) {
        pix = s_pix[r];
        valid = pix >= 0;
      }
    }
    done = true;
  }
  int k_it = 1;  // the lane's own iteration number

  const uint32_t id1 = tc::idesc_bf16(128, MP, false);  // T = D A^T
  const uint32_t idw = tc::idesc_bf16(128, MP, true);   // H = E W
  const uint32_t id2 = tc::idesc_bf16(128, NP, true);   // C = H A
  uint32_t ph_done = 0, ph_buf = 0;  // phase parities (bit b for buffer b)
  uint32_t pending = 0;              // buffers with a commit not yet waited for
  bool failed = false;
  // waits, by every thread, for the MMAs reading buffer b (if any are outstanding)
  auto free_buf = [&](int b) {
    if (pending & (1u << b)) {
      failed |= !tc::mbar_wait(&mb_buf[b], (ph_buf >> b) & 1u, kWaitLimitNs);
      ph_buf ^= 1u << b;
      pending &= ~(1u << b);
    }
  };
  auto wait_done = [&]() {
    failed |= !tc::mbar_wait(&mb_done, ph_done, kWaitLimitNs);
    ph_done ^= 1u;
    tc::fence_after_sync();
  };
  // makes the operand writes visible to the MMAs and lets thread 0 issue
  auto to_mma = [&]() {
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
  };

  if (__syncthreads_or(!done)) {
    for (int i = 1;; ++i) {
      // ---- GEMM1: T = D A^T, D = 2 soft(v) - v, chunk by chunk through the ring
#pragma unroll
      for (int q = 0; q < S::QN; ++q) {
        const int b = q % S::NBUF;
        free_buf(b);
        const int w2 = S::cw(NP, q) / 2, c0 = kChunk * q + g * w2;
        unsigned char* buf = sB + b * kBufBytes;
#pragma unroll
        for (int c2 = 0; c2 < w2; c2 += 16) {
          float vv[2][8];
          tc::tmem_ld8(tV + c0 + c2, vv[0]);
          if (c2 + 8 < w2) tc::tmem_ld8(tV + c0 + c2 + 8, vv[1]);
          tc::tmem_wait_ld();
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            if (c2 + 8 * h < w2) {
              float d8[8];
#pragma unroll
              for (int e = 0; e < 8; ++e) d8[e] = 2.f * soft_thr(vv[h][e], p.thr) - vv[h][e];
              put_operand8(buf, kChunk, r, c0 - kChunk * q + c2 + 8 * h, d8);
            }
          }
        }
        to_mma();
        if (tid == 0 && !(p.inject_timeout && i == 1)) {
          const uint32_t boff = (kChunk * q / 16) * 256;
          issue_steps(tmem, uB + b * kBufBytes, uAh + boff, uAl + boff, S::cw(NP, q) / 16,
                      256, 128, SA, id1, q == 0);
          tc::mma_commit(&mb_buf[b]);
          if (q == S::QN - 1) tc::mma_commit(&mb_done);
        }
        pending |= 1u << b;
      }
      wait_done();
      // ---- GEMMW: H = E W, E = Y - T
#pragma unroll
      for (int k = 0; k < S::QM; ++k) {
        free_buf(k);
        const int w2 = S::cw(MP, k) / 2, c0 = kChunk * k + g * w2;
        unsigned char* buf = sB + k * kBufBytes;
#pragma unroll
        for (int c2 = 0; c2 < w2; c2 += 16) {
          float t[2][8];
          tc::tmem_ld8(tR + c0 + c2, t[0]);
          if (c2 + 8 < w2) tc::tmem_ld8(tR + c0 + c2 + 8, t[1]);
          tc::tmem_wait_ld();
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            if (c2 + 8 * h < w2) {
              float e8[8];
#pragma unroll
              for (int e = 0; e < 8; ++e) e8[e] = yv[S::ro(k) + c2 + 8 * h + e] - t[h][e];
              put_operand8(buf, kChunk, r, c2 + 8 * h + g * w2, e8);
            }
          }
        }
      }
      to_mma();
      if (tid == 0) {
#pragma unroll
        for (int k = 0; k < S::QM; ++k) {
          const uint32_t boff = (kChunk * k / 16) * 2 * SW;
          issue_steps(tmem, uB + k * kBufBytes, uWh + boff, uWl + boff, S::cw(MP, k) / 16,
                      2 * SW, SW, 128, idw, k == 0);
          tc::mma_commit(&mb_buf[k]);
        }
        tc::mma_commit(&mb_done);
      }
      pending |= (1u << S::QM) - 1u;
      wait_done();
      // ---- h: Delta_i = rho ||h - h_prev||, and H, the operand of GEMM2
      float d2 = 0.f;
#pragma unroll
      for (int k = 0; k < S::QM; ++k) {
        free_buf(k);
        const int w2 = S::cw(MP, k) / 2, c0 = kChunk * k + g * w2;
        unsigned char* buf = sB + k * kBufBytes;
#pragma unroll
        for (int c2 = 0; c2 < w2; c2 += 16) {
          float hh[2][8];
          tc::tmem_ld8(tR + c0 + c2, hh[0]);
          if (c2 + 8 < w2) tc::tmem_ld8(tR + c0 + c2 + 8, hh[1]);
          tc::tmem_wait_ld();
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            if (c2 + 8 * h < w2) {
#pragma unroll
              for (int e = 0; e < 8; ++e) {
                const int j = S::ro(k) + c2 + 8 * h + e;
                const float df = hh[h][e] - hp[j];
                d2 = fmaf(df, df, d2);
                hp[j] = hh[h][e];
              }
              put_operand8(buf, kChunk, r, c2 + 8 * h + g * w2, hh[h]);
            }
          }
        }
      }
      red[g * 128 + r] = d2;
      to_mma();
      if (tid == 0) {
#pragma unroll
        for (int k = 0; k < S::QM; ++k) {
          const uint32_t boff = (kChunk * k / 16) * 2 * SA;
          issue_steps(tmem, uB + k * kBufBytes, uAh + boff, uAl + boff, S::cw(MP, k) / 16,
                      2 * SA, SA, 128, id2, k == 0);
          tc::mma_commit(&mb_buf[k]);
        }
        tc::mma_commit(&mb_done);
      }
      pending |= (1u << S::QM) - 1u;
      const float dtot = p.rho * p.rho * (red[r] + red[128 + r]);
      const bool conv_now = !done && dtot < p.eps2;
      const bool fin = !done && (conv_now || k_it == p.iters);
      wait_done();
      // ---- x = d + C, z = soft(v, lambda / rho), w = v - z; the next v = z + C
#pragma unroll
      for (int q = 0; q < S::QN; ++q) {
        const int w2 = S::cw(NP, q) / 2, c0 = kChunk * q + g * w2;
#pragma unroll
        for (int c2 = 0; c2 < w2; c2 += 16) {
          float C[2][8], vv[2][8];
          tc::tmem_ld8(tR + c0 + c2, C[0]);
          tc::tmem_ld8(tV + c0 + c2, vv[0]);
          if (c2 + 8 < w2) {
            tc::tmem_ld8(tR + c0 + c2 + 8, C[1]);
            tc::tmem_ld8(tV + c0 + c2 + 8, vv[1]);
          }
          tc::tmem_wait_ld();
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int c = c2 + 8 * h;
            if (c < w2) {
              float vn[8];
#pragma unroll
              for (int e = 0; e < 8; ++e) {
                const float z = soft_thr(vv[h][e], p.thr);
                const float x = (2.f * z - vv[h][e]) + C[h][e];
                vn[e] = done ? vv[h][e] : z + C[h][e];
                if (fin && c0 + c + e < N) p.X[pix * N + c0 + c + e] = x;
              }
              tc::tmem_st8(tV + c0 + c, vn);
            }
          }
        }
      }
      tc::tmem_wait_st();
      // a finished lane's next pixel starts from v = 0 (out of the hot loop above; the
      // TMEM stores are warp-wide, so the warp's other lanes write their v back)
      if (__any_sync(0xffffffffu, fin)) {
#pragma unroll
        for (int q = 0; q < S::QN; ++q) {
          const int c0 = kChunk * q + g * (S::cw(NP, q) / 2);
#pragma unroll
          for (int c = 0; c < S::cw(NP, q) / 2; c += 8) {
            float vv[8];
            tc::tmem_ld8(tV + c0 + c, vv);
            tc::tmem_wait_ld();
#pragma unroll
            for (int e = 0; e < 8; ++e) vv[e] = fin ? 0.f : vv[e];
            tc::tmem_st8(tV + c0 + c, vv);
          }
        }
        tc::tmem_wait_st();
      }
      if (fin && g == 0) {
        if (p.iters_out) p.iters_out[pix] = k_it;
        if (p.conv_out) p.conv_out[pix] = conv_now ? 1 : 0;
      }
      // a finished lane takes the next pixel: its group-0 thread claims it for the row,
      // one atomic per warp for all of the warp's finished lanes
      if (g == 0) claim_pixels(fin, p.counter, p.P, s_pix, r, lane);
      done = done || fin;
      if (failed) s_fail = 1;
      tc::fence_before_sync();
      if (!__syncthreads_or(!done || (fin && g == 0 && s_pix[r] >= 0))) break;
      tc::fence_after_sync();
      if (s_fail) {
        failed = true;
        break;
      }
      ++k_it;
      if (fin) {
        pix = s_pix[r];
        valid = pix >= 0;
        done = !valid;
        k_it = 1;
        if (valid) load_y();
      }
    }
  }
  // every MMA has completed unless a wait ran out (each product's last commit is waited)
  if (__syncthreads_or(failed)) {
    // a product never completed: report, then one commit that tracks every MMA thread 0
    // issued gets a last bounded wait before TMEM is released
    if (tid == 0) {
      atomicOr(p.status, kStTimeout);
      tc::mma_commit(&mb_drain);
    }
    tc::mbar_wait(&mb_drain, 0, kWaitLimitNs);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, S::TCOLS);
}

template <int NP, int MP>
cudaError_t run(const Ctx& c, const AtcParams& p) {
  auto kern = k_admm_tc<NP, MP>;
  // at least 120 KB so that one CTA (which may take all 512 TMEM columns) runs per SM
  size_t smem = Shape<NP, MP>::SMEM;
  if (smem < 120 * 1024) smem = 120 * 1024;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  long long grid = (p.P + 127) / 128;
  if (grid > c.num_sms) grid = c.num_sms;  // persistent: one CTA (all of TMEM) per SM
  e = cudaMemsetAsync(p.counter, 0, sizeof(unsigned long long), c.stream);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)grid, kTcThreads, smem, c.stream>>>(p);
  return cudaGetLastError();
}

// The tile shapes compiled for the tensor-core ADMM: (N, M) padded to 16.
#define CS_ADMM_TC_SHAPES(X) X(128, 48) X(208, 80) X(224, 96) X(256, 112)

}  // namespace

bool admm_tc_supported(int M, int N) {
  const int Mp = (M + 15) / 16 * 16, Np = (N + 15) / 16 * 16;
#define CS_ADMM_TC_MATCH(NP_, MP_) \
  if (Np == NP_ && Mp == MP_) return true;
  CS_ADMM_TC_SHAPES(CS_ADMM_TC_MATCH)
#undef CS_ADMM_TC_MATCH
  return false;
}

cudaError_t launch_admm_tc(const Ctx& c, const ConvexArgs& a) {
  AtcParams p{};
  p.M = c.M;
  p.N = c.N;
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
  p.counter = a.counter ? a.counter : c.conv_counter;
  p.inject_timeout = tc::inject_timeout();
  if (a.P == 0) return cudaSuccess;
  const int Mp = (c.M + 15) / 16 * 16, Np = (c.N + 15) / 16 * 16;
#define CS_ADMM_TC_RUN(NP_, MP_) \
  if (Np == NP_ && Mp == MP_) return run<NP_, MP_>(c, p);
  CS_ADMM_TC_SHAPES(CS_ADMM_TC_RUN)
#undef CS_ADMM_TC_RUN
  return cudaErrorInvalidValue;
}

}  // namespace cs
