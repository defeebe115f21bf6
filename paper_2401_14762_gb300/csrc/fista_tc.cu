// FISTA (Algorithm 1) on the tcgen05 tensor cores: the mixed-precision path (CS_BF16).
//
// One CTA of 8 warps owns a tile of 128 pixels (one per TMEM lane) for the whole solve.
// Per iteration the two products of Algorithm 1 step 1 run as BF16 MMAs with FP32
// accumulation in TMEM:
//   GEMM2  C = (A z - y) A       (128 x N, K = M)   -- A^T applied to the residual
//   GEMM1  D = (x - x_prev) A^T  (128 x M, K = N)   -- the change of u = A x, whence the
//                                                      residual R = u - y += D and
//                                                      A z - y = R + beta D
// Every operand is split into BF16 hi + lo parts and each product is the three MMAs
// hi*hi + lo*hi + hi*lo, which keeps about 16 bits of each operand: plain BF16 in either
// product leaves a 2^-9 relative error in A z - y, comparable to the residual the method
// drives to zero (a numpy model of the 300-iteration run gives rel-L2 1e-2 against FP64
// for plain BF16, 6e-3 with a 100-iteration split tail, 1e-4 for the split products).
//
// Shared memory holds A_hi and A_lo once, in a layout that GEMM1 reads K-major and GEMM2
// reads MN-major, and a ring of operand buffers of 64 K-columns each (3 or 4, whatever
// fits beside A): the residual's two K-chunks, then the iterate's K-chunks.  TMEM holds
// two product regions T0, T1 (RW columns each) and the FP32 iterate x.  The products are
// split so that the MMAs overlap the epilogues:
//   * GEMM2 runs as two column halves, into the free region and into the region that
//     held D (consumed by the residual epilogue just before);
//   * the x epilogue works through the iterate in K-chunks: half 0 of C (ready first)
//     while GEMM2's half 1 still multiplies, then half 1; GEMM1 accumulates D into the
//     region of C's half 0 chunk by chunk as soon as that half is consumed, so its MMAs
//     run under the epilogue of C's half 1.
// Each phase commits to its own mbarrier; the regions swap roles every iteration.  z and
// R live in registers (warp group g of a tile row owns half of every chunk); y is read
// once.  Multiplying the increment keeps the residual accurate without re-reading y:
// the split product errs relative to |x_i - x_{i-1}|, not to |x| (the numpy model gives
// the same rel-L2 as products of x itself).
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

struct FtcParams {
  int M, N;
  const double* A64;
  const float* Y;
  float* X;
  int64_t P;
  float invL, thr, eps2;
  int start_done, iters;
  int32_t* iters_out;
  uint8_t* conv_out;
  int* status;
  const float* beta;   // momentum weights beta_i, i = 1..iters
  unsigned long long* counter;  // next pixel to hand out (zeroed before the launch)
  int inject_timeout;  // test hook: the first product is not issued (see launch_fista_tc)
};

// Column partition of a tile shape (N and M padded to 16).
template <int NP, int MP>
struct Shape {
  static constexpr int NA = ((NP / 2 + 15) / 16) * 16;  // C's half 0: columns [0, NA)
  static constexpr int NB = NP - NA;                    // half 1: [NA, NP)
  static constexpr int RW0 = NA > NB ? NA : NB;
  static constexpr int RW = RW0 > MP ? RW0 : MP;        // width of a product region
  static constexpr int Q0 = (NA + kChunk - 1) / kChunk;  // x chunks in half 0
  static constexpr int Q1 = (NB + kChunk - 1) / kChunk;
  static constexpr int Q = Q0 + Q1;
  static constexpr int KW = (MP + kChunk - 1) / kChunk;  // residual chunks
  static constexpr int NH = NP / 2, MH = MP / 2;          // columns per thread
  static constexpr int TCOLS = 2 * RW + NP <= 256 ? 256 : 512;
  static constexpr int A_BYTES = 4 * MP * NP;
  // operand buffers: 4 if they fit beside A and the reduction slots, else 3
  static constexpr int NBUF = A_BYTES + 4 * kBufBytes + 2048 <= 227 * 1024 ? 4 : 3;
  static constexpr int SMEM = A_BYTES + NBUF * kBufBytes + 2 * 128 * 4;
  static_assert(2 * RW + NP <= 512, "TMEM columns");
  static_assert(NA % 16 == 0 && NB % 16 == 0 && MP % 16 == 0, "MMA N multiple of 16");
  static_assert(Q <= 4 && KW <= 2, "chunk plan");
  static_assert(A_BYTES + 3 * kBufBytes + 2048 <= 227 * 1024, "shared memory");

  // x chunk q: start column and width
  __host__ __device__ static constexpr int xc(int q) {
    return q < Q0 ? kChunk * q : NA + kChunk * (q - Q0);
  }
  __host__ __device__ static constexpr int xw(int q) {
    return q < Q0 ? (NA - kChunk * q < kChunk ? NA - kChunk * q : kChunk)
                  : (NB - kChunk * (q - Q0) < kChunk ? NB - kChunk * (q - Q0) : kChunk);
  }
  // offset of chunk q's columns in this thread's z registers
  // (every chunk but the last of each half is kChunk wide)
  __host__ __device__ static constexpr int zo(int q) {
    return q < Q0 ? (kChunk / 2) * q : NA / 2 + (kChunk / 2) * (q - Q0);
  }
  // residual chunk k: start, width, offset in the R registers
  __host__ __device__ static constexpr int wc(int k) { return kChunk * k; }
  __host__ __device__ static constexpr int ww(int k) {
    return MP - kChunk * k < kChunk ? MP - kChunk * k : kChunk;
  }
  __host__ __device__ static constexpr int uo(int k) { return (kChunk / 2) * k; }
  // the ring buffer that x chunk q is staged in (residual chunks use buffers 0 and 1)
  __host__ __device__ static constexpr int xbuf(int q) {
    return NBUF == 4 ? (q + 2) & 3 : (q == 0 ? 2 : (q == 1 ? 0 : (q == 2 ? 1 : 2)));
  }
  // x chunk q overwrites a buffer GEMM2 reads: wait for GEMM2 to finish first
  __host__ __device__ static constexpr bool needs_c1(int q) { return q >= Q0 || xbuf(q) < 2; }
  // x chunk q overwrites buffer 2 while GEMM1's first chunks may still read it
  __host__ __device__ static constexpr bool needs_u01(int q) {
    return NBUF == 3 && q > 0 && xbuf(q) == xbuf(0);
  }
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

// Issues the split MMAs (hi*hi, lo*hi, hi*lo) of `steps` K-steps of 16: the operand at
// a (hi; lo at a + kLoOff, K-major, 64 K-columns per buffer row group) against the
// dictionary at bh / bl.
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
__global__ void __launch_bounds__(kTcThreads, 1) k_fista_tc(FtcParams p) {
  using S = Shape<NP, MP>;
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t mb[5];  // GEMM2 half 0, half 1, GEMM1 first chunks, GEMM1,
                                           // and the drain after a failed wait
  __shared__ uint32_t tmem_slot;
  __shared__ int s_fail;  // a bounded wait ran out (set by any thread, read after a barrier)
  __shared__ int s_pix[128];  // the pixel each TMEM lane holds (-1: none left; P < 2^31)
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int sub = warp & 3, g = warp >> 2;
  const int r = 32 * sub + lane;  // tile row == TMEM lane
  const int M = p.M, N = p.N;
  constexpr int SD = NP * 16;  // dual-layout row-group stride of A
  unsigned char* sAh = sm;
  unsigned char* sAl = sAh + MP * NP * 2;
  unsigned char* sB = sAl + MP * NP * 2;  // operand ring
  float* red = reinterpret_cast<float*>(sB + S::NBUF * kBufBytes);  // [2][128]


  // A (M x N) split into BF16 hi + lo (from FP64) in the dual layout, zero padded to
  // MP x NP: GEMM1 reads it K-major (A^T), GEMM2 MN-major
  tc::stage_split(p.A64, M, N, MP, NP, sAh, sAl);
  if (tid == 0) {
    for (int k = 0; k < 5; ++k) tc::mbar_init(&mb[k], 1);
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
  const uint32_t tX = tl + 2 * S::RW;  // iterate x, columns [2 RW, 2 RW + NP)
  // the grid is persistent: every TMEM lane holds one pixel and takes the next one from
  // the counter when its pixel finishes, so converged pixels leave no idle lanes behind
  int64_t pix = (int64_t)s_pix[0] + r;
  __syncthreads();
  if (pix >= p.P) pix = -1;
  bool valid = pix >= 0;
  const uint32_t uB = tc::smem_u32(sB), uAh = tc::smem_u32(sAh), uAl = tc::smem_u32(sAl);

  // z in registers; R = u - y = A x - y, the residual of the iterate, in registers too:
  // GEMM1 multiplies the increment x_i - x_{i-1}, so R is updated as R += D with
  // D = A (x_i - x_{i-1}) = u_i - u_{i-1}, which is also what the extrapolation and Delta
  // need.  The split product of an increment errs relative to the increment, so y is
  // read once and the residual never loses accuracy to the size of A x.
  float z[S::NH], R[S::MH];
#pragma unroll
  for (int j = 0; j < S::NH; ++j) z[j] = 0.f;
  // R = -y of the pixel this lane holds (u^0 = 0)
  auto load_residual = [&]() {
    const float* yrow = p.Y + (valid ? pix : 0) * M;
    bool bad = false;
#pragma unroll
    for (int k = 0; k < S::KW; ++k) {
      const int c0 = S::wc(k) + g * (S::ww(k) / 2);
#pragma unroll
      for (int c = 0; c < S::ww(k) / 2; ++c) {
        const int m = c0 + c;
        const float yv = (valid && m < M) ? __ldg(yrow + m) : 0.f;
        bad |= !isfinite(yv);
        R[S::uo(k) + c] = -yv;
      }
    }
    if (bad) atomicOr(p.status, kStNonFinite);
  };
  {
    load_residual();
    const float zero8[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int q = 0; q < S::Q; ++q)
#pragma unroll
      for (int c = 0; c < S::xw(q) / 2; c += 8)
        tc::tmem_st8(tX + S::xc(q) + g * (S::xw(q) / 2) + c, zero8);
    tc::tmem_wait_st();
  }

  bool done = !valid;
  int k_it = 1;          // the lane's own iteration number (its pixel's x^{k_it - 1} is in TMEM)
  float beta_prev = 0.f;
  uint32_t ph = 0;   // phase parity of the four mbarriers in this iteration
  int ui = 0;        // region holding D (T0 = columns [0, RW), T1 = [RW, 2 RW))
  bool failed = false;

  for (int i = 1;; ++i) {
    const uint32_t tU = tl + ui * S::RW, tO = tl + (1 - ui) * S::RW;
    // ---- residual of the extrapolated point, A z - y = R + beta D with R = u^{i-1} - y
    //      and D = u^{i-1} - u^{i-2}, and Delta_{i-1} = ||D||  (u^0 = 0, D = 0 at i = 1);
    //      operand chunks in buffers 0, 1
    float d2 = 0.f;
#pragma unroll
    for (int k = 0; k < S::KW; ++k) {
      const int half = S::ww(k) / 2, c0 = S::wc(k) + g * half;
      unsigned char* buf = sB + k * kBufBytes;
#pragma unroll
      for (int c2 = 0; c2 < half; c2 += 16) {  // two 8-column blocks per TMEM round trip
        float D[2][8];
        if (i > 1) {
          tc::tmem_ld8(tU + c0 + c2, D[0]);
          if (c2 + 8 < half) tc::tmem_ld8(tU + c0 + c2 + 8, D[1]);
          tc::tmem_wait_ld();
        } else {
#pragma unroll
          for (int e = 0; e < 8; ++e) D[0][e] = D[1][e] = 0.f;
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int c = c2 + 8 * h;
          if (c < half) {
            float v[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              const int j = S::uo(k) + c + e;
              d2 = fmaf(D[h][e], D[h][e], d2);
              R[j] += D[h][e];
              v[e] = fmaf(beta_prev, D[h][e], R[j]);
            }
            put_operand8(buf, kChunk, r, c0 - S::wc(k) + c, v);
          }
        }
      }
    }
    red[g * 128 + r] = d2;
    if (failed) s_fail = 1;
    __syncthreads();
    failed = s_fail != 0;
    const float dtot = red[r] + red[128 + r];
    // x^{k-1} is final if Delta_{k-1} < eps, if the cap is reached, or (eps > 1) at once
    const bool conv_now = !done && k_it > 1 && dtot < p.eps2;
    const bool fin =
        !done && (conv_now || k_it - 1 == p.iters || (k_it == 1 && p.start_done));
    if (__any_sync(0xffffffffu, fin)) {
#pragma unroll
      for (int q = 0; q < S::Q; ++q) {
        const int c0 = S::xc(q) + g * (S::xw(q) / 2);
#pragma unroll
        for (int c = 0; c < S::xw(q) / 2; c += 8) {
          float xv[8];
          tc::tmem_ld8(tX + c0 + c, xv);
          tc::tmem_wait_ld();
          if (fin) {
#pragma unroll
            for (int e = 0; e < 8; ++e)
              if (c0 + c + e < N) p.X[pix * N + c0 + c + e] = xv[e];
          }
        }
      }
      if (fin && g == 0) {
        if (p.iters_out) p.iters_out[pix] = k_it - 1;
        if (p.conv_out) p.conv_out[pix] = conv_now ? 1 : 0;
      }
    }
    // a finished lane takes the next pixel: its group-0 thread claims it for the row, one
    // atomic per warp for all of the warp's finished lanes
    if (g == 0) claim_pixels(fin, p.counter, p.P, s_pix, r, lane);
    done = done || fin;
    tc::fence_async_smem();
    tc::fence_before_sync();
    // a product that never completed ends the solve for the whole tile
    if (!__syncthreads_or(!done || (fin && g == 0 && s_pix[r] >= 0)) || failed) break;
    tc::fence_after_sync();
    // fresh: the lane starts a new pixel; this iteration's products for it are discarded
    // (its increment is 0, so the next D is 0 too, and x and z are then set to 0)
    bool fresh = false;
    if (fin) {
      pix = s_pix[r];
      valid = pix >= 0;
      fresh = valid;
      done = !valid;
    }

    // ---- GEMM2: C = V A in two column halves, half 0 into the free region, half 1 into
    //      the region D was read from (K = MP over the residual's chunks)
    if (tid == 0 && !(p.inject_timeout && i == 1)) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int n0 = h ? S::NA : 0, nh = h ? S::NB : S::NA;
        const uint32_t d = (h ? tmem + ui * S::RW : tmem + (1 - ui) * S::RW);
        const uint32_t idesc = tc::idesc_bf16(128, nh, true);
#pragma unroll
        for (int k = 0; k < S::KW; ++k) {
          const uint32_t boff = (S::wc(k) / 16) * 2 * SD + (n0 / 8) * 128;
          issue_steps(d, uB + k * kBufBytes, uAh + boff, uAl + boff, S::ww(k) / 16, 2 * SD,
                      SD, 128, idesc, k == 0);
        }
        tc::mma_commit(&mb[h]);
      }
    }

    // ---- steps 1-4 chunk by chunk: aux = z - C / L, x = soft(aux, lambda / L), t, z;
    //      x to TMEM and its increment x - x_prev, split, to the ring for GEMM1
    const float beta = p.beta[min(k_it, p.iters > 0 ? p.iters : 1) - 1];
    const bool hold = done || fresh;
#pragma unroll
    for (int q = 0; q < S::Q; ++q) {
      if (q == 0) failed |= !tc::mbar_wait(&mb[0], ph, kWaitLimitNs);
      if (S::needs_c1(q) && (q == 0 || !S::needs_c1(q - 1)))
        failed |= !tc::mbar_wait(&mb[1], ph, kWaitLimitNs);
      if (S::needs_u01(q)) failed |= !tc::mbar_wait(&mb[2], ph, kWaitLimitNs);
      tc::fence_after_sync();
      const int w2 = S::xw(q) / 2, c0 = S::xc(q) + g * w2;
      // C of this chunk: half 0 in the free region, half 1 in D's region
      const uint32_t tC = q < S::Q0 ? tO + c0 : tU + (c0 - S::NA);
      unsigned char* buf = sB + S::xbuf(q) * kBufBytes;
#pragma unroll
      for (int c2 = 0; c2 < w2; c2 += 16) {  // two 8-column blocks per TMEM round trip
        float C[2][8], xp[2][8];
        tc::tmem_ld8(tC + c2, C[0]);
        tc::tmem_ld8(tX + c0 + c2, xp[0]);
        if (c2 + 8 < w2) {
          tc::tmem_ld8(tC + c2 + 8, C[1]);
          tc::tmem_ld8(tX + c0 + c2 + 8, xp[1]);
        }
        tc::tmem_wait_ld();
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int c = c2 + 8 * h;
          if (c < w2) {
            float xn[8], dx[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              const int j = S::zo(q) + c + e;
              float xx = soft_thr(z[j] - C[h][e] * p.invL, p.thr);
              if (!hold) {
                z[j] = xx + beta * (xx - xp[h][e]);
              } else {
                xx = xp[h][e];
              }
              xn[e] = xx;
              dx[e] = xx - xp[h][e];
            }
            tc::tmem_st8(tX + c0 + c, xn);
            put_operand8(buf, kChunk, r, c0 - S::xc(q) + c, dx);
          }
        }
      }
      tc::tmem_wait_st();
      // GEMM1 (D = (X - X_prev) A^T, K = NP): the chunks of half 0 once that half of C is
      // consumed, then each chunk of half 1 as it is written; D accumulates in the free
      // region
      if (q >= S::Q0 - 1) {
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (tid == 0) {
          const uint32_t d = tmem + (1 - ui) * S::RW;
          const uint32_t idesc = tc::idesc_bf16(128, MP, false);
          const int qa = q == S::Q0 - 1 ? 0 : q;
#pragma unroll
          for (int qq = 0; qq < S::Q; ++qq) {
            if (qq < qa || qq > q) continue;
            const uint32_t boff = (S::xc(qq) / 16) * 256;
            issue_steps(d, uB + S::xbuf(qq) * kBufBytes, uAh + boff, uAl + boff,
                        S::xw(qq) / 16, 256, 128, SD, idesc, qq == 0);
          }
          if (q == S::Q0 - 1 && S::NBUF == 3) tc::mma_commit(&mb[2]);
          if (q == S::Q - 1) tc::mma_commit(&mb[3]);
        }
      }
    }
    // a lane starting a new pixel: x = 0 in TMEM and z = 0 (out of the hot loop above;
    // the TMEM stores are warp-wide, so the warp's other lanes write their x back)
    if (__any_sync(0xffffffffu, fresh)) {
#pragma unroll
      for (int q = 0; q < S::Q; ++q) {
        const int c0 = S::xc(q) + g * (S::xw(q) / 2);
#pragma unroll
        for (int c = 0; c < S::xw(q) / 2; c += 8) {
          float xv[8];
          tc::tmem_ld8(tX + c0 + c, xv);
          tc::tmem_wait_ld();
#pragma unroll
          for (int e = 0; e < 8; ++e) xv[e] = fresh ? 0.f : xv[e];
          tc::tmem_st8(tX + c0 + c, xv);
        }
      }
      tc::tmem_wait_st();
      if (fresh) {
#pragma unroll
        for (int j = 0; j < S::NH; ++j) z[j] = 0.f;
      }
    }
    failed |= !tc::mbar_wait(&mb[3], ph, kWaitLimitNs);
    tc::fence_after_sync();
    ph ^= 1u;
    ui = 1 - ui;
    beta_prev = beta;
    ++k_it;
    if (fresh) {  // the new pixel's first iteration comes next
      load_residual();
      k_it = 1;
      beta_prev = 0.f;
    }
  }
  if (__syncthreads_or(failed)) {
    // a product never completed: report, then one commit that tracks every MMA thread 0
    // issued gets a last bounded wait before TMEM is released
    if (tid == 0) {
      atomicOr(p.status, kStTimeout);
      tc::mma_commit(&mb[4]);
    }
    tc::mbar_wait(&mb[4], 0, kWaitLimitNs);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, S::TCOLS);
}

template <int NP, int MP>
cudaError_t run(const Ctx& c, const FtcParams& p) {
  auto kern = k_fista_tc<NP, MP>;
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

// The tile shapes compiled for the tensor-core FISTA: (N, M) padded to 16.
#define CS_FISTA_TC_SHAPES(X) X(128, 48) X(208, 80) X(224, 96) X(256, 112)

}  // namespace

bool fista_tc_supported(int M, int N) {
  const int Mp = (M + 15) / 16 * 16, Np = (N + 15) / 16 * 16;
#define CS_FISTA_TC_MATCH(NP_, MP_) \
  if (Np == NP_ && Mp == MP_) return true;
  CS_FISTA_TC_SHAPES(CS_FISTA_TC_MATCH)
#undef CS_FISTA_TC_MATCH
  return false;
}

cudaError_t launch_fista_tc(const Ctx& c, const ConvexArgs& a) {
  FtcParams p{};
  p.M = c.M;
  p.N = c.N;
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
  p.counter = a.counter ? a.counter : c.conv_counter;
  p.inject_timeout = tc::inject_timeout();
  if (a.P == 0) return cudaSuccess;
  const int Mp = (c.M + 15) / 16 * 16, Np = (c.N + 15) / 16 * 16;
#define CS_FISTA_TC_RUN(NP_, MP_) \
  if (Np == NP_ && Mp == MP_) return run<NP_, MP_>(c, p);
  CS_FISTA_TC_SHAPES(CS_FISTA_TC_RUN)
#undef CS_FISTA_TC_RUN
  return cudaErrorInvalidValue;
}

}  // namespace cs
