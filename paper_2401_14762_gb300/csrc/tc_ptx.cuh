// Thin wrappers around the sm_100-family tensor-core PTX used by the tcgen05 kernels:
// shared-memory matrix descriptors, the kind::f16 instruction descriptor, tcgen05.mma,
// commit to an mbarrier, bounded mbarrier waits, TMEM allocation and 32x32b loads/stores.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>
#include <stdlib.h>

namespace cs {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor, no swizzle.  Operands are stored as 8-row x 16-byte
// core matrices; lbo = byte distance between core matrices adjacent along K, sbo = byte
// distance between core matrices adjacent along M/N (both multiples of 16).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for this architecture family
  return d;
}

// Instruction descriptor of tcgen05.mma kind::f16: BF16 A and B, FP32 accumulation,
// A K-major, B K-major (b_mn = false) or MN-major (b_mn = true), tile M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N, bool b_mn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (0u << 15) | ((b_mn ? 1u : 0u) << 16) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D (TMEM) = A * B^T (+ D if acc), issued by one thread.
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// The mbarrier completes a phase once every tcgen05.mma this thread issued so far is done.
__device__ __forceinline__ void mma_commit(uint64_t* mbar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(mbar)));
}

__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count));
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Fault injection for the tests of the timeout path: with CS_HSI_INJECT_MMA_TIMEOUT=1 in
// the environment, the tensor-core kernels leave out their first product, so its bounded
// wait runs out and the call reports CS_ERR_TIMEOUT without hanging or faulting the GPU.
inline int inject_timeout() {
  const char* v = getenv("CS_HSI_INJECT_MMA_TIMEOUT");
  return v && v[0] == '1' && v[1] == 0;
}

// Waits for the mbarrier phase with the given parity; gives up after limit_ns nanoseconds
// (the caller then reports a timeout instead of hanging the GPU).
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, uint64_t limit_ns) {
  const uint64_t t0 = globaltimer_ns();
  for (;;) {
    uint32_t done = 0;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(mbar)), "r"(parity));
    if (done) return true;
    if (globaltimer_ns() - t0 > limit_ns) return false;
  }
}

__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// TMEM allocation by one full warp; the base address lands in *slot (shared memory).
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(slot)),
               "r"(ncols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}

// 8 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                 "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}
// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const float (&v)[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(
                   taddr),
               "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
               "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
               "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;"); }
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;"); }

// Splits 8 FP32 values into BF16 hi and lo parts (v ~ hi + lo to ~2^-17 relative),
// each packed as 8 consecutive BF16 (16 bytes).
__device__ __forceinline__ void split8(const float (&v)[8], uint4& hi, uint4& lo) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    // packed conversions (round to nearest, element 2j in the low half)
    const __nv_bfloat162 hp = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
    const float2 hf = __bfloat1622float2(hp);
    const __nv_bfloat162 lp = __floats2bfloat162_rn(v[2 * j] - hf.x, v[2 * j + 1] - hf.y);
    h[j] = *reinterpret_cast<const uint32_t*>(&hp);
    l[j] = *reinterpret_cast<const uint32_t*>(&lp);
  }
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// ---- 128-pixel tiles of the convex solvers ----

// A K x N matrix B (row k, column n) in the dual layout: element (k, n) at
// (k/8) S + (n/8) 128 + (k%8) 16 + (n%8) 2, S = 16 Np.  The MMAs read it MN-major as
// the B operand of a product over k (LBO = S, SBO = 128) and K-major as the B operand
// of a product over n, i.e. B^T (LBO = 128, SBO = S).
__device__ __forceinline__ int dual_off(int k, int n, int S) {
  return (k >> 3) * S + (n >> 3) * 128 + (k & 7) * 16 + (n & 7) * 2;
}

// Splits the FP64 matrix B (rows x cols, row-major) into BF16 hi + lo parts stored in the
// dual layout at hi / lo, zero padded to rp x cp; all threads of the block take part.
__device__ __forceinline__ void stage_split(const double* B, int rows, int cols, int rp, int cp,
                                            unsigned char* hi, unsigned char* lo) {
  const int S = 16 * cp;
  for (int e = threadIdx.x; e < rp * cp; e += blockDim.x) {
    int k = e / cp, n = e - k * cp;
    double a = (k < rows && n < cols) ? B[(size_t)k * cols + n] : 0.0;
    __nv_bfloat16 h = __float2bfloat16_rn((float)a);
    __nv_bfloat16 l = __float2bfloat16_rn((float)(a - (double)__bfloat162float(h)));
    *reinterpret_cast<__nv_bfloat16*>(hi + dual_off(k, n, S)) = h;
    *reinterpret_cast<__nv_bfloat16*>(lo + dual_off(k, n, S)) = l;
  }
}

// Writes 8 values of tile row r at columns k0..k0+7 (k0 % 8 == 0) of a K-major 128 x K
// A operand (LBO = 128, SBO = 16 K), hi part at `hi`, lo part at `hi + 256 K`.
__device__ __forceinline__ void put_operand8(unsigned char* hi, int K, int r, int k0,
                                             const float (&v)[8]) {
  uint4 h, l;
  split8(v, h, l);
  int off = (r >> 3) * (K * 16) + (k0 >> 3) * 128 + (r & 7) * 16;
  *reinterpret_cast<uint4*>(hi + off) = h;
  *reinterpret_cast<uint4*>(hi + 256 * K + off) = l;
}

// One product of the tile, issued by one thread: D = O B with the 128 x K operand O at
// o (hi) / o + 256 K (lo) and B at bh / bl, as the three MMAs O_hi B_hi + O_lo B_hi +
// O_hi B_lo (about 16 bits of each operand).  b_mn: B read MN-major (a product over the
// dual layout's k, K-step stride 2 S) or K-major (over its n, K-step stride 256).
__device__ __forceinline__ void split_product(uint32_t d_tmem, uint32_t o, uint32_t bh,
                                              uint32_t bl, int K, int S, bool b_mn,
                                              uint32_t idesc) {
  for (int s = 0; s < K / 16; ++s) {
    uint64_t ah = sdesc(o + s * 256, 128, K * 16);
    uint64_t al = sdesc(o + 256 * K + s * 256, 128, K * 16);
    uint64_t dh = b_mn ? sdesc(bh + s * 2 * S, S, 128) : sdesc(bh + s * 256, 128, S);
    uint64_t dl = b_mn ? sdesc(bl + s * 2 * S, S, 128) : sdesc(bl + s * 256, 128, S);
    mma_bf16(d_tmem, ah, dh, idesc, s > 0 ? 1u : 0u);
    mma_bf16(d_tmem, al, dh, idesc, 1u);
    mma_bf16(d_tmem, ah, dl, idesc, 1u);
  }
}

// sign(a) max(|a| - t, 0) for t >= 0, as a - clamp(a, -t, t): the same value for every
// finite a (a - t and a + t are the rounded |a| - t with a's sign; |a| <= t gives +0),
// in three instructions without a compare.
__device__ __forceinline__ float soft_thr(float a, float t) {
  return a - fminf(fmaxf(a, -t), t);
}

}  // namespace tc
}  // namespace cs
