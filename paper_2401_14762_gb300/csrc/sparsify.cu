// Sparsification pre-processing (Section II): every pixel's spectrum f is taken to the
// transform domain, x = Psi^T f (Psi orthonormal), and the coefficients whose magnitude
// falls short of the pixel's mean magnitude by the margin T sigma are zeroed:
// x_i = 0 where |x_i| - mu < T sigma, mu and sigma the mean and the standard deviation
// of |x| (sigma normalised by N - ddof).  kappa = ||x||_0 of the result.
//
// One warp handles four or eight pixels at a time: their spectra sit in shared memory,
// each lane accumulates its coefficients in FP32 (one float4 of Psi's row n per lane,
// L1/L2 resident), summing blocks of 16 terms by FMA and adding the block sums up; the
// statistics and the decisions follow in FP32.  The decisions must be those of the FP64
// definition, so each one is checked against a rigorous bound: the coefficients' error
// |x~_i - x_i| <= e = (gamma_(16 + ceil(N/16)) + 2u) max_i ||Psi(:, i)|| ||f|| (blocked
// summation, each product rounded once inside its FMA, plus Psi's FP32 rounding;
// Cauchy-Schwarz) moves mu by at most e and sigma by at most e sqrt(N / (N - ddof))
// (sigma is a seminorm of |x|); the FP32 rounding of the sums, of sigma and of the
// margin |x~_i| - mu~ - T sigma~ adds a few units of roundoff of each.  A pixel with a
// margin within its bound is recomputed in FP64, the definition itself.
#include <cuda_runtime.h>

#include "cs_internal.cuh"

namespace cs {
namespace {

constexpr int kSpWarps = 8;
constexpr int kSpBlock = 16;  // terms per FMA block of the transform's sums
constexpr float kU32 = 0x1p-24f;  // FP32 unit roundoff

struct SpParams {
  int N, ddof;
  bool x_vec;           // rows of X may be written as float4s
  const float* Psi32;   // N x 128 ceil(N / 128), Psi[n][i] (column i = atom i), zero padded
  const double* Psi64;  // the same in FP64
  const float* cn;      // column norms of Psi, rounded up
  const float* F;       // P x N spectra
  float* X;             // P x N sparsified coefficients
  int16_t* kappa;       // P, optional
  unsigned long long* recomputed;  // optional, 1 entry: pixels decided in FP64
  int64_t P;
  double T;
  float gam;
  int* status;
};

// FP64 recomputation of one pixel (spectrum f in shared memory): the definition itself.
__device__ __noinline__ void sparsify_fp64(const SpParams& p, const float* f, int64_t pix,
                                           int lane) {
  const int N = p.N;
  double xv[kMaxN / 32];  // this lane's coefficients i = lane, lane + 32, ...
#pragma unroll
  for (int j = 0; j < kMaxN / 32; ++j) xv[j] = 0.0;
  // row by row: each row's loads are independent of the running sums, so they overlap
#pragma unroll 4
  for (int n = 0; n < N; ++n) {
    const double fv = (double)f[n];
    const double* row = p.Psi64 + (size_t)n * N;
#pragma unroll
    for (int j = 0; j < kMaxN / 32; ++j)
      if (lane + 32 * j < N) xv[j] = fma(__ldg(row + lane + 32 * j), fv, xv[j]);
  }
  double s1 = 0.0;
#pragma unroll
  for (int j = 0; j < kMaxN / 32; ++j) s1 += fabs(xv[j]);  // zero past N
  const double mu = warp_sum(s1) / N;
  double s2 = 0.0;
#pragma unroll
  for (int j = 0; j < kMaxN / 32; ++j)
    if (lane + 32 * j < N) s2 += (fabs(xv[j]) - mu) * (fabs(xv[j]) - mu);
  s2 = warp_sum(s2);
  const double sigma = N - p.ddof > 0 ? sqrt(s2 / (N - p.ddof)) : 0.0;
  int nz = 0;
#pragma unroll
  for (int j = 0; j < kMaxN / 32; ++j) {
    const int i = lane + 32 * j;
    if (i < N) {
      const bool keep = !(fabs(xv[j]) - mu < p.T * sigma);
      const float out = keep ? (float)xv[j] : 0.f;
      p.X[pix * N + i] = out;
      nz += keep && xv[j] != 0.0;
    }
  }
  nz = __reduce_add_sync(0xffffffffu, nz);
  if (lane == 0) {
    if (p.kappa) p.kappa[pix] = (int16_t)nz;
    if (p.recomputed) atomicAdd(p.recomputed, 1ull);
  }
}

// Lane l owns the coefficients i = 128 q + 4 l + c (c < 4, q < NQ = ceil(N / 128)), so
// each row of the padded FP32 Psi is read as one float4 per lane and q.
template <int NQ, int kSpPix>
__global__ void __launch_bounds__(kSpWarps * 32, 2) k_sparsify(SpParams p) {
  constexpr int S = 4 * NQ;  // coefficient slots per lane
  extern __shared__ float fsm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, N = p.N, ldp = 128 * NQ;
  float* fw = fsm + (size_t)warp * kSpPix * N;
  // the largest column norm of Psi (1 for an orthonormal Psi), rounded up
  float cnmax = 0.f;
  for (int i = lane; i < N; i += 32) cnmax = fmaxf(cnmax, p.cn[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cnmax = fmaxf(cnmax, __shfl_xor_sync(0xffffffffu, cnmax, o));
  const float denom = N - p.ddof > 0 ? (float)(N - p.ddof) : 0.f;
  const float rN = denom > 0.f ? sqrtf((float)N / denom) * (1.f + 1e-6f) : 0.f;
  const float T = (float)p.T, Tabs = fabsf(T);
  const int64_t groups = (p.P + kSpPix - 1) / kSpPix;
  for (int64_t g = (int64_t)blockIdx.x * kSpWarps + warp; g < groups;
       g += (int64_t)gridDim.x * kSpWarps) {
    const int64_t pix0 = g * kSpPix;
    const int np = p.P - pix0 < kSpPix ? (int)(p.P - pix0) : kSpPix;
    float fn2[kSpPix];
    bool bad = false;
#pragma unroll
    for (int i = 0; i < kSpPix; ++i) {
      float ss = 0.f;
      for (int n = lane; n < N; n += 32) {
        const float v = i < np ? p.F[(pix0 + i) * N + n] : 0.f;
        bad |= !isfinite(v);
        fw[i * N + n] = v;
        ss = fmaf(v, v, ss);
      }
      fn2[i] = warp_sum(ss);
    }
    if (bad) atomicOr(p.status, kStNonFinite);
    __syncwarp();
    float acc[kSpPix][S];
#pragma unroll
    for (int i = 0; i < kSpPix; ++i)
#pragma unroll
      for (int s = 0; s < S; ++s) acc[i][s] = 0.f;
    // Psi's row n + 1 is requested before row n's products (one row of lookahead)
    const float4* prow = reinterpret_cast<const float4*>(p.Psi32) + lane;
    float4 nx[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) nx[q] = __ldg(prow + 32 * q);
    for (int n0 = 0; n0 < N; n0 += kSpBlock) {
      float part[kSpPix][S];
#pragma unroll
      for (int i = 0; i < kSpPix; ++i)
#pragma unroll
        for (int s = 0; s < S; ++s) part[i][s] = 0.f;
      const int n1 = min(n0 + kSpBlock, N);
      for (int n = n0; n < n1; ++n) {
        float ps[S];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          ps[4 * q] = nx[q].x;
          ps[4 * q + 1] = nx[q].y;
          ps[4 * q + 2] = nx[q].z;
          ps[4 * q + 3] = nx[q].w;
        }
        if (n + 1 < N) {
#pragma unroll
          for (int q = 0; q < NQ; ++q) nx[q] = __ldg(prow + (size_t)(n + 1) * (ldp / 4) + 32 * q);
        }
#pragma unroll
        for (int i = 0; i < kSpPix; ++i) {
          const float fv = fw[i * N + n];
#pragma unroll
          for (int s = 0; s < S; ++s) part[i][s] = fmaf(ps[s], fv, part[i][s]);
        }
      }
#pragma unroll
      for (int i = 0; i < kSpPix; ++i)
#pragma unroll
        for (int s = 0; s < S; ++s) acc[i][s] += part[i][s];
    }
#pragma unroll
    for (int i = 0; i < kSpPix; ++i) {
      if (i >= np) break;  // warp-uniform
      const int64_t pix = pix0 + i;
      // statistics in FP32 (padding slots hold exact zeros and are left out)
      float s1 = 0.f;
#pragma unroll
      for (int s = 0; s < S; ++s)
        if (128 * (s >> 2) + 4 * lane + (s & 3) < N) s1 += fabsf(acc[i][s]);
      const float mu = warp_sum(s1) / (float)N;
      float s2 = 0.f;
#pragma unroll
      for (int s = 0; s < S; ++s)
        if (128 * (s >> 2) + 4 * lane + (s & 3) < N) {
          const float d = fabsf(acc[i][s]) - mu;
          s2 = fmaf(d, d, s2);
        }
      const float sig = denom > 0.f ? sqrtf(warp_sum(s2) / denom) : 0.f;
      // bounds: e on each FP32 coefficient; its effect on mu (mean e) and sigma
      // (||e|| / sqrt(N - ddof)); the FP32 rounding of the two sums (at most S + 5 and
      // S + 7 roundings through the lane sums and the butterfly, plus the divide and the
      // square root) and of the margin itself (three operations)
      const float e = p.gam * cnmax * sqrtf(fn2[i] * (1.f + 64.f * kU32));
      const float dmu = (S + 8) * kU32 * mu;
      const float dsig = (S + 12) * kU32 * sig + rN * dmu;
      const float thr = T * sig;
      const float slack = e + Tabs * e * rN + dmu + Tabs * dsig;
      bool amb = false;
      unsigned keep = 0;
      int nz = 0;
#pragma unroll
      for (int s = 0; s < S; ++s) {
        if (128 * (s >> 2) + 4 * lane + (s & 3) < N) {
          const float a = fabsf(acc[i][s]);
          const float m = (a - mu) - thr;
          const float b = (e + slack + 4.f * kU32 * (a + mu + fabsf(thr))) * 1.01f;
          amb |= !(fabsf(m) > b);
          if (m >= 0.f) {
            keep |= 1u << s;
            nz += acc[i][s] != 0.f;
          }
        }
      }
      if (__any_sync(0xffffffffu, amb)) {
        sparsify_fp64(p, fw + i * N, pix, lane);
        continue;
      }
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const int i0 = 128 * q + 4 * lane;
        float o[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) o[c] = (keep >> (4 * q + c)) & 1u ? acc[i][4 * q + c] : 0.f;
        if (p.x_vec) {  // N % 4 == 0 and X 16-byte aligned: whole float4s
          if (i0 < N) *reinterpret_cast<float4*>(p.X + pix * N + i0) = make_float4(o[0], o[1], o[2], o[3]);
        } else {
#pragma unroll
          for (int c = 0; c < 4; ++c)
            if (i0 + c < N) p.X[pix * N + i0 + c] = o[c];
        }
      }
      nz = __reduce_add_sync(0xffffffffu, nz);
      if (lane == 0 && p.kappa) p.kappa[pix] = (int16_t)nz;
    }
    __syncwarp();  // fw is rewritten by the next pass
  }
}

template <int NQ>
cudaError_t run_sparsify(const Ctx& c, const SpParams& p) {
  constexpr int kSpPix = NQ == 1 ? 8 : 4;  // accumulators: 2 x 32 registers either way
  const size_t smem = sizeof(float) * kSpWarps * kSpPix * (size_t)p.N;
  auto kern = k_sparsify<NQ, kSpPix>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kSpWarps * 32, smem);
  const int64_t groups = (p.P + kSpPix - 1) / kSpPix;
  int64_t grid = (int64_t)c.num_sms * (per_sm > 0 ? per_sm : 1);
  const int64_t need = (groups + kSpWarps - 1) / kSpWarps;
  if (grid > need) grid = need;
  kern<<<(unsigned)grid, kSpWarps * 32, smem, c.stream>>>(p);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sparsify(const Ctx& c, const float* F, float* X, int64_t P, double T,
                            int ddof, int16_t* kappa, unsigned long long* recomputed) {
  if (P == 0) return cudaSuccess;
  SpParams p{};
  p.N = c.N;
  p.ddof = ddof;
  p.Psi32 = c.Psi32;
  p.Psi64 = c.Psi64;
  p.cn = c.psi_cn;
  p.F = F;
  p.X = X;
  p.x_vec = (c.N & 3) == 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0;
  p.kappa = kappa;
  p.recomputed = recomputed;
  p.P = P;
  p.T = T;
  // gamma_k = k u / (1 - k u) for the k = 16 + ceil(N / 16) roundings a blocked sum
  // carries at most, plus 2u for Psi's FP32 rounding
  const double u = 0x1p-24;
  const int k = kSpBlock + (c.N + kSpBlock - 1) / kSpBlock;
  p.gam = (float)((k * u / (1.0 - k * u) + 2.0 * u) * (1.0 + 1e-6));
  p.status = c.status;
  return c.N <= 128 ? run_sparsify<1>(c, p) : run_sparsify<2>(c, p);
}

}  // namespace cs
