// Internal declarations shared by the translation units of libcs_hsi.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "cs_hsi.h"

namespace cs {

// Bits of the per-context device status word (atomicOr'ed by kernels).
enum : int {
  kStNonFinite = 1 << 0,
  kStNotSpd = 1 << 1,
  kStTimeout = 1 << 2,
};

constexpr int kMaxM = 128;
constexpr int kMaxN = 256;

// Padded leading dimension (in floats) for a row of `n` floats kept in shared memory:
// at least n rounded up to 4, and == 4 (mod 8) so that eight lanes reading float4s
// from eight consecutive rows at the same column hit 32 distinct banks.
inline int smem_ld(int n) {
  int ld = (n + 3) & ~3;
  while ((ld & 7) != 4) ld += 4;
  return ld;
}

// A launch configuration of the greedy kernel measured best by the autotuner
// (cs_autotune) for one algorithm and its (kappa bound, G): the rows of the FP32 factor
// kept in shared memory (gOMP; the others need their whole support) and the warps per
// CTA (the CTAs per SM follow from the shared memory they take).
struct GreedyTune {
  bool valid = false;
  int kappa = 0, G = 0;
  int d32 = 0, warps = 0;
  double ms = 0.0, ms_default = 0.0;
};

struct Ctx {
  int M = 0, N = 0, device = 0, num_sms = 0;
  GreedyTune tune[3];  // per greedy algorithm (gOMP, BIHT, CoSaMP)
  // cs_create_complex: A is the real form of a complex dictionary and every vector holds
  // complex values as (re, im) pairs; FISTA's and ADMM's thresholds act on the moduli
  bool complex_pairs = false;
  cudaStream_t stream = nullptr;
  cs_precision last_prec = CS_FP32;  // the arithmetic of the last recovery call's products
  double L = 0.0;             // Lipschitz constant lambda_max(A^T A)
  double* A64 = nullptr;      // M x N, FP64
  double* At64 = nullptr;     // N x M, FP64 (column j of A contiguous)
  double* G64 = nullptr;      // N x N, FP64 Gram A^T A
  float* G32 = nullptr;       // N x N, its FP32 rounding (factor gathers)
  float* A32 = nullptr;       // M x N, FP32
  float* At32 = nullptr;      // N x M, FP32
  double rho = 0.0;           // penalty of the cached ADMM factor
  float* W32 = nullptr;       // M x M, FP32 (A A^T + rho I)^{-1}
  double* W64 = nullptr;      // M x M, the same in FP64 (split for the tensor cores)
  float* Wpad = nullptr;      // M x smem_ld(M), the FP32 factor with zero-padded rows
  double* Psi64 = nullptr;    // N x N transform Psi (contexts made from Phi; else NULL)
  float* Psi32 = nullptr;     // its FP32 rounding, rows zero padded to 128 ceil(N / 128)
  float* psi_cn = nullptr;    // column norms of Psi, rounded up to FP32
  double* scratch64 = nullptr;  // setup scratch
  size_t scratch_elems = 0;
  int* status = nullptr;      // device status word
  int* counter = nullptr;     // work counter of the persistent greedy kernel
  // pixel counters of the persistent tensor-core FISTA/ADMM launches: slot 0 for single
  // calls, one per chunk buffer of streamed calls and one per cube of convex batches
  // (launches that may run at the same time need their own)
  unsigned long long* conv_counter = nullptr;
  int conv_counter_cap = 0;
  double* fb64 = nullptr;     // per-warp FP64 fallback slots of the greedy kernel
  double* work = nullptr;     // algorithmic flops of the last greedy call (device, 1 entry)
  float* beta = nullptr;      // FISTA momentum weights (device), capacity beta_cap
  int beta_cap = 0;
  int beta_valid = 0;         // leading entries of beta already computed
  // tables outgrown by a longer call: kept until the context is destroyed, so that a
  // graph captured while one of them was current still reads valid memory
  std::vector<float*> beta_retired;
  void* cube_table = nullptr; // greedy launches' cube descriptors (device), cube_cap entries
  int cube_cap = 0;
  size_t fb64_elems = 0;
  float* stage_in = nullptr;  // staging for host-pointer calls
  float* stage_out = nullptr;
  float* stage_aux = nullptr;
  size_t stage_in_bytes = 0, stage_out_bytes = 0, stage_aux_bytes = 0;
  // fork-join streams of multi-cube FISTA/ADMM batches (created by the first such batch):
  // ev_fork orders them after the context stream, ev_join[k] orders it after aux[k]
  static constexpr int kAux = 4;
  cudaStream_t aux[kAux] = {};
  cudaEvent_t ev_fork = nullptr, ev_join[kAux] = {};
  // double-buffered staging of streamed (pushbroom) recoveries: chunk buffers of
  // pipe_cap pixels and the events of their copy-in, compute and copy-out
  float* pipe_y[2] = {};
  float* pipe_x[2] = {};
  int64_t pipe_cap = 0;
  cudaEvent_t ev_in[2] = {}, ev_comp[2] = {}, ev_out[2] = {};
};

void set_error(const std::string& msg);
cs_status cuda_fail(cudaError_t e, const char* what);

// ---- setup (FP64, one-off) ----
cudaError_t setup_dictionary(Ctx& c, const double* A_host, const double* Phi_host,
                             const double* Psi_host);
cudaError_t setup_admm_factor(Ctx& c, double rho);

// ---- measurement ----
cudaError_t launch_measure(const Ctx& c, const float* X, float* Y, const float* E, int64_t P);

// ---- sparsification pre-processing (Section II) ----
cudaError_t launch_sparsify(const Ctx& c, const float* F, float* X, int64_t P, double T,
                            int ddof, int16_t* kappa, unsigned long long* recomputed);

// ---- convex (FISTA / ADMM) ----
struct ConvexArgs {
  const float* Y;
  float* X;
  int64_t P;
  double lambda;
  double rho;
  double eps;
  int iters;
  int32_t* iters_out;
  uint8_t* conv_out;
  cs_precision prec;
  unsigned long long* counter = nullptr;  // tensor-core pixel counter (null: the context's slot 0)
};
// FISTA's momentum weights beta_i (i = 1..iters) into c.beta, on c.stream (only the
// first time a context needs that many: the table of a shorter run is a prefix)
cudaError_t momentum_table(Ctx& c, int iters);
// table = false: c.beta already holds at least a.iters weights (batches write it once)
cudaError_t launch_fista(Ctx& c, const ConvexArgs& a, bool table = true);
bool fista_tc_supported(int M, int N);
cudaError_t launch_fista_tc(const Ctx& c, const ConvexArgs& a);
cudaError_t launch_admm(Ctx& c, const ConvexArgs& a);
// at least n pixel-counter slots in c.conv_counter
cudaError_t ensure_conv_counters(Ctx& c, int n);
bool admm_tc_supported(int M, int N);
cudaError_t launch_admm_tc(const Ctx& c, const ConvexArgs& a);

// ---- greedy (gOMP / BIHT / CoSaMP) ----
enum GreedyAlgo { kGomp = 0, kBiht = 1, kCosamp = 2 };
struct GreedyArgs {
  const float* Y;
  float* X;
  int64_t P;
  int kappa;
  int G;  // gOMP atoms per iteration (0 = per-pixel rule from kappa_pp)
  double mu;
  double eps;
  int max_iters;
  const int16_t* kappa_pp;
  int kappa_max;  // upper bound of kappa over all pixels
  int32_t* iters_out;
  uint8_t* conv_out;
  cs_precision prec;
  bool cycle_skip;  // BIHT/CoSaMP: stop at a repeated iterate (exact, see k_greedy)
};
cudaError_t launch_greedy(Ctx& c, GreedyAlgo algo, const GreedyArgs& a);
// Times the kernel's launch configurations on the sample a.Y (a.X receives its output)
// and keeps the fastest in c.tune[algo]; *out gets it and the default's time.
cudaError_t tune_greedy(Ctx& c, GreedyAlgo algo, const GreedyArgs& a, GreedyTune* out);
// One cube of a batched greedy launch (device pointers; Y/X/kappa/iters/conv per cube).
struct GreedyCube {
  const Ctx* ctx;
  const float* Y;
  float* X;
  int64_t P;
  const int16_t* kappa_pp;
  int32_t* iters_out;
  uint8_t* conv_out;
};
// All cubes in one persistent launch on c0's stream (its counter, status and slots);
// a's Y, X, P and per-pixel pointers are unused.
cudaError_t launch_greedy_batch(Ctx& c0, GreedyAlgo algo, const GreedyCube* cubes, int n,
                                const GreedyArgs& a);

// ---- allocation-free gOMP (scratch in a static device array) ----
size_t noalloc_scratch_bytes(int M, int N);
size_t noalloc_scratch_capacity();
cudaError_t launch_gomp_noalloc(const double* A64, int M, int N, const GreedyArgs& a,
                                cudaStream_t stream);

// ---- warp helpers ----
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace cs
