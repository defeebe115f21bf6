// Greedy recovery: gOMP (Algorithm 3), BIHT (Algorithm 4) and CoSaMP (Algorithm 5).
//
// One warp recovers one pixel at a time and takes the next pixel from a global work
// counter when it finishes, so pixels that stop early (Delta < eps) free their warp at
// once; a launch may cover several cubes (each with its own dictionary, found through a
// table of cube descriptors), counted as one run of pixels.  Per iteration the warp
//   1. correlates: p = A^T r = A^T y - (A^T A)_{:,q} x_q (FP32, lane l owns atoms l, l+32,
//      ...; A^T y once per pixel, then |q| <= kappa columns of the Gram matrix instead of
//      the M rows of A), for BIHT u = x + mu p,
//   2. selects the G / 2 kappa / kappa largest magnitudes (ties to the lower atom):
//      warp argmax rounds for small k, a 32-step radix search on the magnitude bits for
//      large k; the choice is then certified against FP64: atoms whose FP32 value lies
//      within the FP32 error bound of the cut are recomputed in FP64 and ranked exactly,
//      so every selection is the one FP64 arithmetic makes,
//   3. forms the support c (union of Theta with c or supp(x)): sorted by atom for BIHT
//      and CoSaMP, in order of arrival for gOMP, whose support only grows,
//   4. solves min ||A_c s - y|| through the normal equations G_c s = (A^T y)_c: G_c is
//      gathered from the precomputed Gram matrix A^T A, factored in FP32 (gOMP extends
//      its factor by the rows of the atoms just added instead of refactoring), and the
//      solution is refined to FP64 accuracy with FP64 residuals (an FP64 factorisation
//      is the fallback); (A^T y)_j in FP64 is formed when atom j first enters a support;
//      when |c| > M the minimum-norm solution s = A_c^T (A_c A_c^T)^{-1} y is used,
//   5. prunes to kappa atoms by rank counting on the refined coefficients (and, for
//      gOMP, refits on them, keeping the factor rows of the kept atoms' unchanged
//      prefix from the previous refit),
//   6. recomputes the residual r = y - A x in FP32 and decides Delta = ||r - r_prev|| <
//      eps with the FP32 error bound of r: an unchanged iterate gives Delta = 0 exactly,
//      and a Delta too close to eps for the bound is recomputed in FP64 from the change
//      of x (the paper's absolute eps = 1e-8 lies below FP32 resolution of r).
// FP64 arithmetic is left to the least squares' residuals and right-hand sides and to
// the rare cases that need it (a certification band, an ambiguous Delta, a failed FP32
// factor): the correlation and the residual run in FP32.  On GB300 an FP64 warp
// instruction occupies its scheduler's FP64 pipe for about 76 cycles however many lanes
// are active, so the FP64 loops carry no padding and systems of up to 32 rows take
// one register slot per lane.
// Every step is deterministic and a support keeps its order, so an unchanged support
// reproduces x bit for bit and Delta = 0 exactly, as in the paper's stopping rule; for the
// same reason BIHT and CoSaMP may stop at a repeated iterate (the rest of the run is
// periodic) and report the cap.  All per-pixel state sits in the warp's slice of shared
// memory.
#include <cuda_runtime.h>

#include <mutex>
#include <vector>

#include "cs_internal.cuh"
#include "greedy_kernel.cuh"

namespace cs {

namespace {

// Cube entries reach the device table through kernel parameters (32 per launch), so a
// call copies from no host memory and can be captured in a CUDA graph.
constexpr int kCubesPerPut = 32;
struct CubeBlock {
  GrCube c[kCubesPerPut];
  int n;
};
__global__ void k_put_cubes(CubeBlock b, GrCube* dst) {
  if ((int)threadIdx.x < b.n) dst[threadIdx.x] = b.c[threadIdx.x];
}
cudaError_t put_cubes(const GrCube* host, int n, GrCube* dst, cudaStream_t s) {
  for (int i0 = 0; i0 < n; i0 += kCubesPerPut) {
    CubeBlock b{};
    b.n = n - i0 < kCubesPerPut ? n - i0 : kCubesPerPut;
    for (int i = 0; i < b.n; ++i) b.c[i] = host[i0 + i];
    k_put_cubes<<<1, kCubesPerPut, 0, s>>>(b, dst + i0);
  }
  return cudaGetLastError();
}

// Every launch of a greedy kernel instance may use up to the device's opt-in maximum of
// dynamic shared memory: the attribute is set once per (device, instance), under a
// lock, so launches from several host threads (context calls and the allocation-free
// call) never change it under one another.
std::mutex g_attr_mu;
std::vector<std::pair<int, const void*>> g_attr_done;
cudaError_t allow_full_smem(const void* kern) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_attr_mu);
  for (const auto& d : g_attr_done)
    if (d.first == dev && d.second == kern) return cudaSuccess;
  int mx = 0;
  e = cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  if (e == cudaSuccess) g_attr_done.emplace_back(dev, kern);
  return e;
}

GrCube cube_of(const Ctx& c, const float* Y, float* X, int64_t P, const int16_t* kappa_pp,
               int32_t* iters_out, uint8_t* conv_out, int64_t pix0) {
  GrCube g{};
  g.M = c.M;
  g.N = c.N;
  g.A32 = c.A32;
  g.At32 = c.At32;
  g.At64 = c.At64;
  g.G32 = c.G32;
  g.G64 = c.G64;
  g.Y = Y;
  g.X = X;
  g.P = P;
  g.pix0 = pix0;
  g.kappa_pp = kappa_pp;
  g.iters_out = iters_out;
  g.conv_out = conv_out;
  return g;
}

// Support capacities of a launch (cmax atoms in c, dmax rows of an FP32 factor, kmax
// kept atoms) for cubes of at most Mmax measurements and Nmax atoms.
void capacities(GrParams& p, GreedyAlgo algo, const GreedyArgs& a, int Mmax, int Nmax) {
  const int K = a.kappa_max;
  int cmax;
  if (algo == kGomp) {
    int gmax = a.G > 0 ? a.G : (K / 5 > 1 ? K / 5 : 1);
    int iters = a.max_iters < K ? a.max_iters : K;
    long long cm = (long long)gmax * (iters > 0 ? iters : 1);
    cmax = (int)(cm < Mmax ? cm : Mmax);
    if (a.G == 0) cmax = Mmax;  // per-pixel G: bound by M
  } else if (algo == kCosamp) {
    cmax = 3 * K < Nmax ? 3 * K : Nmax;
  } else {
    cmax = 2 * K < Nmax ? 2 * K : Nmax;
  }
  if (cmax < 1) cmax = 1;
  p.cmax = cmax;
  p.dmax = cmax < Mmax ? cmax : Mmax;
  p.d32 = p.dmax;
  p.kmax = K > 0 ? K : 1;
  int sel = p.kmax;
  if (algo == kCosamp) sel = 2 * p.kmax;
  if (algo == kGomp) {
    const int gmax = a.G > 0 ? a.G : (K / 5 > 1 ? K / 5 : 1);
    if (gmax > sel) sel = gmax;
  }
  p.selmax = sel;
}

void scalars(GrParams& p, GreedyAlgo algo, const GreedyArgs& a) {
  p.algo = algo;
  p.kappa = a.kappa;
  p.G = a.G;
  p.mu = (float)a.mu;
  p.mu64 = a.mu;
  p.eps2 = a.eps * a.eps;
  p.start_done = a.eps > 1.0;
  p.max_iters = a.max_iters;
  p.cycle_skip = a.cycle_skip ? 1 : 0;
}

// One persistent launch over the cubes host[0..n) (ascending pix0, total pixels), on the
// context's stream, with its counter, work word, status word and fallback slots.
cudaError_t run_greedy(Ctx& c, GreedyAlgo algo, const GreedyArgs& a, const GrCube* host, int n,
                       int Mmax, int Nmax, int64_t total, bool pairs = false) {
  if (c.cube_cap < n) {
    cudaFree(c.cube_table);
    c.cube_table = nullptr;
    c.cube_cap = 0;
    cudaError_t ea = cudaMalloc(&c.cube_table, sizeof(GrCube) * (size_t)n);
    if (ea != cudaSuccess) return ea;
    c.cube_cap = n;
  }
  GrCube* table = static_cast<GrCube*>(c.cube_table);
  cudaError_t e = put_cubes(host, n, table, c.stream);
  if (e != cudaSuccess) return e;
  GrParams p{};
  scalars(p, algo, a);
  p.Mmax = Mmax;
  p.Nmax = Nmax;
  p.cubes = table;
  p.ncubes = n;
  p.total = total;
  p.status = c.status;
  p.counter = reinterpret_cast<unsigned long long*>(c.counter);
  p.work = c.work;
  if (pairs) {
    // complex data on the real form: capacities in complex atoms, workspaces in columns
    capacities(p, algo, a, Mmax / 2, Nmax / 2);
    p.cmax *= 2;
    p.kmax *= 2;
    p.dmax = p.cmax < Mmax ? p.cmax : Mmax;
    p.d32 = p.dmax;
  } else {
    capacities(p, algo, a, Mmax, Nmax);
  }
  // FP32 factors in shared memory; the rare FP64 fallback (and the |c| > M minimum-norm
  // solve) use one global slot per resident warp, so more warps fit on an SM.
  if (algo == kGomp) {
    // gOMP's support grows by G atoms per iteration up to dmax, but its residual usually
    // stops changing before the support reaches twice kappa: the FP32 factor in shared
    // memory holds at most 64 rows (two register slots per lane), fewer if that seats 16
    // warps per SM, but never fewer than 2 kappa; a support that outgrows it is solved by
    // the FP64 factorisation in the warp's global slot.
    const int lo = 2 * p.kmax < p.dmax ? 2 * p.kmax : p.dmax;
    int d = p.dmax < 64 ? p.dmax : 64;
    while (d > lo && Layout(Mmax, Nmax, p.cmax, p.dmax, p.kmax, p.selmax, false, true, false,
                            false, d, pairs).total * 8 > 110 * 1024)
      --d;
    p.d32 = d > lo ? d : lo;
  }
  // a configuration the autotuner chose for this call's parameters (single cubes)
  const GreedyTune& tn = c.tune[algo];
  const bool tuned = n == 1 && !pairs && tn.valid && tn.kappa == a.kappa_max && tn.G == a.G;
  if (tuned && algo == kGomp) {
    const int lo = 2 * p.kmax < p.dmax ? 2 * p.kmax : p.dmax;
    p.d32 = tn.d32 < lo ? lo : (tn.d32 > p.dmax ? p.dmax : tn.d32);
  }
  Layout lay(Mmax, Nmax, p.cmax, p.dmax, p.kmax, p.selmax, false, algo == kGomp,
             algo != kGomp, algo == kBiht, p.d32, pairs);
  p.warp_bytes = lay.total;
  // one CTA of up to 8 warps per SM, or two smaller ones if that seats more warps
  int warps1 = (220 * 1024) / lay.total, warps2 = (110 * 1024) / lay.total;
  if (warps1 > 8) warps1 = 8;
  if (warps2 > 8) warps2 = 8;
  int warps = (warps2 >= 1 && 2 * warps2 >= warps1) ? warps2 : warps1;
  if (tuned && tn.warps >= 1 && tn.warps <= 8 && (size_t)tn.warps * lay.total <= 220 * 1024)
    warps = tn.warps;
  if (warps < 1) warps = 1;
  if ((size_t)warps * lay.total > 220 * 1024) return cudaErrorInvalidConfiguration;
  size_t smem = (size_t)warps * lay.total;
  e = cudaMemsetAsync(c.counter, 0, sizeof(unsigned long long), c.stream);
  if (e == cudaSuccess && c.work) e = cudaMemsetAsync(c.work, 0, sizeof(double), c.stream);
  if (e != cudaSuccess) return e;
  auto launch = [&](auto kern) {
    cudaError_t ea = allow_full_smem(reinterpret_cast<const void*>(kern));
    if (ea != cudaSuccess) return ea;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, warps * 32, smem);
    if (per_sm < 1) per_sm = 1;
    long long grid = (long long)c.num_sms * per_sm;
    long long need = (total + warps - 1) / warps;
    if (grid > need) grid = need;
    const int D = p.dmax;
    p.fb_slot = D * (D + 1) / 2 + 3 * D;
    size_t elems = (size_t)grid * warps * p.fb_slot;
    if (c.fb64_elems < elems) {
      cudaFree(c.fb64);
      c.fb64 = nullptr;
      c.fb64_elems = 0;
      cudaError_t ea = cudaMalloc(reinterpret_cast<void**>(&c.fb64), sizeof(double) * elems);
      if (ea != cudaSuccess) return ea;
      c.fb64_elems = elems;
    }
    p.fb64 = c.fb64;
    kern<<<(unsigned)grid, warps * 32, smem, c.stream>>>(p);
    return cudaGetLastError();
  };
  // register slots of the FP32 factor: rows up to d32 (gOMP's refit on q: up to kmax)
  const int rows = p.d32 > p.kmax ? p.d32 : p.kmax;
  const int vr = ((rows < p.dmax ? rows : p.dmax) + 31) / 32;
  if (pairs)  // compiled in greedy_pairs.cu
    return launch(reinterpret_cast<void (*)(GrParams)>(
        const_cast<void*>(greedy_pairs_kernel(algo, vr))));
  if (algo == kGomp) return launch(greedy_kernel<kGomp>(vr));
  if (algo == kBiht) return launch(greedy_kernel<kBiht>(vr));
  return launch(greedy_kernel<kCosamp>(vr));
}

}  // namespace

cudaError_t launch_greedy(Ctx& c, GreedyAlgo algo, const GreedyArgs& a) {
  c.last_prec = CS_FP32;
  if (a.P == 0) return cudaSuccess;
  GrCube cube = cube_of(c, a.Y, a.X, a.P, a.kappa_pp, a.iters_out, a.conv_out, 0);
  return run_greedy(c, algo, a, &cube, 1, c.M, c.N, a.P, c.complex_pairs);
}

cudaError_t tune_greedy(Ctx& c, GreedyAlgo algo, const GreedyArgs& a, GreedyTune* out) {
  if (a.P < 1) return cudaErrorInvalidValue;
  GrParams p{};
  capacities(p, algo, a, c.M, c.N);
  const int lo = 2 * p.kmax < p.dmax ? 2 * p.kmax : p.dmax;
  // candidate factor capacities (gOMP: from 2 kappa to the whole support in steps of 8;
  // the others hold their whole support) and warps per CTA
  std::vector<int> caps;
  if (algo == kGomp) {
    for (int d = lo; d < p.dmax; d += 8) caps.push_back(d);
    caps.push_back(p.dmax);
  } else {
    caps.push_back(p.dmax);
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  auto timed = [&](float* ms) {
    cudaError_t er = cudaEventRecord(e0, c.stream);
    if (er == cudaSuccess) er = launch_greedy(c, algo, a);
    if (er == cudaSuccess) er = cudaEventRecord(e1, c.stream);
    if (er == cudaSuccess) er = cudaEventSynchronize(e1);
    if (er == cudaSuccess) er = cudaEventElapsedTime(ms, e0, e1);
    return er;
  };
  GreedyTune best;
  float ms_def = 0.f;
  c.tune[algo].valid = false;
  if (e == cudaSuccess) e = launch_greedy(c, algo, a);  // warm-up (and workspace sizing)
  if (e == cudaSuccess) e = timed(&ms_def);
  for (size_t ic = 0; ic < caps.size() && e == cudaSuccess; ++ic) {
    const Layout lay(c.M, c.N, p.cmax, p.dmax, p.kmax, p.selmax, false, algo == kGomp,
                     algo != kGomp, algo == kBiht, caps[ic]);
    for (int wp = 2; wp <= 8 && e == cudaSuccess; ++wp) {
      if ((size_t)wp * lay.total > 220 * 1024) break;
      GreedyTune t;
      t.valid = true;
      t.kappa = a.kappa_max;
      t.G = a.G;
      t.d32 = caps[ic];
      t.warps = wp;
      c.tune[algo] = t;
      float ms = 0.f;
      e = timed(&ms);
      if (e == cudaSuccess && (!best.valid || ms < best.ms)) {
        best = t;
        best.ms = ms;
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) {
    c.tune[algo].valid = false;
    return e;
  }
  best.ms_default = ms_def;
  // keep the default when no candidate beats it
  if (!best.valid || best.ms >= ms_def) best.valid = false;
  c.tune[algo] = best;
  *out = best;
  out->ms_default = ms_def;
  if (!best.valid) out->ms = ms_def;
  return cudaSuccess;
}

cudaError_t launch_greedy_batch(Ctx& c0, GreedyAlgo algo, const GreedyCube* cubes, int n,
                                const GreedyArgs& a) {
  std::vector<GrCube> host;
  host.reserve(n);
  int64_t total = 0;
  int Mmax = 1, Nmax = 1;
  for (int i = 0; i < n; ++i) {
    const GreedyCube& g = cubes[i];
    if (g.P == 0) continue;
    host.push_back(cube_of(*g.ctx, g.Y, g.X, g.P, g.kappa_pp, g.iters_out, g.conv_out, total));
    total += g.P;
    if (g.ctx->M > Mmax) Mmax = g.ctx->M;
    if (g.ctx->N > Nmax) Nmax = g.ctx->N;
  }
  if (total == 0) return cudaSuccess;
  // the caller checked that the cubes are all complex (column pairs) or all real
  return run_greedy(c0, algo, a, host.data(), (int)host.size(), Mmax, Nmax, total,
                    c0.complex_pairs);
}

}  // namespace cs

// ---------------------------------------------------------------------------------
// Allocation-free gOMP (cs_recover_gomp_noalloc).
//
// Some callers cannot call cudaMalloc when they recover a cube: code that runs with
// all device memory already handed to its own pool, or in a phase where the
// device-wide synchronisation of cudaMalloc/cudaFree is not acceptable.  They pass
// the FP64 dictionary, the measurements and the output (their own device memory);
// everything else the gOMP kernel reads -- the FP32 copy of A, its transpose in FP32 and
// FP64, the Gram matrix A^T A in FP32 and FP64, the work counter and a status word --
// lives in the file-scope array below, which every GPU that loads this library holds
// until exit (2 MiB; every shape the library accepts, M <= 128 and N <= 256, fits).
// Each call re-derives that data, so all calls share one scratch: calls that overlap
// on the GPU (different streams, different host threads) race and must be ordered by
// the caller.
// ---------------------------------------------------------------------------------
constexpr size_t kNoAllocScratchBytes = (size_t)2 << 20;  // 2 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace cs {
namespace {

struct NoAllocLayout {
  size_t counter, status, A32, At32, At64, G32, G64, cube, total;
  NoAllocLayout(int M, int N) {
    size_t o = 0;
    auto take = [&](size_t bytes) {
      size_t at = o;
      o += (bytes + 255) / 256 * 256;
      return at;
    };
    counter = take(8);
    status = counter + 8;
    A32 = take(sizeof(float) * (size_t)M * N);
    At32 = take(sizeof(float) * (size_t)M * N);
    At64 = take(sizeof(double) * (size_t)M * N);
    G32 = take(sizeof(float) * (size_t)N * N);
    G64 = take(sizeof(double) * (size_t)N * N);
    cube = take(sizeof(GrCube));
    total = o;
  }
};

// FP32 copy of A and its transposes in FP32 and FP64 (same values as the context setup).
__global__ void k_noalloc_casts(int M, int N, const double* A, float* A32, float* At32,
                                double* At64) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M * N) return;
  int m = i / N, n = i % N;
  const double a = A[i];
  A32[i] = (float)a;
  At32[n * M + m] = (float)a;
  At64[n * M + m] = a;
}

// G[r][c] = sum_k A[k][r] A[k][c] in FP64, summed in the same order as the context
// setup, and its FP32 rounding.
__global__ void k_noalloc_gram(int M, int N, const double* A, float* G32, double* G64) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N * N) return;
  int r = i / N, col = i % N;
  double s = 0.0;
  for (int k = 0; k < M; ++k) s += A[r + k * N] * A[k * N + col];
  G64[i] = s;
  G32[i] = (float)s;
}

// Device address of g_noalloc_scratch on the current device, looked up once per device.
constexpr int kMaxDevices = 64;
struct ScratchAddr {
  std::once_flag once;
  unsigned char* ptr = nullptr;
  cudaError_t err = cudaSuccess;
};
ScratchAddr g_scratch_addr[kMaxDevices];

}  // namespace

size_t noalloc_scratch_bytes(int M, int N) { return NoAllocLayout(M, N).total; }
size_t noalloc_scratch_capacity() { return kNoAllocScratchBytes; }

cudaError_t launch_gomp_noalloc(const double* A64, int M, int N, const GreedyArgs& a,
                                cudaStream_t stream) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  ScratchAddr& sa = g_scratch_addr[dev];
  std::call_once(sa.once, [&] {
    void* p = nullptr;
    sa.err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    sa.ptr = static_cast<unsigned char*>(p);
  });
  if (sa.err != cudaSuccess) return sa.err;
  NoAllocLayout lay(M, N);
  if (lay.total > kNoAllocScratchBytes) return cudaErrorInvalidValue;
  unsigned char* s = sa.ptr;
  float* A32 = reinterpret_cast<float*>(s + lay.A32);
  float* At32 = reinterpret_cast<float*>(s + lay.At32);
  double* At64 = reinterpret_cast<double*>(s + lay.At64);
  float* G32 = reinterpret_cast<float*>(s + lay.G32);
  double* G64 = reinterpret_cast<double*>(s + lay.G64);
  // the counter and the status word must start at zero on every call
  e = cudaMemsetAsync(s + lay.counter, 0, 16, stream);
  if (e != cudaSuccess) return e;
  if (a.P == 0) return cudaSuccess;
  k_noalloc_casts<<<(M * N + 255) / 256, 256, 0, stream>>>(M, N, A64, A32, At32, At64);
  k_noalloc_gram<<<(N * N + 255) / 256, 256, 0, stream>>>(M, N, A64, G32, G64);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;

  int num_sms = 0;
  e = cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  GrCube cube{};
  cube.M = M;
  cube.N = N;
  cube.A32 = A32;
  cube.At32 = At32;
  cube.At64 = At64;
  cube.G32 = G32;
  cube.G64 = G64;
  cube.Y = a.Y;
  cube.X = a.X;
  cube.P = a.P;
  cube.pix0 = 0;
  cube.kappa_pp = a.kappa_pp;
  cube.iters_out = a.iters_out;
  cube.conv_out = a.conv_out;
  GrCube* table = reinterpret_cast<GrCube*>(s + lay.cube);
  e = put_cubes(&cube, 1, table, stream);
  if (e != cudaSuccess) return e;
  GrParams p{};
  scalars(p, kGomp, a);
  p.Mmax = M;
  p.Nmax = N;
  p.cubes = table;
  p.ncubes = 1;
  p.total = a.P;
  p.status = reinterpret_cast<int*>(s + lay.status);
  p.counter = reinterpret_cast<unsigned long long*>(s + lay.counter);
  capacities(p, kGomp, a, M, N);
  Layout wl(M, N, p.cmax, p.dmax, p.kmax, p.selmax, true, true, false, false, p.dmax);
  p.warp_bytes = wl.total;
  int warps = (220 * 1024) / wl.total;
  if (warps > 8) warps = 8;
  if (warps < 1) return cudaErrorInvalidConfiguration;
  size_t smem = (size_t)warps * wl.total;
  auto kern = greedy_kernel<kGomp>((p.dmax + 31) / 32);
  e = allow_full_smem(reinterpret_cast<const void*>(kern));
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, warps * 32, smem);
  if (per_sm < 1) per_sm = 1;
  long long grid = (long long)num_sms * per_sm;
  long long need = (a.P + warps - 1) / warps;
  if (grid > need) grid = need;
  kern<<<(unsigned)grid, warps * 32, smem, stream>>>(p);
  return cudaGetLastError();
}

}  // namespace cs
