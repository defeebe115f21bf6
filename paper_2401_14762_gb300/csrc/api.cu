// C ABI of libcs_hsi.so (declared in include/cs_hsi.h): argument checks, context
// lifetime, host-pointer staging and dispatch to the device kernels.
#include <cuda_runtime.h>
#include <stdio.h>

#include <algorithm>
#include <cmath>
#include <vector>
#include <new>
#include <string>

#include "cs_hsi.h"
#include "cs_internal.cuh"

struct cs_ctx {
  cs::Ctx c;
};

namespace cs {

static thread_local std::string g_err;

void set_error(const std::string& msg) { g_err = msg; }

cs_status cuda_fail(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? CS_ERR_OOM : CS_ERR_CUDA;
}

namespace {

cs_status arg_error(const char* msg) {
  set_error(msg);
  return CS_ERR_ARG;
}

template <typename T>
cudaError_t dalloc(T** p, size_t elems) {
  return cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * (elems ? elems : 1));
}

void free_ctx(Ctx& c) {
  cudaFree(c.A64);
  cudaFree(c.At64);
  cudaFree(c.G64);
  cudaFree(c.G32);
  cudaFree(c.A32);
  cudaFree(c.At32);
  cudaFree(c.W32);
  cudaFree(c.W64);
  cudaFree(c.Wpad);
  cudaFree(c.Psi64);
  cudaFree(c.Psi32);
  cudaFree(c.psi_cn);
  cudaFree(c.cube_table);
  cudaFree(c.scratch64);
  cudaFree(c.status);
  cudaFree(c.counter);
  cudaFree(c.stage_in);
  cudaFree(c.stage_out);
  cudaFree(c.stage_aux);
  cudaFree(c.fb64);
  cudaFree(c.work);
  cudaFree(c.conv_counter);
  cudaFree(c.beta);
  for (float* b : c.beta_retired) cudaFree(b);
  for (int k = 0; k < Ctx::kAux; ++k) {
    if (c.aux[k]) cudaStreamDestroy(c.aux[k]);
    if (c.ev_join[k]) cudaEventDestroy(c.ev_join[k]);
  }
  if (c.ev_fork) cudaEventDestroy(c.ev_fork);
  for (int b = 0; b < 2; ++b) {
    cudaFree(c.pipe_y[b]);
    cudaFree(c.pipe_x[b]);
    if (c.ev_in[b]) cudaEventDestroy(c.ev_in[b]);
    if (c.ev_comp[b]) cudaEventDestroy(c.ev_comp[b]);
    if (c.ev_out[b]) cudaEventDestroy(c.ev_out[b]);
  }
}

// The double buffers (chunks of `pixels`) and events of streamed recoveries.
cudaError_t ensure_pipe(Ctx& c, int64_t pixels) {
  cudaError_t e = cudaSuccess;
  if (!c.ev_in[0])
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
      e = cudaEventCreateWithFlags(&c.ev_in[b], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c.ev_comp[b], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c.ev_out[b], cudaEventDisableTiming);
    }
  if (e != cudaSuccess || c.pipe_cap >= pixels) return e;
  for (int b = 0; b < 2; ++b) {
    cudaFree(c.pipe_y[b]);
    cudaFree(c.pipe_x[b]);
    c.pipe_y[b] = c.pipe_x[b] = nullptr;
  }
  c.pipe_cap = 0;
  for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
    e = cudaMalloc(reinterpret_cast<void**>(&c.pipe_y[b]), sizeof(float) * pixels * c.M);
    if (e == cudaSuccess)
      e = cudaMalloc(reinterpret_cast<void**>(&c.pipe_x[b]), sizeof(float) * pixels * c.N);
  }
  if (e == cudaSuccess) c.pipe_cap = pixels;
  return e;
}

}  // namespace

cudaError_t ensure_conv_counters(Ctx& c, int n) {
  if (c.conv_counter_cap >= n) return cudaSuccess;
  cudaFree(c.conv_counter);
  c.conv_counter = nullptr;
  c.conv_counter_cap = 0;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&c.conv_counter),
                             sizeof(unsigned long long) * (size_t)n);
  if (e == cudaSuccess) c.conv_counter_cap = n;
  return e;
}

namespace {

// The fork-join streams and events of multi-cube convex batches, created once.
cudaError_t ensure_aux(Ctx& c) {
  if (c.ev_fork) return cudaSuccess;
  for (int k = 0; k < Ctx::kAux; ++k) {
    cudaError_t e = cudaStreamCreateWithFlags(&c.aux[k], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c.ev_join[k], cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
  }
  return cudaEventCreateWithFlags(&c.ev_fork, cudaEventDisableTiming);
}

// Is ptr device-accessible memory (cudaMalloc / managed)?  Host memory, pinned or not,
// goes through the staging path.
bool is_device_ptr(const void* ptr) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

cudaError_t ensure_stage(float** buf, size_t* have, size_t bytes) {
  if (*have >= bytes) return cudaSuccess;
  cudaFree(*buf);
  *buf = nullptr;
  *have = 0;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(buf), bytes ? bytes : 16);
  if (e == cudaSuccess) *have = bytes;
  return e;
}

cs_status check_ctx(const cs_ctx* ctx) {
  if (!ctx) return arg_error("ctx is NULL");
  return CS_OK;
}

// The option checks every recovery call makes (context calls and the allocation-free
// call alike).
cs_status check_opts(const cs_opts& o) {
  if (!(o.eps >= 0.0) || !std::isfinite(o.eps)) return arg_error("eps must be >= 0");
  if (o.max_iters < 0) return arg_error("max_iters < 0");
  if (o.prec == CS_FP8_E4M3)
    return arg_error("CS_FP8_E4M3 is not offered: E4M3 products do not meet rel-L2 1e-3");
  if (o.prec != CS_FP32 && o.prec != CS_BF16) return arg_error("unknown precision");
  if ((o.iters_out && !is_device_ptr(o.iters_out)) ||
      (o.converged_out && !is_device_ptr(o.converged_out)) ||
      (o.kappa_per_pixel && !is_device_ptr(o.kappa_per_pixel)))
    return arg_error("per-pixel option arrays must be device memory");
  return CS_OK;
}

// Runs `fn(Y_dev, X_dev)` on device buffers; host buffers are staged and copied back.
template <typename F>
cs_status with_cube(cs_ctx* ctx, const float* Y, float* X, int64_t P, int in_cols, int out_cols,
                    F fn) {
  Ctx& c = ctx->c;
  bool dy = is_device_ptr(Y), dx = is_device_ptr(X);
  if (dy != dx) return arg_error("input and output must both be device or both be host memory");
  if (dy) {
    cudaError_t e = fn(Y, X);
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    return CS_OK;
  }
  size_t bin = sizeof(float) * (size_t)P * in_cols, bout = sizeof(float) * (size_t)P * out_cols;
  cudaError_t e = ensure_stage(&c.stage_in, &c.stage_in_bytes, bin);
  if (e == cudaSuccess) e = ensure_stage(&c.stage_out, &c.stage_out_bytes, bout);
  if (e != cudaSuccess) return cuda_fail(e, "staging allocation");
  e = cudaMemcpyAsync(c.stage_in, Y, bin, cudaMemcpyHostToDevice, c.stream);
  if (e != cudaSuccess) return cuda_fail(e, "host-to-device copy");
  e = fn(c.stage_in, c.stage_out);
  if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
  e = cudaMemcpyAsync(X, c.stage_out, bout, cudaMemcpyDeviceToHost, c.stream);
  if (e != cudaSuccess) return cuda_fail(e, "device-to-host copy");
  e = cudaStreamSynchronize(c.stream);
  if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
  return CS_OK;
}

// Eq. 1 on a cube in host memory, in chunks of up to kHostChunk pixels: while chunk k is
// measured, chunk k + 1 (X and E) is copied in and chunk k - 1 (Y) copied out, through
// two device buffers per direction (the context's pipeline buffers; E's in stage_aux).
// Every pixel is computed by the same kernel as in a device-memory call, so the results
// are the same bit for bit.
constexpr int64_t kHostChunk = 262144;
cs_status measure_host(Ctx& c, const float* X, float* Y, const float* E, int64_t P) {
  const int64_t C = std::min(kHostChunk, P);
  cudaError_t e = ensure_aux(c);
  if (e == cudaSuccess) e = ensure_pipe(c, C);
  if (e == cudaSuccess && E)
    e = ensure_stage(&c.stage_aux, &c.stage_aux_bytes, sizeof(float) * 2 * (size_t)C * c.M);
  if (e != cudaSuccess) return cuda_fail(e, "stream buffers");
  e = cudaEventRecord(c.ev_fork, c.stream);
  for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(c.aux[k], c.ev_fork, 0);
  if (e != cudaSuccess) return cuda_fail(e, "stream fork");
  cudaStream_t s_in = c.aux[0], s_out = c.aux[1], s_comp = c.aux[2], own = c.stream;
  int64_t off = 0;
  for (int k = 0; off < P && e == cudaSuccess; ++k, off += C) {
    const int b = k & 1;
    const int64_t n = std::min(C, P - off);
    float* Eb = E ? c.stage_aux + (size_t)b * C * c.M : nullptr;
    if (k >= 2) e = cudaStreamWaitEvent(s_in, c.ev_out[b], 0);  // buffer b copied out
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(c.pipe_x[b], X + off * c.N, sizeof(float) * n * c.N,
                          cudaMemcpyHostToDevice, s_in);
    if (e == cudaSuccess && E)
      e = cudaMemcpyAsync(Eb, E + off * c.M, sizeof(float) * n * c.M, cudaMemcpyHostToDevice,
                          s_in);
    if (e == cudaSuccess) e = cudaEventRecord(c.ev_in[b], s_in);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s_comp, c.ev_in[b], 0);
    if (e != cudaSuccess) break;
    c.stream = s_comp;
    e = launch_measure(c, c.pipe_x[b], c.pipe_y[b], Eb, n);
    c.stream = own;
    if (e == cudaSuccess) e = cudaEventRecord(c.ev_comp[b], s_comp);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s_out, c.ev_comp[b], 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(Y + off * c.M, c.pipe_y[b], sizeof(float) * n * c.M,
                          cudaMemcpyDeviceToHost, s_out);
    if (e == cudaSuccess) e = cudaEventRecord(c.ev_out[b], s_out);
  }
  cudaError_t ej = cudaEventRecord(c.ev_join[1], s_out);
  if (ej == cudaSuccess) ej = cudaStreamWaitEvent(c.stream, c.ev_join[1], 0);
  if (e == cudaSuccess) e = ej;
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
  if (e != cudaSuccess) return cuda_fail(e, "streamed measurement");
  return CS_OK;
}

}  // namespace
}  // namespace cs

using cs::arg_error;
using cs::cuda_fail;

extern "C" {

void cs_opts_default(cs_opts* o) {
  if (!o) return;
  o->eps = 1e-8;
  o->max_iters = 100;
  o->prec = CS_FP32;
  o->mu = 0.1;
  o->iters_out = nullptr;
  o->converged_out = nullptr;
  o->kappa_per_pixel = nullptr;
  o->cycle_skip = 1;
}

const char* cs_last_error(void) { return cs::g_err.c_str(); }

cs_status cs_create(cs_ctx** out, int M, int N, const double* A_host, const double* Phi_host,
                    const double* Psi_host, double admm_rho, void* stream) {
  cs::set_error("");
  if (!out) return arg_error("out is NULL");
  *out = nullptr;
  if (M < 1 || N < 1 || M > N || M > cs::kMaxM || N > cs::kMaxN) {
    cs::set_error("need 1 <= M <= N, M <= 128, N <= 256");
    return CS_ERR_SHAPE;
  }
  if (!A_host && !Phi_host) return arg_error("give A or Phi");
  if (!(admm_rho >= 0.0) || !std::isfinite(admm_rho)) return arg_error("admm_rho must be >= 0");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    cs::set_error(std::string("no CUDA device: ") + cudaGetErrorString(e));
    return CS_ERR_NO_DEVICE;
  }
  cudaDeviceProp prop;
  e = cudaGetDeviceProperties(&prop, dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceProperties");
  if (prop.major != 10 || prop.minor != 3) {
    cs::set_error("libcs_hsi is built for compute capability 10.3 (GB300)");
    return CS_ERR_NO_DEVICE;
  }
  cs_ctx* ctx = new (std::nothrow) cs_ctx();
  if (!ctx) return CS_ERR_OOM;
  cs::Ctx& c = ctx->c;
  c.M = M;
  c.N = N;
  c.device = dev;
  c.num_sms = prop.multiProcessorCount;
  c.stream = static_cast<cudaStream_t>(stream);
  c.scratch_elems = (size_t)M * N + (size_t)N * N + 3 * (size_t)M * M + cs::kMaxM + 8;
  if ((e = cs::dalloc(&c.A64, (size_t)M * N)) != cudaSuccess ||
      (e = cs::dalloc(&c.At64, (size_t)N * M)) != cudaSuccess ||
      (e = cs::dalloc(&c.G64, (size_t)N * N)) != cudaSuccess ||
      (e = cs::dalloc(&c.G32, (size_t)N * N)) != cudaSuccess ||
      (e = cs::dalloc(&c.A32, (size_t)M * N)) != cudaSuccess ||
      (e = cs::dalloc(&c.At32, (size_t)N * M)) != cudaSuccess ||
      (e = cs::dalloc(&c.W32, (size_t)M * M)) != cudaSuccess ||
      (e = cs::dalloc(&c.W64, (size_t)M * M)) != cudaSuccess ||
      (e = cs::dalloc(&c.Wpad, (size_t)M * cs::smem_ld(M))) != cudaSuccess ||
      (e = cs::dalloc(&c.scratch64, c.scratch_elems)) != cudaSuccess ||
      (e = cs::dalloc(&c.status, 1)) != cudaSuccess ||
      (e = cs::dalloc(&c.counter, 2)) != cudaSuccess ||
      (e = cs::dalloc(&c.work, 1)) != cudaSuccess ||
      (e = cs::ensure_conv_counters(c, 2)) != cudaSuccess ||
      (!A_host && ((e = cs::dalloc(&c.Psi64, (size_t)N * N)) != cudaSuccess ||
                   (e = cs::dalloc(&c.Psi32, (size_t)N * 128 * ((N + 127) / 128))) !=
                       cudaSuccess ||
                   (e = cs::dalloc(&c.psi_cn, (size_t)N)) != cudaSuccess))) {
    cs::free_ctx(c);
    delete ctx;
    return cuda_fail(e, "cs_create allocation");
  }
  cudaMemsetAsync(c.status, 0, sizeof(int), c.stream);
  e = cs::setup_dictionary(c, A_host, Phi_host, Psi_host);
  if (e == cudaSuccess && admm_rho > 0.0) e = cs::setup_admm_factor(c, admm_rho);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
  if (e != cudaSuccess) {
    cs::free_ctx(c);
    delete ctx;
    return cuda_fail(e, "cs_create setup");
  }
  *out = ctx;
  return CS_OK;
}

cs_status cs_create_complex(cs_ctx** out, int M, int N, const double* A_host, double admm_rho,
                            void* stream) {
  cs::set_error("");
  if (!out) return arg_error("out is NULL");
  *out = nullptr;
  if (!A_host) return arg_error("A is NULL");
  if (M < 1 || N < 1 || M > N || 2 * M > cs::kMaxM || 2 * N > cs::kMaxN) {
    cs::set_error("complex dictionaries need 1 <= M <= N, M <= 64, N <= 128");
    return CS_ERR_SHAPE;
  }
  // the real form of A acting on (re, im) pairs: rows 2m, 2m + 1 and columns 2k, 2k + 1
  // hold [[Re a, -Im a], [Im a, Re a]] for a = A[m][k]
  std::vector<double> R((size_t)4 * M * N);
  const size_t ld = 2 * (size_t)N;
  for (int m = 0; m < M; ++m)
    for (int k = 0; k < N; ++k) {
      const double re = A_host[2 * ((size_t)m * N + k)], im = A_host[2 * ((size_t)m * N + k) + 1];
      R[(2 * m) * ld + 2 * k] = re;
      R[(2 * m) * ld + 2 * k + 1] = -im;
      R[(2 * m + 1) * ld + 2 * k] = im;
      R[(2 * m + 1) * ld + 2 * k + 1] = re;
    }
  cs_status st = cs_create(out, 2 * M, 2 * N, R.data(), nullptr, nullptr, admm_rho, stream);
  if (st == CS_OK) (*out)->c.complex_pairs = true;
  return st;
}

void cs_destroy(cs_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->c.stream);
  cs::free_ctx(ctx->c);
  delete ctx;
}

cs_status cs_get_lipschitz(const cs_ctx* ctx, double* L) {
  if (cs_status s = cs::check_ctx(ctx)) return s;
  if (!L) return arg_error("L is NULL");
  *L = ctx->c.L;
  return CS_OK;
}

cs_status cs_get_dictionary(const cs_ctx* ctx, double* A_host) {
  if (cs_status s = cs::check_ctx(ctx)) return s;
  if (!A_host) return arg_error("A_host is NULL");
  const cs::Ctx& c = ctx->c;
  cudaError_t e = cudaMemcpyAsync(A_host, c.A64, sizeof(double) * c.M * c.N,
                                  cudaMemcpyDeviceToHost, c.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
  if (e != cudaSuccess) return cuda_fail(e, "cs_get_dictionary");
  return CS_OK;
}

cs_status cs_measure(cs_ctx* ctx, const float* X, float* Y, const float* E, int64_t P) {
  if (cs_status s = cs::check_ctx(ctx)) return s;
  if (P < 0) return arg_error("P < 0");
  if (P == 0) return CS_OK;
  if (!X || !Y) return arg_error("X or Y is NULL");
  cs::Ctx& c = ctx->c;
  if (E && cs::is_device_ptr(E) != cs::is_device_ptr(X))
    return arg_error("E must be the same kind of memory as X and Y");
  if (cs::is_device_ptr(X) != cs::is_device_ptr(Y))
    return arg_error("input and output must both be device or both be host memory");
  if (!cs::is_device_ptr(X)) return cs::measure_host(c, X, Y, E, P);  // copies overlapped
  return cs::with_cube(ctx, X, Y, P, c.N, c.M, [&](const float* Xd, float* Yd) {
    return cs::launch_measure(c, Xd, Yd, E, P);
  });
}

cs_status cs_sparsify(cs_ctx* ctx, const float* F, float* X, int64_t P, double T, int ddof,
                      int16_t* kappa_out, unsigned long long* recomputed_out) {
  cs::set_error("");
  if (cs_status s = cs::check_ctx(ctx)) return s;
  cs::Ctx& c = ctx->c;
  if (!c.Psi64) return arg_error("the context was made from A: it holds no transform Psi");
  if (P < 0) return arg_error("P < 0");
  if (!std::isfinite(T)) return arg_error("T must be finite");
  if (ddof != 0 && ddof != 1) return arg_error("ddof must be 0 or 1");
  if (P > ((int64_t)1 << 31) - 1) {
    cs::set_error("P must be below 2^31");
    return CS_ERR_SHAPE;
  }
  if (P > 0 && (!F || !X)) return arg_error("F or X is NULL");
  if ((P > 0 && (!cs::is_device_ptr(F) || !cs::is_device_ptr(X))) ||
      (kappa_out && !cs::is_device_ptr(kappa_out)) ||
      (recomputed_out && !cs::is_device_ptr(recomputed_out)))
    return arg_error("F, X, kappa_out and recomputed_out must be device memory");
  if (P == 0) return CS_OK;
  cudaError_t e = cs::launch_sparsify(c, F, X, P, T, ddof, kappa_out, recomputed_out);
  if (e != cudaSuccess) return cuda_fail(e, "sparsify launch");
  return CS_OK;
}

static cs_status check_common(const cs_ctx* ctx, const float* Y, float* X, int64_t P,
                              const cs_opts* o) {
  if (cs_status s = cs::check_ctx(ctx)) return s;
  if (P < 0) return arg_error("P < 0");
  if (P > 0 && (!Y || !X)) return arg_error("Y or X is NULL");
  if (P > ((int64_t)1 << 31) - 1) {
    cs::set_error("P must be below 2^31");
    return CS_ERR_SHAPE;
  }
  return cs::check_opts(*o);
}

cs_status cs_recover_fista(cs_ctx* ctx, const float* Y, float* X, int64_t P, double lambda,
                           int iters, const cs_opts* opts) {
  cs_opts o;
  cs_opts_default(&o);
  if (opts) o = *opts;
  if (cs_status s = check_common(ctx, Y, X, P, &o)) return s;
  if (!(lambda >= 0.0) || !std::isfinite(lambda)) return arg_error("lambda must be >= 0");
  if (iters < 0) return arg_error("iters < 0");
  if (P == 0) return CS_OK;
  cs::Ctx& c = ctx->c;
  return cs::with_cube(ctx, Y, X, P, c.M, c.N, [&](const float* Yd, float* Xd) {
    cs::ConvexArgs a{Yd, Xd, P, lambda, 0.0, o.eps, iters, o.iters_out, o.converged_out, o.prec};
    return cs::launch_fista(c, a);
  });
}

cs_status cs_recover_admm(cs_ctx* ctx, const float* Y, float* X, int64_t P, double rho,
                          double lambda, int iters, const cs_opts* opts) {
  cs_opts o;
  cs_opts_default(&o);
  if (opts) o = *opts;
  if (cs_status s = check_common(ctx, Y, X, P, &o)) return s;
  if (!(rho > 0.0) || !std::isfinite(rho)) return arg_error("rho must be > 0");
  if (!(lambda >= 0.0) || !std::isfinite(lambda)) return arg_error("lambda must be >= 0");
  if (iters < 0) return arg_error("iters < 0");
  if (P == 0) return CS_OK;
  cs::Ctx& c = ctx->c;
  if (c.rho != rho) {
    cudaError_t e = cs::setup_admm_factor(c, rho);
    if (e != cudaSuccess) return cuda_fail(e, "ADMM factor");
  }
  return cs::with_cube(ctx, Y, X, P, c.M, c.N, [&](const float* Yd, float* Xd) {
    cs::ConvexArgs a{Yd, Xd, P, lambda, rho, o.eps, iters, o.iters_out, o.converged_out, o.prec};
    return cs::launch_admm(c, a);
  });
}

static cs_status greedy(cs_ctx* ctx, cs::GreedyAlgo algo, const float* Y, float* X, int64_t P,
                        int kappa, int G, const cs_opts* opts) {
  cs_opts o;
  cs_opts_default(&o);
  if (opts) o = *opts;
  if (cs_status s = check_common(ctx, Y, X, P, &o)) return s;
  cs::Ctx& c = ctx->c;
  // a complex context counts complex atoms: N / 2 of them on its real form
  const int Na = c.complex_pairs ? c.N / 2 : c.N;
  int kmax = kappa;
  if (o.kappa_per_pixel) {
    // the caller bounds the per-pixel levels by kappa (used to size the workspace)
    if (kappa < 0 || kappa > Na) return arg_error("kappa (upper bound) out of range");
  } else if (kappa < 0 || kappa > Na) {
    return arg_error("kappa out of range");
  }
  if (algo == cs::kCosamp && 2 * kmax > Na) return arg_error("CoSaMP needs 2 kappa <= N");
  if (algo == cs::kGomp && (G < 0 || G > Na || (G == 0 && !o.kappa_per_pixel)))
    return arg_error("G must be in 1..N (0 only with kappa_per_pixel)");
  if (algo == cs::kBiht && !std::isfinite(o.mu)) return arg_error("mu must be finite");
  if (P == 0) return CS_OK;
  return cs::with_cube(ctx, Y, X, P, c.M, c.N, [&](const float* Yd, float* Xd) {
    cs::GreedyArgs a{Yd, Xd, P, kappa, G, o.mu, o.eps, o.max_iters, o.kappa_per_pixel, kmax,
                     o.iters_out, o.converged_out, o.prec, o.cycle_skip != 0};
    return cs::launch_greedy(c, algo, a);
  });
}

cs_status cs_recover_gomp(cs_ctx* ctx, const float* Y, float* X, int64_t P, int kappa, int G,
                          const cs_opts* opts) {
  return greedy(ctx, cs::kGomp, Y, X, P, kappa, G, opts);
}

cs_status cs_recover_biht(cs_ctx* ctx, const float* Y, float* X, int64_t P, int kappa,
                          const cs_opts* opts) {
  return greedy(ctx, cs::kBiht, Y, X, P, kappa, 0, opts);
}

cs_status cs_recover_cosamp(cs_ctx* ctx, const float* Y, float* X, int64_t P, int kappa,
                            const cs_opts* opts) {
  return greedy(ctx, cs::kCosamp, Y, X, P, kappa, 0, opts);
}

cs_status cs_recover_batch(const cs_batch_item* items, int n_items, cs_algo algo,
                           const cs_algo_params* params, const cs_opts* opts) {
  if (!items || n_items < 1) return arg_error("items is NULL or n_items < 1");
  if (!params) return arg_error("params is NULL");
  if (algo < CS_ALGO_FISTA || algo > CS_ALGO_COSAMP) return arg_error("unknown algorithm");
  cs_opts o;
  cs_opts_default(&o);
  if (opts) o = *opts;
  o.iters_out = nullptr;  // per item instead
  o.converged_out = nullptr;
  o.kappa_per_pixel = nullptr;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return cuda_fail(cudaErrorNoDevice, "cudaGetDevice");
  }
  const bool greedy = algo >= CS_ALGO_GOMP;
  const int kappa = params->kappa, G = params->G;
  for (int i = 0; i < n_items; ++i) {
    const cs_batch_item& it = items[i];
    if (cs_status s = check_common(it.ctx, it.Y, it.X, it.P, &o)) return s;
    const cs::Ctx& c = it.ctx->c;
    if (c.device != dev) return arg_error("every context must be on the current device");
    if (it.P > 0 && (!cs::is_device_ptr(it.Y) || !cs::is_device_ptr(it.X)))
      return arg_error("batch cubes must be in device memory");
    if ((it.iters_out && !cs::is_device_ptr(it.iters_out)) ||
        (it.converged_out && !cs::is_device_ptr(it.converged_out)) ||
        (it.kappa_per_pixel && !cs::is_device_ptr(it.kappa_per_pixel)))
      return arg_error("per-pixel arrays must be device memory");
    if (greedy && c.complex_pairs != items[0].ctx->c.complex_pairs)
      return arg_error("a greedy batch cannot mix complex and real contexts");
    if (greedy && it.P > 0) {
      const int Na = c.complex_pairs ? c.N / 2 : c.N;  // complex contexts count complex atoms
      if (kappa < 0 || kappa > Na) return arg_error("kappa out of range for a cube");
      if (algo == CS_ALGO_COSAMP && 2 * kappa > Na)
        return arg_error("CoSaMP needs 2 kappa <= N for every cube");
      if (algo == CS_ALGO_GOMP && (G < 0 || G > Na || (G == 0 && !it.kappa_per_pixel)))
        return arg_error("G must be in 1..N (0 only with kappa_per_pixel)");
    }
  }
  if (greedy && algo == CS_ALGO_BIHT && !std::isfinite(o.mu)) return arg_error("mu must be finite");
  if (!greedy) {
    if (!(params->lambda >= 0.0) || !std::isfinite(params->lambda))
      return arg_error("lambda must be >= 0");
    if (params->iters < 0) return arg_error("iters < 0");
    if (algo == CS_ALGO_ADMM && (!(params->rho > 0.0) || !std::isfinite(params->rho)))
      return arg_error("rho must be > 0");
  }
  cs::Ctx& c0 = items[0].ctx->c;
  if (greedy) {
    std::vector<cs::GreedyCube> cubes(n_items);
    for (int i = 0; i < n_items; ++i) {
      const cs_batch_item& it = items[i];
      cubes[i] = cs::GreedyCube{&it.ctx->c, it.Y,          it.X,         it.P,
                                it.kappa_per_pixel, it.iters_out, it.converged_out};
    }
    const cs::GreedyAlgo ga =
        algo == CS_ALGO_GOMP ? cs::kGomp : (algo == CS_ALGO_BIHT ? cs::kBiht : cs::kCosamp);
    cs::GreedyArgs a{nullptr, nullptr, 0, kappa, algo == CS_ALGO_GOMP ? G : 0, o.mu, o.eps,
                     o.max_iters, nullptr, kappa, nullptr, nullptr, o.prec, o.cycle_skip != 0};
    cudaError_t e = cs::launch_greedy_batch(c0, ga, cubes.data(), n_items, a);
    if (e != cudaSuccess) return cuda_fail(e, "batched greedy launch");
    return CS_OK;
  }
  // FISTA / ADMM: one launch per cube, every launch reporting to items[0]'s status word.
  // First, on items[0]'s stream, each context's shared data: the ADMM factor for this rho,
  // FISTA's momentum table.  Then the cubes, largest first, round-robin over the fork-join
  // streams, which start after that stream's work and which it waits for at the end: the
  // launches of small cubes (a few tiles, far fewer than the SMs) run side by side.
  std::vector<int> order;
  for (int i = 0; i < n_items; ++i)
    if (items[i].P > 0) order.push_back(i);
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return items[a].P > items[b].P; });
  cudaError_t e = cudaSuccess;
  for (int i : order) {
    cs::Ctx& c = items[i].ctx->c;
    cudaStream_t own_stream = c.stream;
    c.stream = c0.stream;
    if (algo == CS_ALGO_ADMM) {
      if (c.rho != params->rho) e = cs::setup_admm_factor(c, params->rho);
    } else {
      e = cs::momentum_table(c, params->iters);
    }
    c.stream = own_stream;
    if (e != cudaSuccess) return cuda_fail(e, "batched convex setup");
  }
  // each launch counts its pixels in its own slot of c0's counters (the launches of
  // several cubes, even of one context, may run at the same time)
  e = cs::ensure_conv_counters(c0, (int)order.size() + 2);
  if (e != cudaSuccess) return cuda_fail(e, "batch counters");
  const bool fork = order.size() > 1;
  int used = 0;
  if (fork) {
    e = cs::ensure_aux(c0);
    if (e == cudaSuccess) e = cudaEventRecord(c0.ev_fork, c0.stream);
    if (e != cudaSuccess) return cuda_fail(e, "batch fork");
    used = (int)std::min<size_t>(order.size(), cs::Ctx::kAux);
    for (int k = 0; k < used && e == cudaSuccess; ++k)
      e = cudaStreamWaitEvent(c0.aux[k], c0.ev_fork, 0);
    if (e != cudaSuccess) return cuda_fail(e, "batch fork");
  }
  for (size_t j = 0; j < order.size() && e == cudaSuccess; ++j) {
    const cs_batch_item& it = items[order[j]];
    cs::Ctx& c = it.ctx->c;
    cudaStream_t own_stream = c.stream;
    int* own_status = c.status;
    c.stream = fork ? c0.aux[j % cs::Ctx::kAux] : c0.stream;
    c.status = c0.status;
    cs::ConvexArgs a{it.Y, it.X, it.P, params->lambda, params->rho, o.eps, params->iters,
                     it.iters_out, it.converged_out, o.prec, c0.conv_counter + 2 + j};
    e = algo == CS_ALGO_ADMM ? cs::launch_admm(c, a) : cs::launch_fista(c, a, false);
    c.stream = own_stream;
    c.status = own_status;
  }
  // join even after a failed launch, so that the context stream still follows whatever
  // did start
  for (int k = 0; k < used; ++k) {
    cudaError_t ej = cudaEventRecord(c0.ev_join[k], c0.aux[k]);
    if (ej == cudaSuccess) ej = cudaStreamWaitEvent(c0.stream, c0.ev_join[k], 0);
    if (e == cudaSuccess) e = ej;
  }
  if (e != cudaSuccess) return cuda_fail(e, "batched convex launch");
  return CS_OK;
}

cs_status cs_recover_stream(cs_ctx* ctx, cs_algo algo, const cs_algo_params* params,
                            const float* Y, float* X, int64_t P, int64_t chunk_pixels,
                            const cs_opts* opts) {
  cs::set_error("");
  if (!params) return arg_error("params is NULL");
  if (algo < CS_ALGO_FISTA || algo > CS_ALGO_COSAMP) return arg_error("unknown algorithm");
  cs_opts o;
  cs_opts_default(&o);
  if (opts) o = *opts;
  if (cs_status s = check_common(ctx, Y, X, P, &o)) return s;
  if (chunk_pixels < 1) return arg_error("chunk_pixels < 1");
  cs::Ctx& c = ctx->c;
  const bool is_greedy = algo >= CS_ALGO_GOMP;
  const int kappa = params->kappa, G = params->G;
  if (is_greedy) {
    const int Na = c.complex_pairs ? c.N / 2 : c.N;  // complex contexts count complex atoms
    if (kappa < 0 || kappa > Na) return arg_error("kappa out of range");
    if (algo == CS_ALGO_COSAMP && 2 * kappa > Na) return arg_error("CoSaMP needs 2 kappa <= N");
    if (algo == CS_ALGO_GOMP && (G < 0 || G > Na || (G == 0 && !o.kappa_per_pixel)))
      return arg_error("G must be in 1..N (0 only with kappa_per_pixel)");
    if (algo == CS_ALGO_BIHT && !std::isfinite(o.mu)) return arg_error("mu must be finite");
  } else {
    if (!(params->lambda >= 0.0) || !std::isfinite(params->lambda))
      return arg_error("lambda must be >= 0");
    if (params->iters < 0) return arg_error("iters < 0");
    if (algo == CS_ALGO_ADMM && (!(params->rho > 0.0) || !std::isfinite(params->rho)))
      return arg_error("rho must be > 0");
  }
  if (P == 0) return CS_OK;
  if (cs::is_device_ptr(Y) || cs::is_device_ptr(X))
    return arg_error("cs_recover_stream takes Y and X in host memory");
  const int64_t C = std::min(chunk_pixels, P);
  cudaError_t e = cs::ensure_aux(c);
  if (e == cudaSuccess) e = cs::ensure_pipe(c, C);
  if (e != cudaSuccess) return cuda_fail(e, "stream buffers");
  // per-call data every chunk reads, on the context stream before the fork
  if (algo == CS_ALGO_ADMM && c.rho != params->rho) e = cs::setup_admm_factor(c, params->rho);
  if (algo == CS_ALGO_FISTA) e = cs::momentum_table(c, params->iters);
  if (e == cudaSuccess) e = cudaEventRecord(c.ev_fork, c.stream);
  for (int k = 0; k < cs::Ctx::kAux && e == cudaSuccess; ++k)
    e = cudaStreamWaitEvent(c.aux[k], c.ev_fork, 0);
  if (e != cudaSuccess) return cuda_fail(e, "stream fork");
  // copy-in on aux[0], copy-out on aux[1]; the FISTA/ADMM chunks alternate between two
  // compute streams, the greedy ones share one (the persistent kernel's pixel counter
  // and fallback slots belong to the context)
  cudaStream_t s_in = c.aux[0], s_out = c.aux[1], own = c.stream;
  const cs::GreedyAlgo ga =
      algo == CS_ALGO_GOMP ? cs::kGomp : (algo == CS_ALGO_BIHT ? cs::kBiht : cs::kCosamp);
  int64_t off = 0;
  for (int k = 0; off < P && e == cudaSuccess; ++k, off += C) {
    const int b = k & 1;
    const int64_t n = std::min(C, P - off);
    cudaStream_t s_comp = c.aux[is_greedy ? 2 : 2 + b];
    if (k >= 2) e = cudaStreamWaitEvent(s_in, c.ev_out[b], 0);  // buffer b copied out
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(c.pipe_y[b], Y + off * c.M, sizeof(float) * n * c.M,
                          cudaMemcpyHostToDevice, s_in);
    if (e == cudaSuccess) e = cudaEventRecord(c.ev_in[b], s_in);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s_comp, c.ev_in[b], 0);
    if (e != cudaSuccess) break;
    int32_t* it = o.iters_out ? o.iters_out + off : nullptr;
    uint8_t* cv = o.converged_out ? o.converged_out + off : nullptr;
    c.stream = s_comp;
    if (is_greedy) {
      const int16_t* kp = o.kappa_per_pixel ? o.kappa_per_pixel + off : nullptr;
      cs::GreedyArgs a{c.pipe_y[b], c.pipe_x[b], n, kappa, algo == CS_ALGO_GOMP ? G : 0,
                       o.mu, o.eps, o.max_iters, kp, kappa, it, cv, o.prec,
                       o.cycle_skip != 0};
      e = cs::launch_greedy(c, ga, a);
    } else {
      cs::ConvexArgs a{c.pipe_y[b], c.pipe_x[b], n, params->lambda, params->rho, o.eps,
                       params->iters, it, cv, o.prec, c.conv_counter + b};
      e = algo == CS_ALGO_ADMM ? cs::launch_admm(c, a) : cs::launch_fista(c, a, false);
    }
    c.stream = own;
    if (e == cudaSuccess) e = cudaEventRecord(c.ev_comp[b], s_comp);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s_out, c.ev_comp[b], 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(X + off * c.N, c.pipe_x[b], sizeof(float) * n * c.N,
                          cudaMemcpyDeviceToHost, s_out);
    if (e == cudaSuccess) e = cudaEventRecord(c.ev_out[b], s_out);
  }
  // the last copy-out follows every compute and copy-in: join it, then wait for it
  cudaError_t ej = cudaEventRecord(c.ev_join[1], s_out);
  if (ej == cudaSuccess) ej = cudaStreamWaitEvent(c.stream, c.ev_join[1], 0);
  if (e == cudaSuccess) e = ej;
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
  if (e != cudaSuccess) return cuda_fail(e, "streamed recovery");
  return CS_OK;
}

cs_status cs_recover_gomp_noalloc(const double* A_dev, int M, int N, const float* Y, float* X,
                                  int64_t P, int kappa, int G, const cs_opts* opts,
                                  void* stream) {
  cs::set_error("");
  cs_opts o;
  cs_opts_default(&o);
  if (opts) o = *opts;
  if (M < 1 || N < 1 || M > N || M > cs::kMaxM || N > cs::kMaxN) {
    cs::set_error("need 1 <= M <= N, M <= 128, N <= 256");
    return CS_ERR_SHAPE;
  }
  size_t need = cs::noalloc_scratch_bytes(M, N), have = cs::noalloc_scratch_capacity();
  if (need > have) {
    cs::set_error("this M x N dictionary needs " + std::to_string(need) +
                  " bytes of static scratch; cs_recover_gomp_noalloc holds " +
                  std::to_string(have) + " (use cs_recover_gomp)");
    return CS_ERR_SHAPE;
  }
  if (P < 0) return arg_error("P < 0");
  if (P > ((int64_t)1 << 31) - 1) {
    cs::set_error("P must be below 2^31");
    return CS_ERR_SHAPE;
  }
  if (!A_dev || (P > 0 && (!Y || !X))) return arg_error("A, Y or X is NULL");
  if (!cs::is_device_ptr(A_dev) || (P > 0 && (!cs::is_device_ptr(Y) || !cs::is_device_ptr(X))))
    return arg_error("cs_recover_gomp_noalloc takes device memory only (staging host memory "
                     "would allocate)");
  if (cs_status st = cs::check_opts(o)) return st;
  if (kappa < 0 || kappa > N) return arg_error("kappa out of range");
  if (G < 0 || G > N || (G == 0 && !o.kappa_per_pixel))
    return arg_error("G must be in 1..N (0 only with kappa_per_pixel)");
  int dev = 0, major = 0, minor = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  if (e != cudaSuccess || major != 10 || minor != 3) {
    cs::set_error("needs a CUDA device of compute capability 10.3 (GB300)");
    return CS_ERR_NO_DEVICE;
  }
  cs::GreedyArgs a{Y, X, P, kappa, G, o.mu, o.eps, o.max_iters, o.kappa_per_pixel, kappa,
                   o.iters_out, o.converged_out, o.prec, o.cycle_skip != 0};
  e = cs::launch_gomp_noalloc(A_dev, M, N, a, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "cs_recover_gomp_noalloc");
  return CS_OK;
}

cs_status cs_autotune(cs_ctx* ctx, cs_algo algo, const cs_algo_params* params,
                      const float* Y_dev, int64_t P, const cs_opts* opts, cs_tuning* out) {
  cs::set_error("");
  if (cs_status s = cs::check_ctx(ctx)) return s;
  if (!params || !out) return arg_error("params or out is NULL");
  if (algo != CS_ALGO_GOMP && algo != CS_ALGO_BIHT && algo != CS_ALGO_COSAMP)
    return arg_error("only the greedy algorithms have launch configurations to tune");
  cs_opts o;
  cs_opts_default(&o);
  if (opts) o = *opts;
  o.iters_out = nullptr;
  o.converged_out = nullptr;
  o.kappa_per_pixel = nullptr;
  if (cs_status s = cs::check_opts(o)) return s;
  cs::Ctx& c = ctx->c;
  if (c.complex_pairs) return arg_error("complex contexts run the greedy methods as single-cube calls only");
  if (P < 1 || !Y_dev || !cs::is_device_ptr(Y_dev))
    return arg_error("the tuning sample must be P >= 1 pixels in device memory");
  const int kappa = params->kappa, G = algo == CS_ALGO_GOMP ? params->G : 0;
  if (kappa < 0 || kappa > c.N) return arg_error("kappa out of range");
  if (algo == CS_ALGO_COSAMP && 2 * kappa > c.N) return arg_error("CoSaMP needs 2 kappa <= N");
  if (algo == CS_ALGO_GOMP && (G < 1 || G > c.N)) return arg_error("G must be in 1..N");
  cudaError_t e = cs::ensure_stage(&c.stage_out, &c.stage_out_bytes,
                                   sizeof(float) * (size_t)P * c.N);
  if (e != cudaSuccess) return cuda_fail(e, "tuning output buffer");
  const cs::GreedyAlgo ga =
      algo == CS_ALGO_GOMP ? cs::kGomp : (algo == CS_ALGO_BIHT ? cs::kBiht : cs::kCosamp);
  cs::GreedyArgs a{Y_dev, c.stage_out, P, kappa, G, o.mu, o.eps, o.max_iters, nullptr, kappa,
                   nullptr, nullptr, o.prec, o.cycle_skip != 0};
  cs::GreedyTune t;
  e = cs::tune_greedy(c, ga, a, &t);
  if (e != cudaSuccess) return cuda_fail(e, "cs_autotune");
  out->factor_rows = t.d32;
  out->warps_per_cta = t.warps;
  out->ms = t.ms;
  out->ms_default = t.ms_default;
  out->tuned = t.valid ? 1 : 0;
  return CS_OK;
}

cs_status cs_set_tuning(cs_ctx* ctx, cs_algo algo, const cs_algo_params* params,
                        const cs_tuning* t) {
  if (cs_status s = cs::check_ctx(ctx)) return s;
  if (!params) return arg_error("params is NULL");
  if (algo != CS_ALGO_GOMP && algo != CS_ALGO_BIHT && algo != CS_ALGO_COSAMP)
    return arg_error("only the greedy algorithms have launch configurations to tune");
  const int k = algo == CS_ALGO_GOMP ? 0 : (algo == CS_ALGO_BIHT ? 1 : 2);
  cs::GreedyTune g;
  if (t && t->tuned) {
    if (t->warps_per_cta < 1 || t->warps_per_cta > 8 || t->factor_rows < 0)
      return arg_error("warps_per_cta must be in 1..8 and factor_rows >= 0");
    g.valid = true;
    g.kappa = params->kappa;
    g.G = algo == CS_ALGO_GOMP ? params->G : 0;
    g.d32 = t->factor_rows;
    g.warps = t->warps_per_cta;
    g.ms = t->ms;
    g.ms_default = t->ms_default;
  }
  ctx->c.tune[k] = g;
  return CS_OK;
}

cs_status cs_get_last_precision(const cs_ctx* ctx, cs_precision* prec) {
  if (cs_status s = cs::check_ctx(ctx)) return s;
  if (!prec) return arg_error("prec is NULL");
  *prec = ctx->c.last_prec;
  return CS_OK;
}

cs_status cs_get_work(cs_ctx* ctx, double* flops) {
  if (cs_status s = cs::check_ctx(ctx)) return s;
  if (!flops) return arg_error("flops is NULL");
  cs::Ctx& c = ctx->c;
  cudaError_t e = cudaMemcpyAsync(flops, c.work, sizeof(double), cudaMemcpyDeviceToHost, c.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
  if (e != cudaSuccess) return cuda_fail(e, "cs_get_work");
  return CS_OK;
}

cs_status cs_sync(cs_ctx* ctx) {
  if (cs_status s = cs::check_ctx(ctx)) return s;
  cs::Ctx& c = ctx->c;
  cudaError_t e = cudaStreamSynchronize(c.stream);
  if (e != cudaSuccess) return cuda_fail(e, "cs_sync");
  int st = 0;
  e = cudaMemcpy(&st, c.status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "cs_sync status read");
  if (st) {
    cudaMemset(c.status, 0, sizeof(int));
    if (st & cs::kStNonFinite) {
      cs::set_error("non-finite measurements");
      return CS_ERR_NONFINITE;
    }
    if (st & cs::kStNotSpd) {
      cs::set_error("a least-squares system was not positive definite");
      return CS_ERR_NOT_SPD;
    }
    if (st & cs::kStTimeout) {
      cs::set_error("a bounded device wait ran out");
      return CS_ERR_TIMEOUT;
    }
  }
  return CS_OK;
}

}  // extern "C"
