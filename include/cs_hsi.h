/*
 * cs_hsi.h -- C ABI of libcs_hsi.so: per-pixel sparse recovery of a compressively
 * sensed hyperspectral cube on one NVIDIA GB300 (sm_103a).
 *
 * Problem (Justo et al., "A Comparative Study of Compressive Sensing Algorithms for
 * Hyperspectral Imaging Reconstruction", Section II, Eq. 1): every pixel's N-band
 * spectrum is f = Psi x with x (nearly) sparse; the sensor records y = Phi f = A x with
 * A = Phi Psi (M x N, M < N).  All P pixels of a cube share A.  The recovery calls
 * run one of the paper's five algorithms (Section II-A, Algorithms 1-5) on every pixel.
 *
 * Conventions (all entry points):
 *   - Matrices are row-major.  A cube is pixel-major: Y is P x M (Y[p*M + m]) and
 *     X is P x N (X[p*N + n]), float32.  X holds the coefficient vectors x.
 *   - Limits: 1 <= M <= N, M <= 128, N <= 256 (spectral dimension of one pixel).
 *   - Y and X may be device pointers (cudaMalloc / torch) or host pointers (pageable or
 *     pinned).  With device pointers the call is asynchronous on the context's stream.
 *     With host pointers the library stages the cube through device buffers it owns,
 *     copies on its stream and synchronises before returning.  Both must be of the
 *     same kind.  Optional per-pixel outputs in cs_opts are always device pointers.
 *   - Argument errors are reported synchronously, before anything is launched.
 *   - Device-side conditions (non-finite input, a least-squares system that is not
 *     positive definite, an iteration budget that ran out in a bounded wait) are
 *     latched in a per-context status word; cs_sync() returns and clears it.
 *   - The caller owns Y, X and the per-pixel output arrays; the context owns A, its
 *     casts and factorisations and any staging buffers.  A context is not
 *     thread-safe; use one per host thread.
 */
#ifndef CS_HSI_H
#define CS_HSI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cs_ctx cs_ctx;

typedef enum {
  CS_OK = 0,
  CS_ERR_ARG = 1,        /* invalid scalar argument or NULL pointer */
  CS_ERR_SHAPE = 2,      /* M, N or P outside the supported range */
  CS_ERR_CUDA = 3,       /* a CUDA runtime call failed (see cs_last_error) */
  CS_ERR_OOM = 4,        /* device allocation failed */
  CS_ERR_NOT_SPD = 5,    /* a support least-squares system was not positive definite */
  CS_ERR_TIMEOUT = 6,    /* a bounded device wait ran out */
  CS_ERR_NONFINITE = 7,  /* NaN or Inf in the measurements */
  CS_ERR_NO_DEVICE = 8   /* no CUDA device of compute capability 10.3 */
} cs_status;

/* Arithmetic of FISTA's and ADMM's products with A.  CS_FP32 is the plain FP32 (SIMT)
 * path.  CS_BF16 runs the products on the tcgen05 tensor cores with every operand split
 * into BF16 hi + lo parts (hi*hi + lo*hi + hi*lo, FP32 accumulation: about 16 bits of
 * each operand), where a kernel for the shape exists; cs_get_last_precision reports
 * which arithmetic a call used.  CS_FP8_E4M3 is rejected (CS_ERR_ARG) by every call:
 * per-tensor-scaled E4M3 products leave FISTA's 300-iteration iterate about 9e-2 from
 * the FP64 result (3.5e-2 with the last 100 iterations on split BF16), far from the
 * rel-L2 1e-3 bar, and the greedy calls' correlation, the only product FP8 could serve
 * there, takes under 5% of their time.  The greedy calls compute one way whatever prec
 * says: FP32 correlations whose selections are certified against FP64, FP32 Cholesky
 * factors refined to FP64 accuracy. */
typedef enum { CS_FP32 = 0, CS_BF16 = 1, CS_FP8_E4M3 = 2 } cs_precision;

/* Options shared by the recovery calls; pass NULL for the defaults. */
typedef struct {
  /* Stopping tolerance on Delta = ||r^i - r^{i-1}||_2 (Section II-A and every
   * algorithm's step 4/5).  Default 1e-8, the paper's epsilon (Section III).
   * 0 runs a fixed number of iterations. */
  double eps;
  /* Iteration cap for BIHT and CoSaMP (default 100) and an extra cap for gOMP,
   * whose own cap is min(kappa, floor(M/G)).  FISTA and ADMM take theirs as a call
   * argument. */
  int max_iters;
  cs_precision prec;       /* default CS_FP32 */
  double mu;               /* BIHT gradient step (Algorithm 4); default 0.1 (Section III) */
  int32_t *iters_out;      /* optional, device, P entries: iterations each pixel ran */
  uint8_t *converged_out;  /* optional, device, P entries: 1 if Delta < eps was reached,
                              0 if the cap stopped it, 2 if its support LS failed, 3 (greedy
                              calls) if its measurements are not finite */
  const int16_t *kappa_per_pixel; /* optional, device, P entries: per-pixel sparsity
                                     for the greedy calls; the call's kappa is then
                                     their upper bound and values outside 0..kappa
                                     are clamped into it */
  /* BIHT and CoSaMP: 1 (default) lets a pixel stop iterating once its iterate x repeats
   * an earlier one bit for bit.  Each iteration is a deterministic function of x, so the
   * iterates are then periodic, every later Delta repeats one already tested against
   * eps, and the cap decides: the pixel runs only the iterations that bring it to the
   * cap's phase of the cycle.  X, iters_out and converged_out are exactly those of
   * running every iteration.  0 runs every iteration. */
  int cycle_skip;
} cs_opts;

/* Fills *opts with the defaults listed above. */
void cs_opts_default(cs_opts *opts);

/* Creates a context for an M x N dictionary (Eq. 1) on the current CUDA device.
 *   A_host:   M x N row-major FP64 dictionary A = Phi Psi, or NULL to build it from
 *   Phi_host: M x N row-major FP64 measurement matrix, and
 *   Psi_host: N x N row-major FP64 sparsifying basis (f = Psi x), or NULL for the
 *             orthonormal DCT-II basis, Psi[n][k] = a_k cos(pi (2n+1) k / 2N).
 *   admm_rho: ADMM penalty alpha (Algorithm 2) to factor ahead of time; 0 to skip.
 *   stream:   cudaStream_t every call of this context runs on (NULL = legacy default).
 * On the device, in FP64: A = Phi Psi, the Gram matrix A^T A, the Lipschitz constant
 * L = lambda_max(A^T A) (Section II-A) and, for ADMM, (A A^T + alpha I)^{-1}.
 * Host arrays are only read during the call.  Blocks until the setup has finished. */
cs_status cs_create(cs_ctx **out, int M, int N, const double *A_host, const double *Phi_host,
                    const double *Psi_host, double admm_rho, void *stream);

/* The paper's complex setup (Section II): Psi the unitary DFT and Phi keeping M of the N
 * spectral samples make A = Phi Psi complex, and x, y complex.  Creates a context for
 * the complex M x N dictionary A (host, row-major, interleaved (re, im) FP64 pairs:
 * A[2 (m N + k)] = Re a_mk, A[2 (m N + k) + 1] = Im a_mk) through its real form: a
 * 2M x 2N real dictionary acting on vectors of (re, im) pairs.  On such a context
 * cs_measure, cs_recover_fista and cs_recover_admm (also in cs_recover_batch and
 * cs_recover_stream) take Y as P x 2M and X as P x 2N float32, i.e. complex64 arrays of
 * P x M and P x N, and FISTA's and ADMM's soft thresholds act on the moduli |x_k|
 * (x_k scaled by max(|x_k| - t, 0) / |x_k|); L = lambda_max(A^H A).  These run on the
 * FP32 path (prec is ignored).  cs_recover_gomp, cs_recover_biht and cs_recover_cosamp
 * (single-cube calls) take the same arrays: kappa and G count complex atoms, each atom
 * the column pair (2k, 2k + 1) of the real form, selected and pruned by its modulus |x_k|
 * (FP32 moduli certified against the FP64 modulus, ties to the lower k), so supports and
 * iteration counts are those of the FP64 complex algorithms; they also run in
 * cs_recover_stream and in cs_recover_batch (a greedy batch is all complex or all real).
 * cs_autotune and cs_sparsify return CS_ERR_ARG on a complex context.  Limits:
 * 1 <= M <= N, M <= 64, N <= 128 (CS_ERR_SHAPE). */
cs_status cs_create_complex(cs_ctx **out, int M, int N, const double *A, double admm_rho,
                            void *cuda_stream);

/* Releases the context and all device memory it owns. */
void cs_destroy(cs_ctx *ctx);

/* L = lambda_max(A^T A), the FISTA step constant (Section II-A). */
cs_status cs_get_lipschitz(const cs_ctx *ctx, double *L);

/* Copies the FP64 dictionary A (M x N, row-major) the context built into A_host. */
cs_status cs_get_dictionary(const cs_ctx *ctx, double *A_host);

/* Measurement, Eq. 1: Y[p] = A X[p] (+ E[p]) for p < P.  X: P x N, Y: P x M, E: P x M
 * additive noise or NULL (the same kind of memory as X and Y).  FP32 arithmetic.  A
 * cube in host memory is measured in chunks of 262,144 pixels whose copies in and out
 * overlap the kernel (pinned memory lets them); the results equal a device-memory
 * call's bit for bit.  With N a multiple of 4 and a 16-byte-aligned device X, X is read
 * through a tensor map in 256-pixel x 32-column boxes; a box that has not arrived after
 * 100 ms stops the kernel and latches CS_ERR_TIMEOUT, returned by the next cs_sync. */
cs_status cs_measure(cs_ctx *ctx, const float *X, float *Y, const float *E, int64_t P);

/* FISTA, Algorithm 1: x^0 = z^0 = 0, t^0 = 1; per iteration
 *   x = soft(z - A^T(A z - y)/L, lambda/L), t' = (1 + sqrt(1 + 4t^2))/2,
 *   z = x + ((t-1)/t')(x - x_prev), Delta = ||A x - A x_prev||;
 * until Delta < opts->eps or `iters` iterations.  lambda >= 0, iters >= 0.
 * prec = CS_BF16 runs both products on the tensor cores with split-BF16 operands for
 * N and M (each padded to 16) of (128, 48), (208, 80), (224, 96) and (256, 112), i.e.
 * N = 113..128 with M = 33..48 up to N = 241..256 with M = 97..112; it multiplies the
 * increment x - x_prev and carries A x - y in FP32, so the products' rounding is
 * relative to the increment.  Other shapes, and complex contexts, run the FP32 path. */
cs_status cs_recover_fista(cs_ctx *ctx, const float *Y, float *X, int64_t P, double lambda,
                           int iters, const cs_opts *opts);

/* ADMM, Algorithm 2 with the soft threshold lambda/rho (the scaled form whose fixed
 * point is the Eq. 2 LASSO solution): x^0 = z^0 = w^0 = 0; per iteration
 *   x = (A^T A + rho I)^{-1}(A^T y + rho (z - w)), z = soft(x + w, lambda/rho),
 *   w = w + x - z, Delta = ||A x - A x_prev||;
 * until Delta < opts->eps or `iters` iterations.  rho > 0, lambda >= 0.  Returns x.
 * The x-update runs as h = W (y - A d), x = d + A^T h with d = z - w and
 * W = (A A^T + rho I)^{-1} factored once in FP64.  prec = CS_BF16 runs its three
 * products on the tensor cores with split-BF16 operands (about 16 bits each, FP32
 * accumulation) for the same (N, M) shapes as FISTA's: N and M padded to 16 of (128, 48),
 * (208, 80), (224, 96) or (256, 112).  Other shapes, and complex contexts, run the FP32
 * path.  On both tensor-core paths a CTA keeps one pixel per TMEM lane and hands a lane
 * whose pixel has stopped (Delta < eps) to the next pixel of the cube. */
cs_status cs_recover_admm(cs_ctx *ctx, const float *Y, float *X, int64_t P, double rho,
                          double lambda, int iters, const cs_opts *opts);

/* gOMP, Algorithm 3: per iteration select the G largest |A^T r|, add them to the
 * support c, solve least squares on c, keep the kappa largest coefficients q, solve
 * least squares on q, r = y - A x.  At most min(kappa, floor(M/G), max_iters)
 * iterations.  1 <= G <= N, 0 <= kappa <= N.  G = 0 with kappa_per_pixel selects
 * G = max(1, floor(kappa_p / 5)) per pixel (Section III's rule). */
cs_status cs_recover_gomp(cs_ctx *ctx, const float *Y, float *X, int64_t P, int kappa, int G,
                          const cs_opts *opts);

/* BIHT (backtracking IHT), Algorithm 4: u = x + mu A^T(y - A x), c = supp(x) U the
 * kappa largest |u|, least squares on c, keep the kappa largest coefficients. */
cs_status cs_recover_biht(cs_ctx *ctx, const float *Y, float *X, int64_t P, int kappa,
                          const cs_opts *opts);

/* CoSaMP, Algorithm 5: c = c U the 2 kappa largest |A^T r|, least squares on c, keep
 * the kappa largest coefficients (no refit), r = y - A x.  0 <= 2 kappa <= N. */
cs_status cs_recover_cosamp(cs_ctx *ctx, const float *Y, float *X, int64_t P, int kappa,
                            const cs_opts *opts);

/* The arithmetic the last recovery call on this context computed its products in:
 * CS_BF16 when FISTA or ADMM ran on the tensor cores, CS_FP32 otherwise (the FP32 SIMT
 * path, or a greedy call).  Set when the call is queued. */
cs_status cs_get_last_precision(const cs_ctx *ctx, cs_precision *prec);

/* Algorithmic work of the last greedy call on this context (cs_recover_gomp, _biht,
 * _cosamp), in flops: per pixel and iteration the correlation A^T r (2MN), a Cholesky
 * least-squares solve on the support of n atoms (n^3/3 + 2n^2; the minimum-norm form
 * n M^2 + M^3/3 + 2M^2 + nM when n > M; for gOMP, whose factor grows with its support,
 * the rows appended, i^2 flops for row i, + 2n^2), gOMP's refit on its kappa atoms when it
 * is performed, and the residual y - A x (2M|supp x|).  Implementation extras (refinement
 * passes, padding) are not counted.  Waits for the context's stream. */
cs_status cs_get_work(cs_ctx *ctx, double *flops);

/* gOMP exactly as cs_recover_gomp, for callers that cannot allocate device memory when
 * they recover a cube -- for example code whose device memory is all handed to its own
 * pool, or that cannot afford the device-wide synchronisation of cudaMalloc/cudaFree.
 * It needs no context and allocates nothing: the caller passes the FP64 dictionary
 * A_dev (M x N, row-major, e.g. from cs_get_dictionary) and the cube Y, X, all in
 * device memory it owns (host memory is rejected: staging it would allocate).  The
 * FP32 and FP64 copies of A^T, the FP32 copy of A, the Gram matrix A^T A in FP32 and
 * FP64 and the kernel's work counter live in one static device array of 2 MiB that
 * every GPU loading the library holds until exit; a shape needing more (20 M N + 12 N^2
 * bytes plus alignment) returns CS_ERR_SHAPE, but every shape the library accepts
 * (M <= 128, N <= 256) fits.  The first call on a device looks up that array's address;
 * make it before any stream capture.  Every call re-derives the scratch contents and
 * resets the counter, and all calls share the one array: calls that overlap on the GPU
 * race and must be ordered by the caller.  Asynchronous on `stream`; no status word
 * reaches the caller, so device-side conditions are reported only through
 * opts->converged_out (2 = LS failure, 3 = measurements not finite).  Options are
 * checked as in cs_recover_gomp.  The paper has no counterpart of this entry point. */
cs_status cs_recover_gomp_noalloc(const double *A_dev, int M, int N, const float *Y, float *X,
                                  int64_t P, int kappa, int G, const cs_opts *opts,
                                  void *stream);

/* ---- Batches: several cubes, each with its own dictionary, in one call ---- */

typedef enum {
  CS_ALGO_FISTA = 0,
  CS_ALGO_ADMM = 1,
  CS_ALGO_GOMP = 2,
  CS_ALGO_BIHT = 3,
  CS_ALGO_COSAMP = 4
} cs_algo;

/* One cube of a batch.  Y, X and the optional per-pixel arrays are device pointers the
 * caller owns, in the layouts of the single-cube calls. */
typedef struct {
  cs_ctx *ctx;                    /* the cube's dictionary (its M and N), from cs_create */
  const float *Y;                 /* P x M */
  float *X;                       /* P x N */
  int64_t P;
  const int16_t *kappa_per_pixel; /* optional, greedy: per-pixel sparsity (<= params.kappa) */
  int32_t *iters_out;             /* optional, P entries */
  uint8_t *converged_out;         /* optional, P entries */
} cs_batch_item;

/* The algorithm's parameters, shared by every cube of the batch. */
typedef struct {
  double lambda; /* FISTA, ADMM */
  double rho;    /* ADMM */
  int iters;     /* FISTA, ADMM */
  int kappa;     /* gOMP, BIHT, CoSaMP: sparsity, or the bound of kappa_per_pixel */
  int G;         /* gOMP: atoms per iteration; 0 = max(1, floor(kappa_p / 5)) per pixel */
} cs_algo_params;

/* Recovers the n_items cubes with one algorithm (the paper's per-pixel problem, Section
 * II, on every pixel of every cube).  The cubes may differ in M, N (each within the
 * context limits), P and per-pixel sparsity.  gOMP, BIHT and CoSaMP run every cube in one
 * persistent launch: warps take pixels from one counter over all cubes' pixels, so cubes
 * and pixels that finish early free their warps for the rest.  FISTA and ADMM, whose
 * per-pixel work is fixed by the iteration count, run one launch per cube, largest cube
 * first, spread over four streams of items[0].ctx that fork from its stream and join
 * back into it (small cubes, of fewer tiles than the GPU has SMs, run side by side).
 * Results equal the single-cube calls' bit for bit.
 * opts gives eps, max_iters, prec, mu and cycle_skip for every cube; its per-pixel
 * pointers are ignored (each item has its own).  Everything runs, asynchronously, on
 * items[0].ctx's stream; device-side conditions of the whole batch latch in items[0].ctx's
 * status word (cs_sync(items[0].ctx)).  Every context must be on the current device.
 * CUDA graphs: the call queues only kernels, memsets and event records/waits on that
 * stream (and the streams it forks), so once a first call with the same cubes has run
 * (which creates the fork streams and sizes the scratch), a caller may capture the call
 * on items[0].ctx's stream (relaxed capture mode) and replay the graph on new
 * measurements written into the same Y buffers.
 * Argument errors (a NULL or host pointer, P < 0, kappa out of any cube's range) return
 * before anything is launched. */
cs_status cs_recover_batch(const cs_batch_item *items, int n_items, cs_algo algo,
                           const cs_algo_params *params, const cs_opts *opts);

/* ---- Autotuning of the greedy kernels' launch configuration ---- */

/* A launch configuration of the greedy kernel (one warp per pixel, persistent). */
typedef struct {
  int factor_rows;   /* gOMP: rows of its FP32 Cholesky factor kept in shared memory (a
                        support that outgrows them is solved in FP64 in global memory);
                        BIHT and CoSaMP keep their whole support */
  int warps_per_cta; /* the CTAs per SM follow from the shared memory they take */
  double ms;         /* time on the tuning sample with this configuration */
  double ms_default; /* time on the sample with the built-in choice */
  int tuned;         /* 1 if this configuration replaced the built-in one */
} cs_tuning;

/* Measures the greedy kernel's launch configurations -- factor capacity (gOMP, from
 * 2 kappa to the whole support in steps of 8) x warps per CTA (2..8, as shared memory
 * allows) -- on a sample of the caller's cube (Y_dev: P x M device measurements; a few
 * tens of thousands of pixels suffice), with CUDA events on the context's stream, and
 * keeps the fastest for later calls of `algo` (gOMP, BIHT or CoSaMP) with the same kappa
 * and G on this context, unless none beats the built-in choice.  Results do not depend
 * on the configuration (every pixel computes the same iterates).  Writes the outcome to
 * *out.  Blocks until the measurements are done.  CS_ERR_ARG for FISTA/ADMM: their tile
 * is fixed by the 128 TMEM lanes and the shared memory a shape takes. */
cs_status cs_autotune(cs_ctx *ctx, cs_algo algo, const cs_algo_params *params, const float *Y_dev,
                      int64_t P, const cs_opts *opts, cs_tuning *out);

/* Installs a configuration (for example one cs_autotune chose earlier and the caller
 * cached) for later calls of `algo` with params->kappa and params->G; t == NULL or
 * t->tuned == 0 restores the built-in choice. */
cs_status cs_set_tuning(cs_ctx *ctx, cs_algo algo, const cs_algo_params *params,
                        const cs_tuning *t);

/* Pushbroom streaming (Section II: a pushbroom sensor delivers a frame of pixels at a
 * time, and per-pixel recovery needs none of the rest of the cube).  Recovers a cube
 * held in HOST memory (Y: P x M, X: P x N, row-major; pinned memory lets the copies
 * overlap) in chunks of chunk_pixels pixels (a number of sensor lines): while chunk k is
 * recovered, chunk k + 1 is copied in and chunk k - 1 copied out, through two device
 * buffers per direction (context-owned, grown on demand).  FISTA/ADMM chunks alternate
 * between two compute streams; gOMP/BIHT/CoSaMP chunks run in order on one.  algo and
 * params as in cs_recover_batch; opts as in the single-cube calls, its per-pixel arrays
 * (device, P entries) indexed by the pixel's position in the whole cube.  Results equal
 * the single-cube call's bit for bit.  Returns once X is in host memory.  Errors: as the
 * single-cube calls, plus CS_ERR_ARG for device Y or X or chunk_pixels < 1. */
cs_status cs_recover_stream(cs_ctx *ctx, cs_algo algo, const cs_algo_params *params,
                            const float *Y, float *X, int64_t P, int64_t chunk_pixels,
                            const cs_opts *opts);

/* Sparsification pre-processing (Section II): the paper makes each pixel kappa-sparse
 * before it is measured.  For every pixel p (row of F, P x N spectra, FP32, row-major,
 * device memory) the call takes x = Psi^T f to the transform domain (Psi is the
 * context's transform, which must be orthonormal; the default DCT-II is) and zeroes
 * x_i where |x_i| - mu < T sigma, mu and sigma the mean and the standard deviation of
 * |x| over the N coefficients (sigma normalised by N - ddof: ddof = 1 the sample form,
 * 0 the population form).  Larger T keeps fewer coefficients.
 *   X            P x N output coefficients (device), ready for cs_measure.
 *   kappa_out    optional, P entries (device): ||x_p||_0 after sparsification, usable
 *                as kappa_per_pixel of the greedy calls.
 *   recomputed_out optional, 1 entry (device), incremented by the number of pixels
 *                whose decisions were taken in FP64 (see below).
 * Every decision equals the one the FP64 definition takes: the transform runs in FP32
 * and a pixel with a coefficient whose margin to the threshold is within the FP32
 * error bound is recomputed in FP64.  Kept values are the FP32 (or FP64-rounded)
 * coefficients.  Errors: CS_ERR_ARG for a context made from A (no Psi), P < 0,
 * non-finite T, ddof other than 0/1, a NULL or host pointer; non-finite spectra latch
 * CS_ERR_NONFINITE.  Asynchronous on the context's stream. */
cs_status cs_sparsify(cs_ctx *ctx, const float *F, float *X, int64_t P, double T, int ddof,
                      int16_t *kappa_out, unsigned long long *recomputed_out);

/* Waits for the context's stream and returns (and clears) the latched device status. */
cs_status cs_sync(cs_ctx *ctx);

/* Message of the last error on this thread ("" if none). */
const char *cs_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* CS_HSI_H */
