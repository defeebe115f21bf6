// The greedy recovery kernel (gOMP, BIHT, CoSaMP) and its device code, included by
// greedy.cu, which instantiates it for real data and holds the host side, and by
// greedy_pairs.cu, which instantiates it for complex data on the real form (column
// pairs); the two compile in parallel.  The method is described at the top of greedy.cu.
#pragma once

#include <cuda_runtime.h>

#include "cs_internal.cuh"

namespace cs {

// One cube of a launch: its dictionary data and its pixels, which are the launch's
// pixels [pix0, pix0 + P).
struct GrCube {
  int M, N;
  const float* A32;    // M x N, FP32 rounding of A
  const float* At32;   // N x M, the same transposed (column j of A contiguous)
  const double* At64;  // N x M, FP64
  const float* G32;    // N x N, FP32 rounding of the Gram matrix A^T A
  const double* G64;   // N x N, FP64 Gram matrix
  const float* Y;
  float* X;
  int64_t P, pix0;
  const int16_t* kappa_pp;
  int32_t* iters_out;
  uint8_t* conv_out;
};

struct GrParams {
  int Mmax, Nmax, algo;  // the shared-memory slices are laid out for the largest cube
  const GrCube* cubes;   // device table, ascending pix0
  int ncubes;
  int64_t total;         // pixels over all cubes
  int kappa, G;
  float mu;
  double mu64;
  double eps2;
  int start_done;
  int max_iters;
  int cmax, dmax, kmax, selmax;
  int d32;           // rows of the FP32 factor kept in shared memory (<= dmax)
  int warp_bytes;
  int* status;
  unsigned long long* counter;
  double* fb64;      // per-warp global FP64 fallback slots (nullptr: FP64 factors in smem)
  int fb_slot;       // doubles per slot
  double* work;      // optional: algorithmic flops of the call are added here
  int cycle_skip;    // BIHT/CoSaMP: finish at the cap's phase once x repeats
};

namespace {

constexpr int kNK = kMaxN / 32;  // atoms per lane

// Byte offsets of one warp's shared-memory slice.  With fp64_smem the factor regions are
// sized for FP64 (the fallback factorisation then runs in place); otherwise they hold
// the FP32 factors only and the fallback uses the warp's global slot.
struct Layout {
  int y, y64, rf, xd, b32, bx, bk, inc, c, q, qp, qf, sel, xq, xqp, xqf, L, invd, v, s, wv, Lq,
      invq, vq, sq, svals, cx, cq, ring, total;
  __host__ __device__ Layout(int M, int N, int cmax, int dmax, int kmax, int selmax,
                             bool fp64_smem, bool need_q, bool need_cyc, bool need_xd,
                             int d32, bool pairs = false) {
    const int fw = fp64_smem ? 8 : 4;
    int o = 0;
    auto take = [&](int bytes, int align) {
      o = (o + align - 1) / align * align;
      int at = o;
      o += bytes;
      return at;
    };
    bx = take(8 * N, 8);  // A^T y in FP64, filled in for support atoms
    y64 = take(8 * M, 8);  // y in FP64 (exact), for the FP64 products with y
    xq = take(8 * kmax, 8);
    xqp = take(8 * kmax, 8);  // the previous iterate's kept coefficients (Delta)
    const int df = fp64_smem ? dmax : d32;  // factor rows held here
    L = take(fw * (df * (df + 1) / 2), 8);
    invd = take(fw * df, 8);
    // the in-place FP64 fallback's vectors (else they live in the warp's global slot)
    v = take(fp64_smem ? 8 * dmax : 0, 8);
    s = take(8 * cmax, 8);
    wv = take(fp64_smem ? 8 * dmax : 0, 8);
    const int kq = need_q ? kmax : 0;
    Lq = take(fw * (kq * (kq + 1) / 2), 8);
    invq = take(fw * kq, 8);
    vq = take(fp64_smem ? 8 * kq : 0, 8);
    sq = take(8 * kq, 8);
    // the minimum-norm solve's H^{-1} y (BIHT and CoSaMP; gOMP's support never exceeds M)
    // and the complex atoms' coefficient moduli of a prune (pairs)
    svals = take(need_q && !pairs ? 0 : 8 * cmax, 8);
    const int kc = need_cyc ? kmax : 0;  // saved iterate of the cycle search
    cx = take(8 * kc, 8);
    ring = take(need_cyc ? 8 * 32 : 0, 8);  // hashes of the last 32 iterates
    y = take(4 * M, 4);
    rf = take(4 * M, 4);   // FP32 residual of the current iterate
    b32 = take(4 * N, 4);  // A^T y in FP32 (the correlation)
    xqf = take(4 * kmax, 4);  // FP32 copies of xq (the correlation and the residual)
    xd = take(need_xd ? 4 * N : 0, 4);  // FP32 x row (BIHT's u = x + mu A^T r)
    c = take(2 * cmax, 2);
    q = take(2 * kmax, 2);
    qp = take(2 * kmax, 2);
    qf = take(2 * kq, 2);  // atoms of the rows the refit factor Lq holds (gOMP)
    cq = take(2 * kc, 2);
    sel = take(2 * selmax, 2);  // a selection: G, 2 kappa or kappa atoms, or kappa positions
    inc = take(N, 1);
    bk = take(N, 1);  // bx[j] holds A^T y for atom j
    total = (o + 15) / 16 * 16;
  }
};

// Column-major packed lower-triangular storage with column capacity `cap`:
// entry (t, i), t >= i, lives at i*cap - i*(i+1)/2 + t.
__device__ __forceinline__ int lidx(int t, int i, int cap) { return i * cap - i * (i + 1) / 2 + t; }

struct Warp {
  const GrParams& p;
  int lane;
  const GrCube* cb;  // the cube of the pixel in hand (device table entry)
  float *y, *rf, *xd, *b32, *xqf;
  double *y64, *bx, *xq, *xqp, *L, *invd, *v, *s, *wv, *Lq, *invq, *vq, *sq, *svals;
  uint8_t *inc, *bk;
  int16_t *c, *q, *qp, *qf, *sel;
  double* fb;  // this warp's global FP64 fallback slot, or nullptr
};

// b32 = A^T y in FP32 for every atom (the correlation's first term): lanes own atoms,
// rows of A are read coalesced, each sum in the order m = 0, 1, ...
__device__ void load_rhs32(Warp& w) {
  const int N = w.cb->N, M = w.cb->M;
  float acc[kNK];
#pragma unroll
  for (int kk = 0; kk < kNK; ++kk) acc[kk] = 0.f;
  for (int m = 0; m < M; ++m) {
    const float ym = w.y[m];
    const float* arow = w.cb->A32 + (size_t)m * N;
#pragma unroll
    for (int kk = 0; kk < kNK; ++kk) {
      const int n = w.lane + 32 * kk;
      if (n < N) acc[kk] = fmaf(__ldg(arow + n), ym, acc[kk]);
    }
  }
#pragma unroll
  for (int kk = 0; kk < kNK; ++kk) {
    const int n = w.lane + 32 * kk;
    if (n < N) w.b32[n] = acc[kk];
  }
  __syncwarp();
}

// (A^T y)_j in FP64 for every atom of atoms[0..n) not yet known: the M products of
// column j of A with y, lanes over the rows (contiguous in A^T), summed across the warp.
// Up to four atoms share one reduction: a first exchange (lanes 16 apart) trades two of
// the four partial sums, a second (8 apart) one of the remaining two, and three more
// finish the sum, which leaves atom i's total on lanes 8i..8i+7 after six FP64 additions
// instead of twenty.  Every total is added in the order a single-value butterfly over
// lanes 16, 8, 4, 2, 1 apart uses.
__device__ __forceinline__ void ensure_rhs_body(const double* At, int M, const double* y64,
                                                double* bx, uint8_t* bk, const int16_t* atoms,
                                                int n, int lane) {
  int t = 0;
  for (;;) {
    int j0 = -1, j1 = -1, j2 = -1, j3 = -1;  // warp-uniform (shared-memory broadcasts)
    for (; t < n && j3 < 0; ++t) {
      const int j = atoms[t];
      if (bk[j]) continue;
      if (j0 < 0) j0 = j;
      else if (j1 < 0) j1 = j;
      else if (j2 < 0) j2 = j;
      else j3 = j;
    }
    if (j0 < 0) return;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    for (int m = lane; m < M; m += 32) {
      const double ym = y64[m];
      a0 = fma(__ldg(At + (size_t)j0 * M + m), ym, a0);
      if (j1 >= 0) a1 = fma(__ldg(At + (size_t)j1 * M + m), ym, a1);
      if (j2 >= 0) a2 = fma(__ldg(At + (size_t)j2 * M + m), ym, a2);
      if (j3 >= 0) a3 = fma(__ldg(At + (size_t)j3 * M + m), ym, a3);
    }
    const bool h4 = (lane & 16) != 0, h3 = (lane & 8) != 0;
    double k0 = h4 ? a2 : a0, k1 = h4 ? a3 : a1;
    k0 += __shfl_xor_sync(0xffffffffu, h4 ? a0 : a2, 16);
    k1 += __shfl_xor_sync(0xffffffffu, h4 ? a1 : a3, 16);
    double v = h3 ? k1 : k0;
    v += __shfl_xor_sync(0xffffffffu, h3 ? k0 : k1, 8);
    v += __shfl_xor_sync(0xffffffffu, v, 4);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    __syncwarp();
    if ((lane & 7) == 0) {
      const int i = lane >> 3;  // 2 (lane bit 4) + (lane bit 3)
      const int j = i == 0 ? j0 : i == 1 ? j1 : i == 2 ? j2 : j3;
      if (j >= 0) {
        bx[j] = v;
        bk[j] = 1;
      }
    }
    __syncwarp();
  }
}

__device__ __forceinline__ void ensure_rhs(Warp& w, const int16_t* atoms, int n) {
  ensure_rhs_body(w.cb->At64, w.cb->M, w.y64, w.bx, w.bk, atoms, n, w.lane);
}

// One out-of-line copy of ensure_rhs for CoSaMP on supports of more than 64 atoms, whose
// larger least squares leave the hot loop short of instruction-cache room (5% faster
// there; gOMP, BIHT and smaller CoSaMP instances lose with it).
__device__ __noinline__ void ensure_rhs_ool(const double* At, int M, const double* y64, double* bx,
                                           uint8_t* bk, const int16_t* atoms, int n, int lane) {
  ensure_rhs_body(At, M, y64, bx, bk, atoms, n, lane);
}

// Appends row n to the factor L of a growing normal-equation system.  g(t) gives the
// system entry (n, t) for t <= n.  Forward substitution L_{0:n} w = g(0:n) by columns,
// then l_nn = sqrt(g(n,n) - w.w).  Also extends v = L^{-1} rhs with rhs_n.
// Returns false if the pivot is not positive (system not numerically definite).
template <typename GF>
__device__ bool append_row(int lane, double* wv, double* L, double* invd, double* v, int cap,
                           int n, GF g, double rhs_n) {
  for (int t = lane; t < n; t += 32) wv[t] = g(t);
  double gnn = g(n);
  __syncwarp();
  for (int i = 0; i < n; ++i) {
    double wi = wv[i] * invd[i];
    __syncwarp();
    if (lane == 0) wv[i] = wi;
    const double* col = L + lidx(0, i, cap);
    for (int t = i + 1 + lane; t < n; t += 32) wv[t] -= col[t] * wi;
    __syncwarp();
  }
  double ww = 0.0, wvv = 0.0;
  for (int t = lane; t < n; t += 32) {
    ww += wv[t] * wv[t];
    wvv += wv[t] * v[t];
    L[lidx(n, t, cap)] = wv[t];
  }
  ww = warp_sum(ww);
  wvv = warp_sum(wvv);
  double d = gnn - ww;
  bool ok = d > 1e-13 * fabs(gnn) && isfinite(d);
  double lnn = sqrt(ok ? d : 1.0);
  __syncwarp();
  if (lane == 0) {
    L[lidx(n, n, cap)] = lnn;
    invd[n] = 1.0 / lnn;
    v[n] = (rhs_n - wvv) / lnn;
  }
  __syncwarp();
  return ok;
}

// Solves L^T s = v (n x n) by rows, right-looking.
__device__ void back_solve(int lane, const double* L, const double* invd, const double* v,
                           double* s, int cap, int n) {
  for (int t = lane; t < n; t += 32) s[t] = v[t];
  __syncwarp();
  for (int i = n - 1; i >= 0; --i) {
    double si = s[i] * invd[i];
    __syncwarp();
    if (lane == 0) s[i] = si;
    for (int t = lane; t < i; t += 32) s[t] -= L[lidx(i, t, cap)] * si;
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------------
// Mixed-precision support least squares: FP32 Cholesky of G_c, FP32 triangular solves
// on vectors held in registers (lane l owns entries l, l+32, ...), and FP64 iterative
// refinement s <- s + G_c^{-1}(b - G_c s) whose residual uses the FP64 Gram matrix.
// FP64 work per solve is one n^2 residual (rarely two) instead of an n^3/3 factorisation,
// which matters on GB300, whose FP64 rate is 1/64 of its FP32 rate.
// ---------------------------------------------------------------------------------
template <int VR, typename T>
__device__ __forceinline__ T rpick(const T (&v)[VR], int slot) {
  T r = v[0];
#pragma unroll
  for (int k = 1; k < VR; ++k)
    if (slot == k) r = v[k];
  return r;
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// FP32 factors are packed row-major lower triangles: entry (i, k), k <= i, at
// i(i+1)/2 + k.  The triangular numbers i(i+1)/2 for 32 consecutive i are distinct
// mod 32, so 32 lanes reading one column of 32 consecutive rows hit 32 different banks,
// as do lanes reading along a row.
__device__ __forceinline__ int ridx(int i, int k) { return (i * (i + 1) >> 1) + k; }

// Gathers G_c (FP32) into L and factors it in place, left-looking in blocks of CB
// columns (four for systems of up to 64 rows, one beyond): lane l owns rows l, l+32, ...;
// for the block's columns j..j+CB-1 every owned row i accumulates
// t_i,c = G(i, j+c) - sum_{k<j} L(i, k) L(j+c, k) (one load of L(i, k) feeds CB
// products; rows j..j+CB-1 are read by broadcast), then the block's columns
// are finished in order: t_i,c -= L(i, j+c') L(j+c, j+c') for the block's earlier
// columns c' (shuffled from the owners of rows j+c), L(j+c, j+c) = sqrt(t_{j+c},c) and
// L(i, j+c) = t_i,c / L(j+c, j+c).  Returns false when a pivot drops below 1e-4 of its
// original diagonal (FP32 would lose the factor).  The factor is left in the unit form
// the solves use: U (unit lower triangle, packed as L) and invd(j) = 1 / L(j, j)^2.
template <int VR>
__device__ bool chol32(Warp& w, float* L, float* invd, int n, const int16_t* atoms) {
  const int lane = w.lane, N = w.cb->N;
  // gather: G row atoms[k] (read at the sorted atoms, a few sectors) into column k;
  // several columns of loads are in flight before their stores
  constexpr int kB = 4;
  const float* G32 = w.cb->G32;
  for (int k0 = 0; k0 < n; k0 += kB) {
    float g[kB][VR];
#pragma unroll
    for (int kk = 0; kk < kB; ++kk) {
      const int k = k0 + kk;
      const size_t row = (size_t)atoms[min(k, n - 1)] * N;
#pragma unroll
      for (int r = 0; r < VR; ++r) {
        const int i = k + lane + 32 * r;
        const int col = atoms[min(i, n - 1)];  // clamped lanes are not stored
        g[kk][r] = 0.f;
        if (k + 32 * r < n) g[kk][r] = __ldg(G32 + row + col);
      }
    }
#pragma unroll
    for (int kk = 0; kk < kB; ++kk) {
      const int k = k0 + kk;
#pragma unroll
      for (int r = 0; r < VR; ++r) {
        const int i = k + lane + 32 * r;
        if (k < n && i < n) {
          L[ridx(i, k)] = g[kk][r];
          if (i == k) invd[k] = g[kk][r];  // original diagonal, for the pivot test
        }
      }
    }
  }
  __syncwarp();
  int base[VR];  // start of each owned row (clamped in range for lanes past n)
#pragma unroll
  for (int r = 0; r < VR; ++r) base[r] = ridx(min(lane + 32 * r, n - 1), 0);
  constexpr int CB = VR <= 2 ? 4 : 1;  // columns per block (measured: wider systems lose)
  for (int j = 0; j < n; j += CB) {
    const int nb = min(CB, n - j);  // columns in this block
    const float* R[CB];             // rows j..j+CB-1 (clamped past n: read, unused)
#pragma unroll
    for (int c = 0; c < CB; ++c) R[c] = L + ridx(min(j + c, n - 1), 0);
    float t[VR][CB];
#pragma unroll
    for (int r = 0; r < VR; ++r)
#pragma unroll
      for (int c = 0; c < CB; ++c)
        t[r][c] = c < nb ? L[base[r] + j + c] : 0.f;  // G(i, j+c); rows above are discarded
    // rows that end before k read into the next row, inside the triangle (discarded)
    for (int k = 0; k < j; ++k) {
      float b[CB];
#pragma unroll
      for (int c = 0; c < CB; ++c) b[c] = R[c][k];
#pragma unroll
      for (int r = 0; r < VR; ++r) {
        if (32 * r + 31 >= j && 32 * r < n) {  // warp-uniform: the slot owns rows >= j
          const float l = L[base[r] + k];
#pragma unroll
          for (int c = 0; c < CB; ++c) t[r][c] = fmaf(-l, b[c], t[r][c]);
        }
      }
    }
    float lc[VR][CB];  // the block's finished columns, L(i, j+c), per owned row
#pragma unroll
    for (int c = 0; c < CB; ++c) {
      if (c < nb) {  // warp-uniform
        const int col = j + c, src = col & 31, slot = col >> 5;
#pragma unroll
        for (int c2 = 0; c2 < c; ++c2) {
          // L(j+c, j+c2) from the owner of row j+c
          float own[VR];
#pragma unroll
          for (int r = 0; r < VR; ++r) own[r] = lc[r][c2];
          const float lcc = __shfl_sync(0xffffffffu, rpick<VR>(own, slot), src);
#pragma unroll
          for (int r = 0; r < VR; ++r) t[r][c] = fmaf(-lc[r][c2], lcc, t[r][c]);
        }
        float tc[VR];
#pragma unroll
        for (int r = 0; r < VR; ++r) tc[r] = t[r][c];
        const float d = __shfl_sync(0xffffffffu, rpick<VR>(tc, slot), src);
        if (!(d > 1e-4f * invd[col])) return false;  // warp-uniform
        // the FP32 factor only preconditions the FP64 refinement: the hardware reciprocal
        // square root (a couple of ulps) serves for both the pivot and its inverse
        const float inv = rsqrtf(d), dj = d * inv;
#pragma unroll
        for (int r = 0; r < VR; ++r) {
          const int i = lane + 32 * r;
          lc[r][c] = i > col ? t[r][c] * inv : 0.f;
          if (i > col && i < n) L[base[r] + col] = lc[r][c];
        }
        if (lane == 0) {
          L[ridx(col, col)] = dj;
          invd[col] = inv;
        }
      }
    }
    __syncwarp();
  }
  // unit form for the solves: U(i, k) = L(i, k) / L(k, k) below the diagonal and
  // invd(k) = 1 / L(k, k)^2 (G_c = U D U^T with D = diag(L(k, k)^2))
#pragma unroll
  for (int r = 0; r < VR; ++r) {
    const int i = lane + 32 * r;
    if (32 * r < n) {
      for (int k = 0; k < n - 1; ++k)
        if (k < i && i < n) L[base[r] + k] *= invd[k];
    }
  }
  __syncwarp();
  for (int k = lane; k < n; k += 32) invd[k] = invd[k] * invd[k];
  __syncwarp();
  return true;
}

// Solves with G_c = U D U^T, U unit lower triangular (packed rows, the diagonal slot
// unused) and d2 = diag(D)^-1, on register-distributed vectors (lane l owns rows l,
// l+32, ...).  v := U^{-1} v by column sweeps (lanes t > i read U(t, i)); v := U^{-T} v
// by row sweeps (lanes t < i read U(i, t)).  With a unit diagonal, each step of a sweep
// is a shuffle and one FMA per owned row: the row's value needs no division, and rows
// that must not change multiply a zero.  Reads past the stored rows (lanes of rows >= n,
// or past row i's last entry) stay inside the triangle region and are multiplied by
// zero or land in rows >= n, which no one reads.
// fwd_unit<VR, K> sweeps only the first K slots (n <= 32 K): the rest are left alone.
template <int VR, int K = VR>
__device__ void fwd_unit(const float* U, int n, float (&v)[VR], int lane) {
  int base[K];
#pragma unroll
  for (int k = 0; k < K; ++k) base[k] = ridx(min(lane + 32 * k, n > 0 ? n - 1 : 0), 0);
#pragma unroll
  for (int S = 0; S < K; ++S) {
    if (32 * S >= n) break;  // warp-uniform
    const int iend = min(n, 32 * S + 32);
    const int t = lane + 32 * S;
    for (int i = 32 * S; i < iend; ++i) {
      const float zi = __shfl_sync(0xffffffffu, v[S], i - 32 * S);
      const float l = t > i ? U[base[S] + i] : 0.f;
      v[S] = fmaf(-l, zi, v[S]);
#pragma unroll
      for (int k = S + 1; k < K; ++k) v[k] = fmaf(-U[base[k] + i], zi, v[k]);
    }
  }
}
template <int VR>
__device__ void bwd_unit(const float* U, int n, float (&v)[VR], int lane) {
#pragma unroll
  for (int S = VR - 1; S >= 0; --S) {
    if (32 * S >= n) continue;  // warp-uniform
    const int iend = min(n, 32 * S + 32);
    const int t = lane + 32 * S;
    for (int i = iend - 1; i >= 32 * S; --i) {
      const float si = __shfl_sync(0xffffffffu, v[S], i - 32 * S);
      const float* row = U + ridx(i, 0);
      const float l = t < i ? row[min(t, i)] : 0.f;
      v[S] = fmaf(-l, si, v[S]);
#pragma unroll
      for (int k = 0; k < S; ++k) v[k] = fmaf(-row[lane + 32 * k], si, v[k]);
    }
  }
}
// v := G_c^{-1} v
template <int VR>
__device__ __forceinline__ void solve_unit(const float* U, const float* d2, int n, float (&v)[VR],
                                           int lane) {
  fwd_unit<VR>(U, n, v, lane);
#pragma unroll
  for (int k = 0; k < VR; ++k) v[k] *= d2[min(lane + 32 * k, n - 1)];
  bwd_unit<VR>(U, n, v, lane);
}

// Iterative refinement on the FP32 factor: returns true once a correction falls below
// 1e-9 of the solution (the solution then carries FP64 accuracy: the next correction,
// about cond(G_c) 2^-24 times this one, is below FP64 resolution), false if the
// corrections stop contracting (the system is too ill-conditioned for an FP32 factor).
// A solution only FP32-corrected once (about 1e-14 relative) would be cheaper, but it
// can turn an exact tie of the FP64 iterate, as in small integer examples, the other
// way.  The right-hand side is (A^T y)_c from w.bx.
template <int VR>
__device__ __forceinline__ bool refine32(const float* L, const float* invd, int n,
                                         const int16_t* atoms, double* s, const double* bx,
                                         const double* G, int N, int lane) {
  double sr[VR], rr[VR];
  int col[VR];
#pragma unroll
  for (int k = 0; k < VR; ++k) {
    const int t = lane + 32 * k;
    col[k] = atoms[min(t, n - 1)];
    sr[k] = 0.0;
    rr[k] = t < n ? bx[col[k]] : 0.0;
  }
  float prev = 3.0e38f, smax = 0.f;  // smax: max |s| of the first solve, the test's scale
  for (int step = 0; step < 5; ++step) {
    float f[VR];
#pragma unroll
    for (int k = 0; k < VR; ++k) f[k] = (float)rr[k];
    solve_unit<VR>(L, invd, n, f, lane);
    float dm = 0.f;
#pragma unroll
    for (int k = 0; k < VR; ++k) {
      int t = lane + 32 * k;
      if (t < n) {
        sr[k] += (double)f[k];
        dm = fmaxf(dm, fabsf(f[k]));
        s[t] = sr[k];
      }
    }
    dm = warp_max(dm);
    if (step == 0) smax = dm;  // the first correction is the FP32 solution itself
    __syncwarp();
    if (dm <= 1e-9f * smax) return true;
    if (step > 0 && dm > 0.5f * prev) return false;
    prev = dm;
    // r = b - G_c s in FP64; by symmetry lane t reads G(c_j, c_t) from row c_j, so a
    // warp's loads fall in one row at the sorted atoms; eight rows of loads in flight
    {
      double acc[VR][2];
#pragma unroll
      for (int k = 0; k < VR; ++k) {
        const int t = lane + 32 * k;
        acc[k][0] = t < n ? bx[col[k]] : 0.0;
        acc[k][1] = 0.0;
      }
      // whole blocks of kB columns, then the rest one by one (an FP64 instruction costs
      // the pipe as much with one useful lane as with 32, so none is spent on padding)
      constexpr int kB = VR <= 2 ? 8 : 4;
      int j0 = 0;
      for (; j0 + kB <= n; j0 += kB) {
        double g[kB][VR];
#pragma unroll
        for (int jj = 0; jj < kB; ++jj) {
          const double* grow = G + (size_t)atoms[j0 + jj] * N;
#pragma unroll
          for (int k = 0; k < VR; ++k) g[jj][k] = 32 * k < n ? __ldg(grow + col[k]) : 0.0;
        }
#pragma unroll
        for (int jj = 0; jj < kB; ++jj) {
          const double sj = s[j0 + jj];
#pragma unroll
          for (int k = 0; k < VR; ++k) acc[k][jj & 1] = fma(-g[jj][k], sj, acc[k][jj & 1]);
        }
      }
      for (; j0 < n; ++j0) {
        const double* grow = G + (size_t)atoms[j0] * N;
        const double sj = s[j0];
#pragma unroll
        for (int k = 0; k < VR; ++k)
          acc[k][j0 & 1] = fma(-(32 * k < n ? __ldg(grow + col[k]) : 0.0), sj, acc[k][j0 & 1]);
      }
#pragma unroll
      for (int k = 0; k < VR; ++k) rr[k] = lane + 32 * k < n ? acc[k][0] + acc[k][1] : 0.0;
    }
  }
  return false;
}

// One out-of-line copy of the refinement for gOMP, which refines twice per iteration (its
// growing support and the refit on q): a single copy of its code keeps the kernel's hot
// loop small enough for the instruction cache (13% faster on the 2048^2 x 256 cube); the
// arguments are pointers and scalars, so nothing is spilled to pass them.
template <int VR>
__device__ __noinline__ bool refine32_ool(const float* L, const float* invd, int n,
                                          const int16_t* atoms, double* s, const double* bx,
                                          const double* G, int N, int lane) {
  return refine32<VR>(L, invd, n, atoms, s, bx, G, N, lane);
}
// A copy takes as many register slots per lane as the system has rows in use: slots past
// them would only add instructions, FP64 ones in the residual among them.
template <int VR, bool OOL>
__device__ __forceinline__ bool refine(const float* L, const float* invd, int n,
                                       const int16_t* atoms, double* s, const double* bx,
                                       const double* G, int N, int lane) {
  if (OOL) {
    if (VR > 1 && n <= 32) return refine32_ool<1>(L, invd, n, atoms, s, bx, G, N, lane);
    if (VR > 2 && n <= 64) return refine32_ool<(VR > 2 ? 2 : VR)>(L, invd, n, atoms, s, bx, G, N, lane);
    return refine32_ool<VR>(L, invd, n, atoms, s, bx, G, N, lane);
  }
  return refine32<VR>(L, invd, n, atoms, s, bx, G, N, lane);
}

// Extends the unit-form FP32 factor of G_c (U, d2 = invd) from its first nf rows to n
// rows, for atoms appended at the end of c (gOMP's growing support): for row i,
// z = U_{0:i}^{-1} G(c_{0:i}, c_i) by one forward sweep with the factor built so far,
// U(i, k) = z_k d2_k, pivot D(i) = G(c_i, c_i) - sum_k z_k^2 d2_k and d2_i = 1 / D(i).
// Returns false when a pivot drops below 1e-4 of its diagonal.  One out-of-line copy
// serves gOMP's two callers (its growing support and the refit on q), which keeps the
// kernel's hot loop within the instruction cache (12% faster on the 2048^2 x 256 cube);
// pointer and scalar arguments keep the caller's state in registers.
template <int VR>
__device__ __noinline__ bool chol32_append(const float* G32, int N, float* L, float* invd,
                                           int nf, int n, const int16_t* atoms, int lane) {
  for (int i = nf; i < n; ++i) {
    const size_t row = (size_t)atoms[i] * N;
    float g[VR];
#pragma unroll
    for (int k = 0; k < VR; ++k) {
      const int t = lane + 32 * k;
      const int col = atoms[min(t, i)];
      const float v = __ldg(G32 + row + col);
      g[k] = t < i ? v : 0.f;
    }
    const float gii = __ldg(G32 + row + atoms[i]);
    // g := U_{0:i}^{-1} g (the first rows need one register slot)
    if (VR > 1 && i <= 32) fwd_unit<VR, 1>(L, i, g, lane);
    else fwd_unit<VR>(L, i, g, lane);
    float ss = 0.f;
#pragma unroll
    for (int k = 0; k < VR; ++k) {
      const int t = lane + 32 * k;
      if (t < i) {
        const float u = g[k] * invd[t];
        ss = fmaf(g[k], u, ss);
        L[ridx(i, t)] = u;
      }
    }
    const float d = gii - warp_sum(ss);
    if (!(d > 1e-4f * gii)) return false;  // warp-uniform
    if (lane == 0) invd[i] = 1.f / d;
    __syncwarp();
  }
  return true;
}

// Least squares on atoms[0..n) (n <= M): mixed precision first, FP64 factorisation if
// the FP32 factor fails.  b goes to vbuf; Lbuf/invdbuf hold FP32 or FP64 factors.
template <int VR, bool OOL>
__device__ bool ls_solve(Warp& w, const int16_t* atoms, int n, double* Lbuf, double* invdbuf,
                         double* vbuf, double* s, int cap);

// The k largest |val| over atoms lane + 32 kk < nvalid, ties to the lower atom: a bitwise
// search for the k-th largest magnitude (IEEE bits of |v| order like the values), then a
// ballot compaction of everything above it plus the lowest-indexed ties.  32 warp steps
// whatever k is; output in ascending atom order.
__device__ float topk_select_atoms(Warp& w, const float (&val)[kNK], int nvalid, int k,
                                   int16_t* out) {
  const int lane = w.lane;
  unsigned key[kNK];
  bool ok[kNK];
#pragma unroll
  for (int kk = 0; kk < kNK; ++kk) {
    ok[kk] = lane + 32 * kk < nvalid;
    key[kk] = __float_as_uint(fabsf(val[kk]));
  }
  unsigned T = 0;
  for (int b = 31; b >= 0; --b) {
    unsigned cand = T | (1u << b), cnt = 0;
#pragma unroll
    for (int kk = 0; kk < kNK; ++kk) cnt += (ok[kk] && key[kk] >= cand) ? 1u : 0u;
    if (__reduce_add_sync(0xffffffffu, cnt) >= (unsigned)k) T = cand;
  }
  unsigned gt = 0;
#pragma unroll
  for (int kk = 0; kk < kNK; ++kk) gt += (ok[kk] && key[kk] > T) ? 1u : 0u;
  const int need = k - (int)__reduce_add_sync(0xffffffffu, gt);
  const unsigned below = (1u << lane) - 1u;
  int pos = 0, eq_before = 0;
#pragma unroll
  for (int kk = 0; kk < kNK; ++kk) {
    bool isgt = ok[kk] && key[kk] > T, iseq = ok[kk] && key[kk] == T;
    unsigned eqm = __ballot_sync(0xffffffffu, iseq);
    bool take = isgt || (iseq && eq_before + __popc(eqm & below) < need);
    unsigned tm = __ballot_sync(0xffffffffu, take);
    if (take) out[pos + __popc(tm & below)] = (int16_t)(lane + 32 * kk);
    pos += __popc(tm);
    eq_before += __popc(eqm);
  }
  __syncwarp();
  return __uint_as_float(T);
}

// The k largest |vals[p]| over positions p < cnt (FP64, ties to the lower position) by
// rank counting: each position counts the positions that beat it -- a larger magnitude
// (compared as IEEE bit patterns, which order like the values), or an equal one at a
// lower position -- and is chosen when fewer than k do.  The order is total, so exactly
// min(k, cnt) positions are chosen, NaN included.  Output in ascending position order.
__device__ __forceinline__ void topk_positions_body(const double* vals, int cnt, int k,
                                                    int16_t* out, int lane) {
  const unsigned below = (1u << lane) - 1u;
  const unsigned long long mag = 0x7fffffffffffffffull;
  int pos = 0;
  for (int b0 = 0; b0 < cnt; b0 += 64) {  // two positions per lane per pass
    const int p0 = b0 + lane, p1 = b0 + 32 + lane;
    const unsigned long long k0 =
        p0 < cnt ? (unsigned long long)__double_as_longlong(vals[p0]) & mag : 0ull;
    const unsigned long long k1 =
        p1 < cnt ? (unsigned long long)__double_as_longlong(vals[p1]) & mag : 0ull;
    int r0 = 0, r1 = 0;
    for (int i = 0; i < cnt; ++i) {
      const unsigned long long ki = (unsigned long long)__double_as_longlong(vals[i]) & mag;
      r0 += (ki > k0 || (ki == k0 && i < p0)) ? 1 : 0;
      r1 += (ki > k1 || (ki == k1 && i < p1)) ? 1 : 0;
    }
    const bool t0 = p0 < cnt && r0 < k, t1 = p1 < cnt && r1 < k;
    const unsigned m0 = __ballot_sync(0xffffffffu, t0);
    if (t0) out[pos + __popc(m0 & below)] = (int16_t)p0;
    pos += __popc(m0);
    const unsigned m1 = __ballot_sync(0xffffffffu, t1);
    if (t1) out[pos + __popc(m1 & below)] = (int16_t)p1;
    pos += __popc(m1);
  }
  __syncwarp();
}

__device__ __forceinline__ void topk_select_positions(Warp& w, const double* vals, int cnt, int k,
                                                     int16_t* out) {
  topk_positions_body(vals, cnt, k, out, w.lane);
}
// The same, one out-of-line copy (CoSaMP, as ensure_rhs_ool).
__device__ __noinline__ void topk_select_positions_ool(const double* vals, int cnt, int k,
                                                      int16_t* out, int lane) {
  topk_positions_body(vals, cnt, k, out, lane);
}

// k rounds of warp argmax over the lane-held values val[kk] (atom lane + 32 kk, only
// atoms < nvalid compete): largest |val| first, ties to the lower atom; NaN ranks below
// every number, so k distinct atoms are always chosen.  Writes them to out[0..k).
__device__ float topk_atoms(Warp& w, const float (&val)[kNK], int nvalid, int k, int16_t* out) {
  unsigned taken = 0;
  float bv = -2.f;
  for (int j = 0; j < k; ++j) {
    bv = -2.f;
    int bn = 1 << 30;
#pragma unroll
    for (int kk = 0; kk < kNK; ++kk) {
      int n = w.lane + 32 * kk;
      if (n < nvalid && !((taken >> kk) & 1u)) {
        float a = isnan(val[kk]) ? -1.f : fabsf(val[kk]);
        if (a > bv || (a == bv && n < bn)) {
          bv = a;
          bn = n;
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      float ov = __shfl_xor_sync(0xffffffffu, bv, o);
      int on = __shfl_xor_sync(0xffffffffu, bn, o);
      if (ov > bv || (ov == bv && on < bn)) {
        bv = ov;
        bn = on;
      }
    }
    if ((bn & 31) == w.lane) taken |= 1u << (bn >> 5);
    if (w.lane == 0) out[j] = (int16_t)bn;
  }
  __syncwarp();
  return bv;
}

// Makes a top-k choice taken on FP32 values equal to the one FP64 arithmetic takes.
// Every |val| lies within E of the FP64 magnitude it approximates, and t is the k-th
// largest |val|.  An atom more than 2E above t beats every atom at or below t in FP64,
// and fewer than k atoms lie above t, so it is chosen; an atom more than 2E below t
// loses to the k (or more) atoms at or above t, so it is not.  When the band between
// holds more atoms than the slots left, the band is recomputed in FP64 (exact64(atom))
// and the slots go to its largest magnitudes, ties to the lower atom, by a bitwise
// search on the FP64 patterns.  out[0..k) is rewritten in ascending atom order.  Skipped
// when a value is not finite (the pixel is flagged non-finite elsewhere).
template <typename F>
__device__ void certify_topk(Warp& w, const float (&val)[kNK], int nvalid, int k, float t,
                             float E, F exact64, int16_t* out) {
  const int lane = w.lane;
  if (!(isfinite(t) && isfinite(E))) return;  // warp-uniform
  // half-width 2E, widened for the FP32 rounding of the band edges themselves
  const float W = 2.01f * E + t * 0x1p-21f;
  const float hi = t + W, lo = t - W;
  unsigned nin = 0, nband = 0;
  bool fin = true;
#pragma unroll
  for (int kk = 0; kk < kNK; ++kk) {
    if (lane + 32 * kk < nvalid) {
      const float a = fabsf(val[kk]);
      fin &= isfinite(a);
      nin += a > hi ? 1u : 0u;
      nband += (a >= lo && a <= hi) ? 1u : 0u;
    }
  }
  if (!__all_sync(0xffffffffu, fin)) return;
  nin = __reduce_add_sync(0xffffffffu, nin);
  nband = __reduce_add_sync(0xffffffffu, nband);
  if (nin + nband <= (unsigned)k) return;  // every atom of the band is chosen: certain
  unsigned long long key[kNK];
  bool ok[kNK];
#pragma unroll
  for (int kk = 0; kk < kNK; ++kk) {
    const int n = lane + 32 * kk;
    const float a = fabsf(val[kk]);
    ok[kk] = n < nvalid && a >= lo;
    key[kk] = 0ull;
    if (ok[kk]) {
      key[kk] = a > hi ? 0x7ff0000000000000ull  // surely chosen: above any finite value
                       : (unsigned long long)__double_as_longlong(fabs(exact64(n)));
    }
  }
  unsigned long long T = 0;
  for (int b = 63; b >= 0; --b) {
    unsigned long long cand = T | (1ull << b);
    unsigned c = 0;
#pragma unroll
    for (int kk = 0; kk < kNK; ++kk) c += (ok[kk] && key[kk] >= cand) ? 1u : 0u;
    if (__reduce_add_sync(0xffffffffu, c) >= (unsigned)k) T = cand;
  }
  unsigned gt = 0;
#pragma unroll
  for (int kk = 0; kk < kNK; ++kk) gt += (ok[kk] && key[kk] > T) ? 1u : 0u;
  const int need = k - (int)__reduce_add_sync(0xffffffffu, gt);
  const unsigned below = (1u << lane) - 1u;
  int pos = 0, eq_before = 0;
  __syncwarp();
#pragma unroll
  for (int kk = 0; kk < kNK; ++kk) {
    bool isgt = ok[kk] && key[kk] > T, iseq = ok[kk] && key[kk] == T;
    unsigned eqm = __ballot_sync(0xffffffffu, iseq);
    bool take = isgt || (iseq && eq_before + __popc(eqm & below) < need);
    unsigned tm = __ballot_sync(0xffffffffu, take);
    if (take) out[pos + __popc(tm & below)] = (int16_t)(lane + 32 * kk);
    pos += __popc(tm);
    eq_before += __popc(eqm);
  }
  __syncwarp();
}

// Fresh factorisation of the normal equations on atoms[0..n) and solve into s.
__device__ __noinline__ bool ls_fresh_impl(const int16_t* atoms, int n, double* L, double* invd,
                                           double* v, double* s, int cap, const double* G,
                                           int N, const double* bx, double* wv, int lane) {
  bool ok = true;
  for (int k = 0; k < n; ++k) {
    const double* grow = G + (size_t)atoms[k] * N;
    ok &= append_row(lane, wv, L, invd, v, cap, k, [&](int t) { return grow[atoms[t]]; },
                     bx[atoms[k]]);
    if (!ok) return false;
  }
  back_solve(lane, L, invd, v, s, cap, n);
  return true;
}
__device__ __forceinline__ bool ls_fresh(Warp& w, const int16_t* atoms, int n, double* L,
                                         double* invd, double* v, double* s, int cap) {
  return ls_fresh_impl(atoms, n, L, invd, v, s, cap, w.cb->G64, w.cb->N, w.bx, w.wv, w.lane);
}
// The FP64 fallback in the warp's global slot: factor, inverse pivots, forward solution
// and the row scratch of append_row, for systems of up to dmax rows.
__device__ __forceinline__ bool ls_fresh_global(Warp& w, const int16_t* atoms, int n, double* s) {
  const int D = w.p.dmax;
  double* Lg = w.fb;
  double* inv = Lg + D * (D + 1) / 2;
  return ls_fresh_impl(atoms, n, Lg, inv, inv + D, s, D, w.cb->G64, w.cb->N, w.bx, inv + 2 * D,
                       w.lane);
}

template <int VR, bool OOL>
__device__ bool ls_solve(Warp& w, const int16_t* atoms, int n, double* Lbuf, double* invdbuf,
                         double* vbuf, double* s, int cap) {
  float* L32 = reinterpret_cast<float*>(Lbuf);
  float* inv32 = reinterpret_cast<float*>(invdbuf);
  if (chol32<VR>(w, L32, inv32, n, atoms) &&
      refine<VR, OOL>(L32, inv32, n, atoms, s, w.bx, w.cb->G64, w.cb->N, w.lane))
    return true;
  // FP64 fallback: in place when the shared regions are FP64-sized, else in the warp's
  // global slot (capacity dmax >= n)
  if (w.fb) {
    return ls_fresh_global(w, atoms, n, s);
  }
  return ls_fresh(w, atoms, n, Lbuf, invdbuf, vbuf, s, cap);
}

// Least squares on a support that only grows (gOMP): the FP32 factor of its first nf
// atoms carries over from the last call and is extended to n rows; nf is updated to the
// rows it holds afterwards (0 when the factor must be rebuilt).
template <int VR>
__device__ bool ls_solve_grow(Warp& w, const int16_t* atoms, int& nf, int n, double* Lbuf,
                              double* invdbuf, double* vbuf, double* s, int cap) {
  if (n > w.p.d32 && w.fb) {
    // the support outgrew the shared-memory factor: FP64 in the warp's global slot
    nf = 0;
    return ls_fresh_global(w, atoms, n, s);
  }
  float* L32 = reinterpret_cast<float*>(Lbuf);
  float* inv32 = reinterpret_cast<float*>(invdbuf);
  const bool factored = chol32_append<VR>(w.cb->G32, w.cb->N, L32, inv32, nf, n, atoms, w.lane);
  nf = factored ? n : 0;
  if (factored && refine<VR, true>(L32, inv32, n, atoms, s, w.bx, w.cb->G64, w.cb->N, w.lane))
    return true;
  if (w.fb) {
    return ls_fresh_global(w, atoms, n, s);
  }
  nf = 0;  // the FP64 fallback below overwrites the FP32 factor's region
  return ls_fresh(w, atoms, n, Lbuf, invdbuf, vbuf, s, cap);
}

// gOMP's refit on the kept atoms q: the FP32 factor Lq of the last refit holds the atoms
// qf[0..nqf) in that order, and rows of a Cholesky factor depend only on the rows before
// them, so the rows of the longest common prefix of q and qf are kept and only the rest
// is appended (q keeps c's arrival order, and the strongest atoms, which stay, arrive
// first).  nqf is updated to the rows Lq holds afterwards.  An unchanged q reuses the
// whole factor and so reproduces the last solution bit for bit.
template <int VR>
__device__ bool ls_solve_refit(Warp& w, const int16_t* q, int n, int& nqf, double* Lbuf,
                               double* invdbuf, double* vbuf, double* s, int cap) {
  const int lane = w.lane;
  int pre = 0;
  const int common = min(n, nqf);
  for (int t0 = 0; t0 < common; t0 += 32) {
    const int t = t0 + lane;
    const unsigned diff = __ballot_sync(0xffffffffu, t < common && q[t] != w.qf[t]);
    if (diff) {
      pre = t0 + __ffs(diff) - 1;
      break;
    }
    pre = min(t0 + 32, common);
  }
  __syncwarp();
  float* L32 = reinterpret_cast<float*>(Lbuf);
  float* inv32 = reinterpret_cast<float*>(invdbuf);
  const bool factored = chol32_append<VR>(w.cb->G32, w.cb->N, L32, inv32, pre, n, q, lane);
  for (int t = pre + lane; t < n; t += 32) w.qf[t] = q[t];
  nqf = factored ? n : 0;
  __syncwarp();
  if (factored && refine<VR, true>(L32, inv32, n, q, s, w.bx, w.cb->G64, w.cb->N, lane))
    return true;
  if (w.fb) {
    return ls_fresh_global(w, q, n, s);
  }
  nqf = 0;  // the FP64 fallback below overwrites the FP32 factor's region
  return ls_fresh(w, q, n, Lbuf, invdbuf, vbuf, s, cap);
}

// Minimum-norm solution for |c| > M: s = A_c^T H^{-1} y with H = A_c A_c^T (M x M).
__device__ bool ls_min_norm(Warp& w, const int16_t* atoms, int n, double* s) {
  const int M = w.cb->M;
  const double* At = w.cb->At64;
  // FP64 M x M factor: the warp's global slot (dmax = M here), else the FP64-sized smem
  double* L = w.fb ? w.fb : w.L;
  double* invd = w.fb ? w.fb + M * (M + 1) / 2 : w.invd;
  double* v = w.fb ? w.fb + M * (M + 1) / 2 + M : w.v;
  double* wv = w.fb ? w.fb + M * (M + 1) / 2 + 2 * M : w.wv;
  const int cap = M;
  bool ok = true;
  for (int k = 0; k < M; ++k) {
    // row k of H: H(k, t) = sum_j A[k][c_j] A[t][c_j]
    ok &= append_row(
        w.lane, wv, L, invd, v, cap, k,
        [&](int t) {
          double h = 0.0;
          for (int j = 0; j < n; ++j) {
            const double* a = At + (size_t)atoms[j] * M;
            h += a[k] * a[t];
          }
          return h;
        },
        (double)w.y[k]);
    if (!ok) return false;
  }
  double* zv = w.svals;  // z = H^{-1} y
  back_solve(w.lane, L, invd, v, zv, cap, M);
  for (int j = w.lane; j < n; j += 32) {
    double acc = 0.0;
    const double* a = At + (size_t)atoms[j] * M;
    for (int m = 0; m < M; ++m) acc += a[m] * zv[m];
    s[j] = acc;
  }
  __syncwarp();
  return true;
}

// SplitMix64's output mixing function (Steele, Lea and Flood, OOPSLA 2014).
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// 64-bit hash of the iterate x (its nq kept atoms w.q and values w.xq, bit patterns and
// positions), the same on every lane.  A match only nominates a cycle; the cycle search
// confirms it bit for bit.
__device__ unsigned long long iterate_hash(Warp& w, int nq) {
  unsigned long long h = 0;
  for (int j = w.lane; j < nq; j += 32)
    h ^= mix64(mix64((unsigned long long)__double_as_longlong(w.xq[j])) ^
               ((unsigned long long)(uint16_t)w.q[j] | ((unsigned long long)j << 16)));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) h ^= __shfl_xor_sync(0xffffffffu, h, o);
  return h ^ mix64(0x5eedull + (unsigned long long)nq);
}

// Complex data on the real form (PR): the selection key of complex atom j is the modulus
// of the column pair (2j, 2j + 1).  val[] holds the columns (lane l: columns l + 32 kk);
// afterwards it holds the moduli of the complex atoms l + 32 kk for kk < kNK / 2 (the
// pair (2j, 2j + 1) sits in lanes 2 (j mod 16), + 1 at slot 2 (j / 32) + (j mod 32 >= 16))
// and 0 above.  FP32: within sqrt(2) E + 4 u |m| of the modulus when each column is
// within E of its value.
__device__ __forceinline__ void pair_moduli(float (&val)[kNK], int lane) {
  float m2[kNK];
#pragma unroll
  for (int kk = 0; kk < kNK; ++kk) {
    const float o = __shfl_xor_sync(0xffffffffu, val[kk], 1);
    m2[kk] = fmaf(val[kk], val[kk], o * o);
  }
  const int src = 2 * (lane & 15);
  const bool upper = lane >= 16;
#pragma unroll
  for (int kk = 0; kk < kNK / 2; ++kk) {
    const float a = __shfl_sync(0xffffffffu, m2[2 * kk], src);
    const float b = __shfl_sync(0xffffffffu, m2[2 * kk + 1], src);
    val[kk] = sqrtf(upper ? b : a);
  }
#pragma unroll
  for (int kk = kNK / 2; kk < kNK; ++kk) val[kk] = 0.f;
}

template <int ALGO, int VR, bool PR = false>
__global__ void __launch_bounds__(256, 2) k_greedy(GrParams p) {
  extern __shared__ __align__(16) unsigned char gsm[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  Layout lay(p.Mmax, p.Nmax, p.cmax, p.dmax, p.kmax, p.selmax, p.fb64 == nullptr,
             ALGO == kGomp, ALGO != kGomp, ALGO == kBiht, p.d32, PR);
  unsigned char* base = gsm + (size_t)wid * p.warp_bytes;
  Warp w{p, lane, p.cubes};
  w.y = (float*)(base + lay.y);
  w.rf = (float*)(base + lay.rf);
  w.xd = (float*)(base + lay.xd);
  w.b32 = (float*)(base + lay.b32);
  w.xqf = (float*)(base + lay.xqf);
  w.bx = (double*)(base + lay.bx);
  w.y64 = (double*)(base + lay.y64);
  w.xq = (double*)(base + lay.xq);
  w.xqp = (double*)(base + lay.xqp);
  w.L = (double*)(base + lay.L);
  w.invd = (double*)(base + lay.invd);
  w.v = (double*)(base + lay.v);
  w.s = (double*)(base + lay.s);
  w.wv = (double*)(base + lay.wv);
  w.Lq = (double*)(base + lay.Lq);
  w.invq = (double*)(base + lay.invq);
  w.vq = (double*)(base + lay.vq);
  w.sq = (double*)(base + lay.sq);
  w.svals = (double*)(base + lay.svals);
  double* const cyc_x = (double*)(base + lay.cx);
  int16_t* const cyc_q = (int16_t*)(base + lay.cq);
  unsigned long long* const ring = (unsigned long long*)(base + lay.ring);
  w.inc = base + lay.inc;
  w.bk = base + lay.bk;
  w.c = (int16_t*)(base + lay.c);
  w.q = (int16_t*)(base + lay.q);
  w.qp = (int16_t*)(base + lay.qp);
  w.qf = (int16_t*)(base + lay.qf);
  w.sel = (int16_t*)(base + lay.sel);
  w.fb = p.fb64 ? p.fb64 + (size_t)(blockIdx.x * (blockDim.x >> 5) + wid) * p.fb_slot : nullptr;

  for (int n = lane; n < p.Nmax; n += 32) {
    if (ALGO == kBiht) w.xd[n] = 0.f;
    w.inc[n] = 0;
    w.bk[n] = 0;
  }
  __syncwarp();
  int cur = -1;        // cube whose data w.cb holds
  float cnorm = 0.f;   // its largest column norm, rounded up
  constexpr float u32 = 0x1p-24f;

  for (;;) {
    unsigned long long pix_u = 0;
    if (lane == 0) pix_u = atomicAdd(p.counter, 1ull);
    pix_u = __shfl_sync(0xffffffffu, pix_u, 0);
    if (pix_u >= (unsigned long long)p.total) break;
    // the pixel's cube: the last one starting at or before it (warp-uniform search)
    int ci = 0;
    if (p.ncubes > 1) {
      int lo = 0, hi = p.ncubes - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((unsigned long long)p.cubes[mid].pix0 <= pix_u) lo = mid;
        else hi = mid - 1;
      }
      ci = lo;
    }
    if (ci != cur) {
      w.cb = p.cubes + ci;
      cur = ci;
      // largest column norm of A (square root of the Gram matrix's largest diagonal
      // entry), rounded up: the FP32 error bounds of the correlation and the residual
      float cn2 = 0.f;
      for (int n = lane; n < w.cb->N; n += 32) cn2 = fmaxf(cn2, w.cb->G32[(size_t)n * w.cb->N + n]);
      cnorm = __fsqrt_ru(warp_max(cn2) * 1.0000005f) * 1.000001f;
    }
    const GrCube& cb = *w.cb;
    const int M = cb.M, N = cb.N;
    const int64_t pix = (int64_t)pix_u - cb.pix0;
    const float gmax = cnorm * cnorm * 1.000001f;  // bounds every |(A^T A)_jk|

    // a per-pixel level outside 0..kappa bound is clamped: the workspace holds kmax atoms
    // (complex data, PR: kappa, G and the selections count complex atoms, each the pair of
    // real-form columns 2j, 2j + 1; the workspace counts columns)
    const int kbound = PR ? p.kmax / 2 : p.kmax;
    const int kappa = cb.kappa_pp ? min(max((int)cb.kappa_pp[pix], 0), kbound) : p.kappa;
    const int G = p.G > 0 ? p.G : (kappa / 5 > 1 ? kappa / 5 : 1);
    int cap = p.max_iters;
    if (ALGO == kGomp) {
      const int Mc = PR ? M / 2 : M;
      if (kappa < cap) cap = kappa;
      if (Mc / G < cap) cap = Mc / G;
    }
    bool bad = false;
    float y2 = 0.f;
    for (int m = lane; m < M; m += 32) {
      float yv = cb.Y[pix * M + m];
      bad |= !isfinite(yv);
      w.y[m] = yv;
      w.y64[m] = (double)yv;
      w.rf[m] = yv;  // r^0 = y
      y2 = fmaf(yv, yv, y2);
    }
    const bool bad_pixel = __any_sync(0xffffffffu, bad);
    if (bad_pixel && lane == 0) atomicOr(p.status, kStNonFinite);
    // ||y||_2 rounded up (with room for the M roundings of the sum of squares)
    const float ynorm = __fsqrt_ru(warp_sum(y2) * (1.f + (M + 2) * u32)) * 1.000001f;
    __syncwarp();
    if (!p.start_done && cap > 0) load_rhs32(w);

    int nc = 0, nq = 0, nqp = 0, it = 0;
    int nf = 0;  // gOMP: rows of the FP32 factor of G_c carried over between iterations
    int nqf = 0;  // gOMP: rows of the refit factor of G_q carried over between iterations
    float x1 = 0.f;     // sum |x_q| of the current iterate, rounded up
    float rerr = 0.f;   // error bound of the FP32 residual of the current iterate (r^0 = y)
    uint8_t conv = 0;
    // cycle search over the iterates x_it (BIHT, CoSaMP): ring[it % 32] holds a hash of
    // x_it; a hash seen `period` iterations ago nominates a cycle, which is confirmed by
    // comparing x bit for bit one period later (verify_at); `full` is the cap reported
    int saved_n = 0, full = 0, period = 0, verify_at = -1;
    bool cycled = false;
    if (ALGO != kGomp) {
      const unsigned long long h0 = iterate_hash(w, 0);  // x_0 = 0 (all lanes shuffle)
      if (lane == 0) ring[0] = h0;
      __syncwarp();
    }
    // algorithmic flops of the method for this pixel, times 3 (an integer; integer
    // arithmetic keeps the count off the FP64 pipe): correlation 2MN, Cholesky least
    // squares n^3/3 + 2n^2 per support of n atoms (min-norm form for n > M), residual 2M|q|
    long long work3 = 0;
    bool fail = false;
    while (!p.start_done && it < cap) {
      // ---- step 1: correlation p = A^T r = A^T y - (A^T A)_{:,q} x_q (u = x + mu p for
      //      BIHT): lane l owns atoms l + 32 kk; row q_t of the Gram matrix is column q_t
      float val[kNK];
#pragma unroll
      for (int kk = 0; kk < kNK; ++kk) {
        const int n = lane + 32 * kk;
        val[kk] = n < N ? w.b32[n] : 0.f;
      }
      // rows of the Gram matrix in flight: BIHT gains from four; gOMP's larger hot loop
      // loses instruction-cache hits with more than two
#pragma unroll(ALGO == kBiht ? 4 : 2)
      for (int t = 0; t < nq; ++t) {
        const float xt = w.xqf[t];
        const float* grow = cb.G32 + (size_t)w.q[t] * N;
#pragma unroll
        for (int kk = 0; kk < kNK; ++kk) {
          const int n = lane + 32 * kk;
          if (n < N) val[kk] = fmaf(-__ldg(grow + n), xt, val[kk]);
        }
      }
      // FP32 error bound of p_j: A^T y errs by at most (M + 2) u ||A_j|| ||y|| (rounded A,
      // M rounded FMAs), the |q| FMAs of the Gram part by (|q| + 3) u sum_t |G_jt| |x_t|
      // <= (|q| + 3) u gmax ||x||_1 (rounded G and x included) plus |q| u |A^T y|; the 1%
      // margin covers the FP32 evaluation of the bound itself
      const float pbound =
          ((M + nq + 2) * cnorm * ynorm + (nq + 3) * gmax * x1) * u32 * 1.01f;
      if (ALGO == kBiht) {
#pragma unroll
        for (int kk = 0; kk < kNK; ++kk) {
          int n = lane + 32 * kk;
          if (n < N) val[kk] = w.xd[n] + p.mu * val[kk];
        }
      }
      const int ksel = ALGO == kGomp ? G : (ALGO == kCosamp ? 2 * kappa : kappa);
      // the exact value of an atom's selection key, in FP64: p_j = (A^T y)_j -
      // sum_t G(j, q_t) x_t (the certification's recompute of the band)
      auto exact_p = [&](int j) {
        const double* a = cb.At64 + (size_t)j * M;
        const double* grow = cb.G64 + (size_t)j * N;
        double g = 0.0;
        for (int m = 0; m < M; ++m) g += a[m] * (double)w.y[m];
        for (int t = 0; t < nq; ++t) g -= grow[w.q[t]] * w.xq[t];
        return g;
      };
      // BIHT's key u = x + mu p in FP64
      auto exact_u = [&](int j) {
        double xj = 0.0;
        for (int t = 0; t < nq; ++t)
          if (w.q[t] == j) xj = w.xq[t];
        return xj + p.mu64 * exact_p(j);
      };
      // every column's FP32 key lies within pbound (gOMP, CoSaMP) or this bound (BIHT) of
      // its FP64 value
      auto biht_bound = [&]() {
        // u = x + mu p adds the roundings of x, mu and of the update itself
        float um = 0.f, xm = 0.f;
#pragma unroll
        for (int kk = 0; kk < kNK; ++kk) {
          int n = lane + 32 * kk;
          if (n < N) {
            um = fmaxf(um, fabsf(val[kk]));
            xm = fmaxf(xm, fabsf(w.xd[n]));
          }
        }
        um = warp_max(um);
        xm = warp_max(xm);
        const float mu_up = fabsf(p.mu) * 1.000001f;  // |mu| rounded to FP32, and up
        // |p_j| <= ||A_j|| ||y|| + gmax ||x||_1 bounds the FP32 product's magnitude
        const float pm = cnorm * ynorm + gmax * x1;
        return mu_up * pbound + u32 * 1.01f * (um + xm + mu_up * pm);
      };
      if (PR) {
        // complex atoms: moduli of the column pairs, ranked with the FP64 modulus
        const float Ecol = ALGO == kBiht ? biht_bound() : pbound;
        pair_moduli(val, lane);
        float mm = 0.f;
#pragma unroll
        for (int kk = 0; kk < kNK / 2; ++kk) mm = fmaxf(mm, val[kk]);
        const float Emod = 1.4143f * Ecol + 0x1p-22f * warp_max(mm);
        const float tk = ksel > 8 ? topk_select_atoms(w, val, N / 2, ksel, w.sel)
                                  : topk_atoms(w, val, N / 2, ksel, w.sel);
        if (ALGO == kBiht)
          certify_topk(w, val, N / 2, ksel, tk, Emod * 1.001f,
                       [&](int j) { return hypot(exact_u(2 * j), exact_u(2 * j + 1)); }, w.sel);
        else
          certify_topk(w, val, N / 2, ksel, tk, Emod * 1.001f,
                       [&](int j) { return hypot(exact_p(2 * j), exact_p(2 * j + 1)); }, w.sel);
      } else {
        const float tk = ksel > 8 ? topk_select_atoms(w, val, N, ksel, w.sel)
                                  : topk_atoms(w, val, N, ksel, w.sel);
        if (ALGO == kBiht)
          certify_topk(w, val, N, ksel, tk, biht_bound() * 1.001f, exact_u, w.sel);
        else
          certify_topk(w, val, N, ksel, tk, pbound * 1.001f, exact_p, w.sel);
      }

      // ---- support c = Theta U c (gOMP: the growing support, new atoms appended in
      // selection order so its factor can be extended; CoSaMP: the last pruned support;
      // BIHT: supp(x)), marked in inc[]; CoSaMP's and BIHT's c in ascending atom order ----
      if (ALGO == kGomp) {
        const unsigned below = (1u << lane) - 1u;
        constexpr int kw = PR ? 2 : 1;  // columns per atom
        for (int b0 = 0; b0 < ksel; b0 += 32) {
          const int j = b0 + lane;
          const int a = kw * (j < ksel ? w.sel[j] : 0);  // the atom's first column
          const bool isnew = j < ksel && !w.inc[a];
          const unsigned m = __ballot_sync(0xffffffffu, isnew);
          if (isnew) {
            const int at = nc + kw * __popc(m & below);
            w.c[at] = (int16_t)a;
            w.inc[a] = 1;
            if (PR) {
              w.c[at + 1] = (int16_t)(a + 1);
              w.inc[a + 1] = 1;
            }
          }
          nc += kw * __popc(m);
          __syncwarp();
        }
      }
      if (ALGO == kBiht) {
        for (int n = lane; n < N; n += 32) w.inc[n] = 0;
        __syncwarp();
        for (int j = lane; j < nq; j += 32)
          if (w.xq[j] != 0.0) {
            w.inc[w.q[j]] = 1;
            if (PR) w.inc[w.q[j] ^ 1] = 1;  // a complex atom is in supp(x) by its modulus
          }
      }
      if (ALGO != kGomp) {
        for (int j = lane; j < ksel; j += 32) {
          if (PR) {
            w.inc[2 * w.sel[j]] = 1;
            w.inc[2 * w.sel[j] + 1] = 1;
          } else {
            w.inc[w.sel[j]] = 1;
          }
        }
        __syncwarp();
        const unsigned below = (1u << lane) - 1u;
        int cnt = 0;
        for (int a0 = 0; a0 < N; a0 += 32) {
          const int a = a0 + lane;
          const bool in = a < N && w.inc[a];
          const unsigned m = __ballot_sync(0xffffffffu, in);
          if (in) w.c[cnt + __popc(m & below)] = (int16_t)a;
          cnt += __popc(m);
        }
        nc = cnt;
        __syncwarp();
      }
      // (A^T y)_c as FP32 pairs for the least squares (new atoms only)
      if (ALGO == kCosamp && VR >= 3)
        ensure_rhs_ool(cb.At64, M, w.y64, w.bx, w.bk, w.c, nc, lane);
      else
        ensure_rhs(w, w.c, nc);

      // ---- step 2: least squares on c ----
      const int nf0 = nf;
      if (nc > 0) {
        if (ALGO == kGomp)
          fail |= !ls_solve_grow<VR>(w, w.c, nf, nc, w.L, w.invd, w.v, w.s, p.dmax);
        else if (nc <= M)
          fail |= !ls_solve<VR, false>(w, w.c, nc, w.L, w.invd, w.v, w.s, p.dmax);
        else
          fail |= !ls_min_norm(w, w.c, nc, w.s);
      }
      if (fail) break;
      {
        const long long n = nc, m = M;
        long long ls3;
        if (ALGO == kGomp) {
          // rows appended to the factor: a forward sweep of i^2 flops for row i, i in
          // [a, b); (b-1) b (2b-1) is a multiple of 6
          const long long a = nf0, b = nc;
          ls3 = ((b - 1) * b * (2 * b - 1) - (a - 1) * a * (2 * a - 1)) / 2 + 6 * n * n;
        } else {
          ls3 = nc <= M ? n * n * n + 6 * n * n
                        : 3 * n * m * m + m * m * m + 6 * m * m + 3 * n * m;
        }
        work3 += 6 * m * N + ls3;
      }

      // ---- step 3: prune to kappa (and refit for gOMP) ----
      // the previous iterate, for Delta; BIHT's leaves xd
      for (int j = lane; j < nq; j += 32) {
        w.qp[j] = w.q[j];
        w.xqp[j] = w.xq[j];
        if (ALGO == kBiht) w.xd[w.q[j]] = 0.f;
      }
      nqp = nq;
      __syncwarp();
      int keep;  // columns kept
      if (PR) {
        // complex atoms (column pairs at positions 2i, 2i + 1 of c) ranked by the FP64
        // modulus of their coefficient
        const int np = nc / 2, keepp = np < kappa ? np : kappa;
        if (np > kappa) {
          for (int i = lane; i < np; i += 32) w.svals[i] = hypot(w.s[2 * i], w.s[2 * i + 1]);
          __syncwarp();
          topk_select_positions(w, w.svals, np, keepp, w.sel);
        } else {
          for (int i = lane; i < np; i += 32) w.sel[i] = (int16_t)i;
          __syncwarp();
        }
        keep = 2 * keepp;
        for (int j = lane; j < keep; j += 32) {
          const int pos = 2 * w.sel[j >> 1] + (j & 1);
          w.q[j] = w.c[pos];
          w.xq[j] = w.s[pos];
        }
      } else {
        keep = nc < kappa ? nc : kappa;
        if (nc > kappa) {
          // ascending positions of c
          if (ALGO == kCosamp && VR >= 3) topk_select_positions_ool(w.s, nc, keep, w.sel, lane);
          else topk_select_positions(w, w.s, nc, keep, w.sel);
        } else {
          for (int j = lane; j < nc; j += 32) w.sel[j] = (int16_t)j;
          __syncwarp();
        }
        for (int j = lane; j < keep; j += 32) {
          int pos = w.sel[j];
          w.q[j] = w.c[pos];
          w.xq[j] = w.s[pos];
        }
      }
      __syncwarp();
      nq = keep;  // q keeps the order of c
      // the refit on q; when q is all of c (in c's order) it would repeat the solve just
      // made, bit for bit, so x keeps that solution
      if (ALGO == kGomp && nq > 0 && nq < nc) {
        fail |= !ls_solve_refit<VR>(w, w.q, nq, nqf, w.Lq, w.invq, w.vq, w.sq, p.kmax);
        work3 += (long long)nq * nq * nq + 6ll * nq * nq;
        if (fail) break;
        for (int j = lane; j < nq; j += 32) w.xq[j] = w.sq[j];
        __syncwarp();
      }
      if (ALGO == kCosamp) {
        // c = c(q)
        for (int j = lane; j < nc; j += 32) w.inc[w.c[j]] = 0;
        __syncwarp();
        for (int j = lane; j < nq; j += 32) {
          w.c[j] = w.q[j];
          w.inc[w.q[j]] = 1;
        }
        __syncwarp();
        nc = nq;
      }
      // FP32 copies of x_q (the next correlation and the residual) and ||x||_1
      float xs = 0.f;
      for (int j = lane; j < nq; j += 32) {
        const float xf = (float)w.xq[j];
        w.xqf[j] = xf;
        xs += fabsf(xf);
        if (ALGO == kBiht) w.xd[w.q[j]] = xf;
      }
      x1 = warp_sum(xs) * (1.f + (nq + 2) * u32) * 1.000001f;
      __syncwarp();

      // ---- step 4: r = y - A x (FP32, lanes own rows m = lane + 32 kk; columns of A^T are
      //      contiguous) and the stopping test Delta = ||r - r_prev|| < eps ----
      float d2 = 0.f;
      {
        float acc[4];
        const int mc = M - 1;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) acc[kk] = w.y[min(lane + 32 * kk, mc)];
        // columns in flight: two for gOMP (1% faster than four on 1,048,576 pixels of the
        // 2048^2 x 256 cube: its hot loop is short of instruction-cache room), four for
        // BIHT and CoSaMP
#pragma unroll(ALGO == kGomp ? 2 : 4)
        for (int t = 0; t < nq; ++t) {
          const float* col = cb.At32 + (size_t)w.q[t] * M;
          const float xt = w.xqf[t];
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
            if (32 * kk < M) acc[kk] = fmaf(-__ldg(col + min(lane + 32 * kk, mc)), xt, acc[kk]);
        }
        __syncwarp();
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const int m = lane + 32 * kk;
          if (m < M) {
            const float df = acc[kk] - w.rf[m];
            d2 = fmaf(df, df, d2);
            w.rf[m] = acc[kk];
          }
        }
      }
      d2 = warp_sum(d2);
      work3 += 6ll * M * nq;
      ++it;
      // each FP32 residual errs from r = y - A x by at most (|q| + 3) u (||y|| + ||A_j||max
      // ||x||_1) in norm (rounded A and x, |q| rounded FMAs)
      const float rerr_now = (nq + 3) * u32 * (ynorm + cnorm * x1) * 1.01f;
      bool done_now = false;
      if (p.eps2 > 0.0) {
        // an unchanged iterate reproduces r bit for bit: Delta = 0 exactly
        bool same = nq == nqp;
        if (same) {
          bool eq = true;
          for (int j = lane; j < nq; j += 32)
            eq &= w.q[j] == w.qp[j] &&
                  __double_as_longlong(w.xq[j]) == __double_as_longlong(w.xqp[j]);
          same = __all_sync(0xffffffffu, eq);
        }
        if (same) {
          done_now = true;
        } else {
          const float dl = sqrtf(d2);
          const float E = (rerr_now + rerr) * 1.001f + dl * (M + 4) * u32;
          const double hi = (double)dl + (double)E, lo = (double)dl - (double)E;
          if (hi * hi < p.eps2) {
            done_now = true;
          } else if (!(lo > 0.0 && lo * lo >= p.eps2)) {
            // too close to eps for the FP32 bound: Delta = ||A (x_it - x_it-1)|| in FP64
            double dd = 0.0;
            for (int m = lane; m < M; m += 32) {
              double v = 0.0;
              for (int t = 0; t < nq; ++t) v += cb.At64[(size_t)w.q[t] * M + m] * w.xq[t];
              for (int t = 0; t < nqp; ++t) v -= cb.At64[(size_t)w.qp[t] * M + m] * w.xqp[t];
              dd += v * v;
            }
            done_now = warp_sum(dd) < p.eps2;
          }
        }
      }
      rerr = rerr_now;
      __syncwarp();
      if (done_now) {
        conv = 1;
        break;
      }
      if (ALGO != kGomp && p.cycle_skip && !cycled) {
        // x_it determines everything the next iteration computes (r, the correlation,
        // c, the least squares and the prune run deterministically on it), so once
        // x_{i+period} equals x_i bit for bit the iterates repeat with that period.
        // Every later Delta then repeats one already tested against eps, so only the
        // cap can stop the pixel: run just the iterations that reach the cap's phase of
        // the cycle and report the cap.
        const unsigned long long h = iterate_hash(w, nq);
        if (it == verify_at) {
          bool same = nq == saved_n;
          if (same) {
            bool eq = true;
            for (int j = lane; j < nq; j += 32)
              eq &= cyc_q[j] == w.q[j] &&
                    __double_as_longlong(cyc_x[j]) == __double_as_longlong(w.xq[j]);
            same = __all_sync(0xffffffffu, eq);
          }
          if (same) {
            full = cap;
            cap = it + (cap - it) % period;
            cycled = true;
          }
          verify_at = -1;
        } else if (verify_at < 0) {
          // lane l tests the iterate l + 1 iterations back
          const bool hit = lane + 1 <= it && ring[(it - lane - 1) & 31] == h;
          const unsigned m = __ballot_sync(0xffffffffu, hit);
          if (m) {
            period = __ffs(m);
            for (int j = lane; j < nq; j += 32) {
              cyc_q[j] = w.q[j];
              cyc_x[j] = w.xq[j];
            }
            saved_n = nq;
            verify_at = it + period;
          }
        }
        __syncwarp();
        if (lane == 0) ring[it & 31] = h;
        __syncwarp();
      }
    }
    if (cycled && !fail && conv == 0) it = full;
    if (fail) {
      conv = 2;
      if (lane == 0) atomicOr(p.status, kStNotSpd);
    }
    if (bad_pixel) conv = 3;  // measurements not finite (also latched in the status word)
    // output and reset
    if (ALGO == kBiht) {
      for (int n = lane; n < N; n += 32) {
        cb.X[pix * N + n] = w.xd[n];
        w.xd[n] = 0.f;
        w.inc[n] = 0;
        w.bk[n] = 0;
      }
    } else {
      // x = xq on the atoms q, zero elsewhere
      for (int n = lane; n < N; n += 32) {
        cb.X[pix * N + n] = 0.f;
        w.inc[n] = 0;
        w.bk[n] = 0;
      }
      __syncwarp();
      for (int j = lane; j < nq; j += 32) cb.X[pix * N + w.q[j]] = (float)w.xq[j];
    }
    if (lane == 0) {
      if (cb.iters_out) cb.iters_out[pix] = it;
      if (cb.conv_out) cb.conv_out[pix] = conv;
      if (p.work) atomicAdd(p.work, (double)work3 / 3.0);
    }
    __syncwarp();
  }
}

// The kernel instance whose register-held vectors cover systems of up to 32 vr rows.
template <int ALGO, bool PR = false>
auto greedy_kernel(int vr) {
  if (vr <= 1) return k_greedy<ALGO, 1, PR>;
  if (vr == 2) return k_greedy<ALGO, 2, PR>;
  if (vr == 3) return k_greedy<ALGO, 3, PR>;
  return k_greedy<ALGO, 4, PR>;
}

}  // namespace

// The complex-data (column pair) instance of the greedy kernel for algo and vr register
// slots, as a host function pointer of type void (*)(GrParams) (greedy_pairs.cu).
const void* greedy_pairs_kernel(int algo, int vr);

}  // namespace cs
