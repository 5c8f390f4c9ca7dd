// amg_cycle.cu -- AMG V-cycle (Sec. 5.1: one V-cycle, direct coarse solve)
// and the dense inverse of the coarsest operator.
//
// V(nu_pre, nu_post) with damped Jacobi or Chebyshev smoothing from a zero
// initial guess, restriction R = P^T, prolongation P, and the direct coarse
// solve applied as a dense matrix-vector product with the explicit inverse.
// The kernels are templates on the storage type V of the operator values and
// the compute type C of the vectors: FP64 / FP64 for the plain method, BF16 /
// FP32 for the mixed-precision form (the set-up always runs in FP64; the
// BF16 and FP32 copies are packed from it).
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <mutex>

#include "common.cuh"
#include "vcycle_rows.cuh"

namespace cg = cooperative_groups;

namespace mss {
namespace {

using namespace dev;

// ---- coarse inverse: Gauss-Jordan with partial pivoting ------------------
// M is the n x 2n augmented matrix [A | I] (row-major). Every block finds
// the pivot of column k itself (same data, same decision); rows are not
// swapped, the pivot row of column k is recorded instead. One grid-wide
// barrier per column. The identity half is stored by pivot order: slot k
// holds the identity column of the k-th pivot row, which only becomes nonzero
// when that row is chosen, so step k touches the left columns > k and the
// slots <= k, n entries per row (n^3 multiply-adds in all, not 1.5 n^3).
__global__ void k_gauss_jordan(int n, double* __restrict__ M, int* __restrict__ pivrow,
                               int* __restrict__ status) {
  extern __shared__ unsigned char used[];   // n flags, per block
  __shared__ double s_val[32];
  __shared__ int s_idx[32];
  __shared__ int s_piv;
  cg::grid_group grid = cg::this_grid();
  const int ld = 2 * n;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int i = threadIdx.x; i < n; i += blockDim.x) used[i] = 0;
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    // pivot: largest |M[i][k]| over unused rows, ties to the smaller row
    double best = -1.0;
    int bi = n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      if (used[i]) continue;
      double a = fabs(M[(size_t)i * ld + k]);
      if (a > best || (a == best && i < bi)) { best = a; bi = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      double ob = __shfl_down_sync(0xffffffffu, best, o);
      int oi = __shfl_down_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (lane == 0) { s_val[wid] = best; s_idx[wid] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double b = s_val[0];
      int ii = s_idx[0];
      for (int w = 1; w < nw; ++w)
        if (s_val[w] > b || (s_val[w] == b && s_idx[w] < ii)) { b = s_val[w]; ii = s_idx[w]; }
      s_piv = (b > 0.0 && isfinite(b) && ii < n) ? ii : -1;
    }
    __syncthreads();
    const int p = s_piv;
    if (p < 0) {
      if (blockIdx.x == 0 && threadIdx.x == 0) *status = k + 1;
      return;   // every block reaches the same decision, so none waits below
    }
    if (threadIdx.x == 0) used[p] = 1;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      pivrow[k] = p;
      M[(size_t)p * ld + n + k] = 1.0;   // read from the next step on
    }
    const double* prow = M + (size_t)p * ld;
    const double pk = prow[k];
    for (int i = gwarp; i < n; i += nwarps) {
      if (i == p) continue;
      double* row = M + (size_t)i * ld;
      const double f = row[k] / pk;
      if (f == 0.0) continue;
      // left columns k+1..n-1 and slots 0..k-1; slot k: 0 - f * 1
      for (int j = k + 1 + lane; j < n + k; j += 32) row[j] = fma(-f, prow[j], row[j]);
      if (lane == 0) row[n + k] = -f;
    }
    grid.sync();
    __syncthreads();
  }
}

// slot[c] = the step at which row c was the pivot
__global__ void k_gj_slots(int n, const int* __restrict__ pivrow, int* __restrict__ slot) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) slot[pivrow[k]] = k;
}

// inv[k][c] = (identity column c of the pivot row of column k) / pivot
__global__ void k_gj_extract(int n, const double* __restrict__ M, const int* __restrict__ pivrow,
                             const int* __restrict__ slot, double* __restrict__ inv) {
  long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= (long long)n * n) return;
  int k = (int)(tid / n), c = (int)(tid % n);
  int p = pivrow[k];
  inv[tid] = M[(size_t)p * 2 * n + n + slot[c]] / M[(size_t)p * 2 * n + k];
}

__global__ void k_dense_from_csr(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                 const double* __restrict__ v, double* __restrict__ M) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double* row = M + (size_t)i * 2 * n;
  for (int k = rp[i]; k < rp[i + 1]; ++k) row[ci[k]] = v[k];
}

// ---- coarse inverse: blocked Gauss-Jordan without pivoting -----------------
// In-place inversion by b x b blocks (b = 32): for each diagonal block K,
//   D = A_KK^-1;  A_Kj <- D A_Kj;  A_ij <- A_ij - A_iK A_Kj;  A_iK <- -A_iK D;
//   A_KK <- D   (i, j outside K),
// which leaves A^-1 in place after the last block (n^3 multiply-adds). No
// grid-wide barrier: five ordinary launches per block, so it can run beside
// the other hierarchy's set-up. Without pivoting it needs every diagonal
// block's pivots to stay away from zero; a pivot below 1e-10 times its
// column's magnitude sets *status and the caller falls back to the pivoting
// Gauss-Jordan above.
constexpr int GB = 32;     // block size
constexpr int GT = 32;     // tile of the trailing update
constexpr int GP = 8;      // columns (rows) of the row (column) panel per CTA

__global__ void k_dense_square(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                               const double* __restrict__ v, double* __restrict__ M) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double* row = M + (size_t)i * n;
  for (int k = rp[i]; k < rp[i + 1]; ++k) row[ci[k]] = v[k];
}

// D = A_KK^-1 by Gauss-Jordan in shared memory, one thread per entry
// (GB x GB threads; row r is warp r, so a row's entries, its column-k entry
// included, are read and written by one warp). Per pivot k, warp k has
// formed the reciprocal and the scaled pivot row (double-buffered), one
// block barrier publishes them, every other row is updated, and warp k + 1
// forms the next pivot row from its updated row while the others finish.
__global__ void __launch_bounds__(GB * GB)
k_bgj_diag(int n, const double* __restrict__ M, int k0, int kw, double* __restrict__ D,
           int* __restrict__ status) {
  __shared__ double a[GB][GB + 1];
  __shared__ double cmax[GB];
  __shared__ double prow[2][GB];
  __shared__ int sbad[2];
  const int r = threadIdx.x / GB, c = threadIdx.x % GB;
  a[r][c] = (r < kw && c < kw) ? M[(size_t)(k0 + r) * n + k0 + c] : (r == c ? 1.0 : 0.0);
  __syncthreads();
  if (threadIdx.x < GB) {
    double m = 0.0;
    for (int rr = 0; rr < GB; ++rr) m = fmax(m, fabs(a[rr][threadIdx.x]));
    cmax[threadIdx.x] = m;
  }
  __syncthreads();
  // warp k: pivot k's reciprocal (lane 0) and scaled row into prow[k & 1]
  auto publish = [&](int k) {
    const double p = a[k][k];
    const bool bad = !(fabs(p) > 1e-10 * cmax[k]) || !isfinite(p);
    double ip = 0.0;
    if (c == 0 && !bad) ip = 1.0 / p;
    ip = __shfl_sync(0xffffffffu, ip, 0);
    prow[k & 1][c] = c == k ? ip : a[k][c] * ip;
    if (c == 0) sbad[k & 1] = bad ? 1 : 0;
  };
  if (r == 0) publish(0);
  __syncthreads();
  for (int k = 0; k < GB; ++k) {
    const int buf = k & 1;
    if (sbad[buf]) {
      if (threadIdx.x == 0) atomicExch(status, 1);
      return;   // the whole block returns: the flag is uniform per block
    }
    if (r == k) {
      a[k][c] = prow[buf][c];
    } else {
      const double f = a[r][k];      // column k, before the step
      __syncwarp();
      // entry (r, k) becomes -f / p: the same update with a = -0 and the
      // pivot row's entry 1 / p
      const double ar = c == k ? -0.0 : a[r][c];
      a[r][c] = ar - f * prow[buf][c];
    }
    __syncwarp();
    if (r == k + 1) publish(k + 1);
    __syncthreads();
  }
  D[threadIdx.x] = a[r][c];
}

// row panel: A_Kj <- D A_Kj for GP columns j per CTA (columns of block K
// skipped); GB x GP threads, one entry each
__global__ void __launch_bounds__(GB * GP)
k_bgj_row(int n, double* __restrict__ M, int k0, int kw, const double* __restrict__ D) {
  __shared__ double d[GB][GB + 1];
  __shared__ double x[GB][GP];
  const int j0 = blockIdx.x * GP;
  for (int e = threadIdx.x; e < GB * GB; e += blockDim.x) d[e / GB][e % GB] = D[e];
  const int r = threadIdx.x / GP, cc = threadIdx.x % GP, j = j0 + cc;
  x[r][cc] = (r < kw && j < n) ? M[(size_t)(k0 + r) * n + j] : 0.0;
  __syncthreads();
  if (r >= kw || j >= n || (j >= k0 && j < k0 + kw)) return;
  double s = 0.0;
  for (int k = 0; k < kw; ++k) s += d[r][k] * x[k][cc];
  M[(size_t)(k0 + r) * n + j] = s;
}

// trailing update on a GT x GT tile: A_ij -= A_iK A_Kj (i, j outside block K),
// each of the 256 threads owns a 2 x 2 patch
__global__ void __launch_bounds__(256) k_bgj_trail(int n, double* __restrict__ M, int k0, int kw) {
  __shared__ double ai[GT][GB + 1];
  __shared__ double bk[GB][GT];
  const int i0 = blockIdx.y * GT, j0 = blockIdx.x * GT;
  for (int e = threadIdx.x; e < GT * GB; e += blockDim.x) {
    const int r = e / GB, k = e % GB, i = i0 + r;
    ai[r][k] = (i < n && k < kw) ? M[(size_t)i * n + k0 + k] : 0.0;
  }
  for (int e = threadIdx.x; e < GB * GT; e += blockDim.x) {
    const int k = e / GT, c = e % GT, j = j0 + c;
    bk[k][c] = (j < n && k < kw) ? M[(size_t)(k0 + k) * n + j] : 0.0;
  }
  __syncthreads();
  const int tr = (threadIdx.x / 16) * 2, tc = (threadIdx.x % 16) * 2;
  double acc[2][2] = {};
  for (int k = 0; k < kw; ++k) {
    double av[2], bv[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      av[u] = ai[tr + u][k];
      bv[u] = bk[k][tc + u];
    }
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
      for (int w = 0; w < 2; ++w) acc[u][w] = fma(av[u], bv[w], acc[u][w]);
  }
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int i = i0 + tr + u;
    if (i >= n || (i >= k0 && i < k0 + kw)) continue;
#pragma unroll
    for (int w = 0; w < 2; ++w) {
      const int j = j0 + tc + w;
      if (j >= n || (j >= k0 && j < k0 + kw)) continue;
      M[(size_t)i * n + j] -= acc[u][w];
    }
  }
}

// column panel: A_iK <- -A_iK D for GP rows i per CTA (rows of block K
// skipped); GP x GB threads, one entry each
__global__ void __launch_bounds__(GB * GP)
k_bgj_col(int n, double* __restrict__ M, int k0, int kw, const double* __restrict__ D) {
  __shared__ double d[GB][GB + 1];
  __shared__ double x[GP][GB + 1];
  const int i0 = blockIdx.x * GP;
  for (int e = threadIdx.x; e < GB * GB; e += blockDim.x) d[e / GB][e % GB] = D[e];
  const int rr = threadIdx.x / GB, c = threadIdx.x % GB, i = i0 + rr;
  x[rr][c] = (i < n && c < kw) ? M[(size_t)i * n + k0 + c] : 0.0;
  __syncthreads();
  if (c >= kw || i >= n || (i >= k0 && i < k0 + kw)) return;
  double s = 0.0;
  for (int k = 0; k < kw; ++k) s += x[rr][k] * d[k][c];
  M[(size_t)i * n + k0 + c] = -s;
}

__global__ void k_bgj_store(int n, double* __restrict__ M, int k0, int kw,
                            const double* __restrict__ D) {
  for (int e = threadIdx.x; e < kw * kw; e += blockDim.x) {
    const int r = e / kw, c = e % kw;
    M[(size_t)(k0 + r) * n + k0 + c] = D[r * GB + c];
  }
}

// ---- V-cycle kernels ----------------------------------------------------
// x = omega D^-1 b (one Jacobi sweep from zero) and r = b - A x
template <class V, class C>
__global__ void k_jacobi0_residual(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                   const V* __restrict__ v, const C* __restrict__ dinv,
                                   const C* __restrict__ b, C omega, C* __restrict__ x,
                                   C* __restrict__ r) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  C s = 0;
  for (int k = rp[i]; k < rp[i + 1]; ++k) {
    int j = ci[k];
    s += cvt<C>(v[k]) * (omega * dinv[j] * b[j]);
  }
  x[i] = omega * dinv[i] * b[i];
  r[i] = b[i] - s;
}

// Two Jacobi sweeps from zero in one pass: with x1 = omega D^-1 b, the second
// sweep x2 = x1 + omega D^-1 (b - A x1) only needs A x1 = sum_j a_ij omega
// d_j b_j, which is formed from b here; the same expressions as k_jacobi0_residual
// followed by k_jacobi, so the same values, with one pass over A fewer.
template <class V, class C>
__global__ void k_jacobi0_twice(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                const V* __restrict__ v, const C* __restrict__ dinv,
                                const C* __restrict__ b, C omega, C* __restrict__ x) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  C s = 0;
  for (int k = rp[i]; k < rp[i + 1]; ++k) {
    int j = ci[k];
    s += cvt<C>(v[k]) * (omega * dinv[j] * b[j]);
  }
  const C x1 = omega * dinv[i] * b[i];
  x[i] = x1 + omega * (dinv[i] * (b[i] - s));
}

template <class V, class C>
__global__ void k_jacobi(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                         const V* __restrict__ v, const C* __restrict__ dinv,
                         const C* __restrict__ b, C omega, const C* __restrict__ xin,
                         C* __restrict__ xout) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  jacobi_row<V, C, LdPlain>(i, i, rp, ci, v, dinv, b, omega, xin, xout);
}

// Chebyshev step: r = b - A x_in; d = c1 d + c2 D^-1 r; x_out = x_in + d
template <class V, class C>
__global__ void k_cheb(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                       const V* __restrict__ v, const C* __restrict__ dinv,
                       const C* __restrict__ b, C c1, C c2, const C* __restrict__ xin,
                       C* __restrict__ d, C* __restrict__ xout) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  C s = 0;
  for (int k = rp[i]; k < rp[i + 1]; ++k) s += cvt<C>(v[k]) * xin[ci[k]];
  C di = c1 * d[i] + c2 * (dinv[i] * (b[i] - s));
  d[i] = di;
  xout[i] = xin[i] + di;
}

// One colour of a Gauss-Seidel sweep, in place: x_i = (b_i - sum_{j != i}
// a_ij x_j) / a_ii for the points i of the colour. A colour's points are not
// coupled, so every row reads only other colours' values.
template <class V, class C>
__global__ void k_mcgs(int q0, int q1, const int* __restrict__ order, const int* __restrict__ rp,
                       const int* __restrict__ ci, const V* __restrict__ v,
                       const C* __restrict__ dinv, const C* __restrict__ b, C* x) {
  const int q = q0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= q1) return;
  const int i = order[q];
  C s = b[i];
  for (int k = rp[i]; k < rp[i + 1]; ++k) {
    const int j = ci[k];
    if (j != i) s -= cvt<C>(v[k]) * x[j];
  }
  x[i] = s * dinv[i];
}

// One damped block-Jacobi sweep of the system AMG (2 unknowns per point):
// r = b - A x_in on the point's two rows, x_out = x_in + omega D_i^{-1} r
template <class V, class C>
__global__ void k_bjac2(int np, const int* __restrict__ rp, const int* __restrict__ ci,
                        const V* __restrict__ v, const C* __restrict__ dinv2,
                        const C* __restrict__ b, C omega, const C* __restrict__ xin,
                        C* __restrict__ xout) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  C r[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int row = 2 * i + k;
    C s = 0;
    for (int q = rp[row]; q < rp[row + 1]; ++q) s += cvt<C>(v[q]) * xin[ci[q]];
    r[k] = b[row] - s;
  }
  const C* d = dinv2 + (size_t)4 * i;
  xout[2 * i] = xin[2 * i] + omega * (d[0] * r[0] + d[1] * r[1]);
  xout[2 * i + 1] = xin[2 * i + 1] + omega * (d[2] * r[0] + d[3] * r[1]);
}

// CPTR: out[2i] = v[i*nb + p], out[2i+1] = v[i*nb + t]
template <class C>
__global__ void k_gather_pair(int N, int nb, const double* __restrict__ v, int p, int t,
                              C* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  out[2 * i] = (C)v[(size_t)i * nb + p];
  out[2 * i + 1] = (C)v[(size_t)i * nb + t];
}

template <class C>
__global__ void k_split_pair(int N, const C* __restrict__ pair, C* __restrict__ vP,
                             C* __restrict__ xT) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  vP[i] = pair[2 * i];
  xT[i] = pair[2 * i + 1];
}

__global__ void k_scatter_pair_zero(int N, int nb, const double* __restrict__ pair, int p, int t,
                                    double* __restrict__ out) {
  long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= (long long)N * nb) return;
  const int i = (int)(tid / nb), k = (int)(tid % nb);
  out[tid] = k == p ? pair[2 * i] : (k == t ? pair[2 * i + 1] : 0.0);
}

template <class V, class C>
__global__ void k_residual(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                           const V* __restrict__ v, const C* __restrict__ b,
                           const C* __restrict__ x, C* __restrict__ r) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  residual_row<V, C, LdPlain>(i, i, rp, ci, v, b, x, r);
}

template <class V, class C>
__global__ void k_restrict(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                           const V* __restrict__ v, const C* __restrict__ r,
                           C* __restrict__ b, const C* __restrict__ dinv, C omega,
                           C* __restrict__ x1) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  restrict_row<V, C, LdPlain>(i, i, rp, ci, v, r, b, dinv, omega, x1);
}

template <class V, class C>
__global__ void k_prolong(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                          const V* __restrict__ v, const C* __restrict__ xc,
                          const C* x, C* xout) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  prolong_row<V, C, LdPlain>(i, i, rp, ci, v, xc, x, xout);
}

// x = Ainv b, one warp per row
template <class C>
__global__ void k_dense_gemv(int n, const C* __restrict__ A, const C* __restrict__ b,
                             C* __restrict__ x) {
  int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (row >= n) return;
  const C s = gemv_row<C, LdPlain>(A + (size_t)row * n, lane, n, b);
  if (lane == 0) x[row] = s;
}

// ---- fused coarse levels -------------------------------------------------
// The levels from the first one whose rows fit the blocks' shared memory down
// to the coarsest run in one cooperative launch of one block per SM. Block b
// owns a contiguous slice of the rows of every level (rows [b R_l, (b+1) R_l),
// R_l = ceil(n_l / blocks)); at the start it copies its rows of A, of P, of R
// for its rows of the next level, of D^-1 and of the coarse inverse into
// shared memory. Then it runs the per-level steps of the V-cycle (Jacobi
// sweeps, residual, restriction with the next level's first sweep, the
// coarse product, prolongation, post-sweeps) over its rows, with a grid
// barrier between steps, so a step waits on the gathers of other blocks'
// vector entries (from L2) and no longer on its matrix rows. Each barrier's
// wait is bounded: past the limit it sets *err, every block leaves the
// kernel, and the solve reports the error.
constexpr unsigned kBarrierSpins = 1u << 20;   // polls of L2: well under a second
constexpr int kMaxTail = 16;                    // levels of the fused launch
constexpr int kTailThreads = 512;
constexpr size_t kTailSmemCap = 200 * 1024;     // shared memory of one block, at most

template <class V, class C>
struct TailLevel {
  int n, nc;
  const int *rp, *ci, *prp, *pci, *rrp, *rci;
  const V *v, *pv, *rv;
  const C* dinv;
  C *b, *x, *x2, *r;
};

template <class C>
struct TailCoarse {
  int n;
  const C* ainv;
  C *b, *x;
};

// rows [r0, r1) of n owned by block b of G
__host__ __device__ __forceinline__ void tail_rows(int n, int G, int b, int& r0, int& r1) {
  const int R = (n + G - 1) / G;
  const long long a = (long long)b * R;
  r0 = (int)(a < n ? a : n);
  r1 = r0 + R < n ? r0 + R : n;
}

// Bytes of one level's shared-memory copy: rows nr (next level nc), entries
// na of A, np of P, nq of R; every array starts on an 8-byte boundary.
__host__ __device__ __forceinline__ size_t al8(size_t x) { return (x + 7) & ~(size_t)7; }
template <class V, class C>
__host__ __device__ __forceinline__ size_t tail_level_bytes(int nr, int nc, int na, int np,
                                                            int nq) {
  return al8(sizeof(C) * nr) + al8(sizeof(V) * na) + al8(sizeof(V) * np) +
         al8(sizeof(V) * nq) + al8(sizeof(int) * (nr + 1)) + al8(sizeof(int) * na) +
         al8(sizeof(int) * (nr + 1)) + al8(sizeof(int) * np) + al8(sizeof(int) * (nc + 1)) +
         al8(sizeof(int) * nq);
}

// One block's copy of one level: its rows [r0, r1) and the next level's [c0,
// c1); row pointers rebased to the copy
template <class V, class C>
struct TailSlice {
  int r0, r1, c0, c1;
  C* dinv;
  V *v, *pv, *rv;
  int *rp, *ci, *prp, *pci, *rrp, *rci;
};

// One word per barrier sequence: every block adds 1, block 0 adds 2^31 minus
// (blocks - 1), so the word's top bit flips once all blocks have arrived and
// its low bits return to their value. Thread 0 of each block spins on the
// top bit (bounded; *err is checked every 256 polls). Returns false once
// *err is set.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, int* err, unsigned nblocks) {
  __shared__ int bad;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vb = bar;
    volatile int* verr = err;
    const unsigned add = blockIdx.x == 0 ? 0x80000000u - (nblocks - 1) : 1u;
    __threadfence();
    const unsigned old = atomicAdd(bar, add);
    unsigned spins = 0;
    int e = 0;
    while (((old ^ *vb) & 0x80000000u) == 0) {
      if ((++spins & 255u) == 0) {
        e = *verr;
        if (e) break;
        if (spins > kBarrierSpins) {
          atomicExch(err, 1);
          e = 1;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
    bad = e ? 1 : *verr;
  }
  __syncthreads();
  return bad == 0;
}

// A barrier that expects a second block which is never launched: its wait
// runs out, sets *err and returns (the bounded-wait path, exercised by a test).
__global__ void k_wait_probe(unsigned* bar, int* err) { grid_barrier(bar, err, 2u); }

// dst[k] = src[k] (minus sub: row pointers rebased) for k < n by the block,
// eight loads in flight per thread (otherwise the copies are a chain of
// dependent round trips)
template <class T, bool REBASE = false>
__device__ __forceinline__ void copy_in(T* dst, const T* __restrict__ src, int n, int sub = 0) {
  constexpr int U = 8;
  const int nt = blockDim.x;
  for (int k0 = threadIdx.x; k0 < n; k0 += U * nt) {
    T t[U];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (k0 + u * nt < n) t[u] = src[k0 + u * nt];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (k0 + u * nt < n) {
        if constexpr (REBASE) dst[k0 + u * nt] = t[u] - sub;
        else dst[k0 + u * nt] = t[u];
      }
  }
}

template <class T>
__device__ __forceinline__ T* carve(unsigned char* base, size_t& off, size_t count) {
  T* p = reinterpret_cast<T*>(base + off);
  off += al8(sizeof(T) * count);
  return p;
}

template <class V, class C>
__global__ void __launch_bounds__(kTailThreads, 1)
k_vcycle_tail(const TailLevel<V, C>* __restrict__ lev, int nlev, TailCoarse<C> co, int nu_pre,
              int nu_post, C omega, unsigned* bar, int* err) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ TailSlice<V, C> S[kMaxTail];
  __shared__ int bnd[kMaxTail][6];
  __shared__ C* ainv_s;
  __shared__ int cr0, cr1;
  const int G = gridDim.x, blk = blockIdx.x, nt = blockDim.x;
  // ---- the block's rows and the extents of its copies
  for (int q = threadIdx.x; q < nlev * 6; q += nt) {
    const int l = q / 6, k = q - 6 * (q / 6);
    const TailLevel<V, C>& L = lev[l];
    int r0, r1, c0, c1;
    tail_rows(L.n, G, blk, r0, r1);
    tail_rows(L.nc, G, blk, c0, c1);
    const int* src[6] = {L.rp + r0, L.rp + r1, L.prp + r0, L.prp + r1, L.rrp + c0, L.rrp + c1};
    bnd[l][k] = *src[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    size_t off = 0;
    for (int l = 0; l < nlev; ++l) {
      TailSlice<V, C>& T = S[l];
      tail_rows(lev[l].n, G, blk, T.r0, T.r1);
      tail_rows(lev[l].nc, G, blk, T.c0, T.c1);
      const int nr = T.r1 - T.r0, nc = T.c1 - T.c0;
      const int na = bnd[l][1] - bnd[l][0], np = bnd[l][3] - bnd[l][2], nq = bnd[l][5] - bnd[l][4];
      T.dinv = carve<C>(smem, off, nr);
      T.v = carve<V>(smem, off, na);
      T.pv = carve<V>(smem, off, np);
      T.rv = carve<V>(smem, off, nq);
      T.rp = carve<int>(smem, off, nr + 1);
      T.ci = carve<int>(smem, off, na);
      T.prp = carve<int>(smem, off, nr + 1);
      T.pci = carve<int>(smem, off, np);
      T.rrp = carve<int>(smem, off, nc + 1);
      T.rci = carve<int>(smem, off, nq);
    }
    int c0, c1;
    tail_rows(co.n, G, blk, c0, c1);
    cr0 = c0;
    cr1 = c1;
    ainv_s = carve<C>(smem, off, (size_t)(c1 - c0) * co.n);
  }
  __syncthreads();
  // ---- copies (row pointers rebased to the block's first entry)
  for (int l = 0; l < nlev; ++l) {
    const TailLevel<V, C>& L = lev[l];
    const TailSlice<V, C>& T = S[l];
    const int nr = T.r1 - T.r0, nc = T.c1 - T.c0;
    const int a0 = bnd[l][0], p0 = bnd[l][2], q0 = bnd[l][4];
    const int na = bnd[l][1] - a0, np = bnd[l][3] - p0, nq = bnd[l][5] - q0;
    copy_in(T.dinv, L.dinv + T.r0, nr);
    copy_in<int, true>(T.rp, L.rp + T.r0, nr + 1, a0);
    copy_in<int, true>(T.prp, L.prp + T.r0, nr + 1, p0);
    copy_in<int, true>(T.rrp, L.rrp + T.c0, nc + 1, q0);
    copy_in(T.v, L.v + a0, na);
    copy_in(T.ci, L.ci + a0, na);
    copy_in(T.pv, L.pv + p0, np);
    copy_in(T.pci, L.pci + p0, np);
    copy_in(T.rv, L.rv + q0, nq);
    copy_in(T.rci, L.rci + q0, nq);
  }
  copy_in(ainv_s, co.ainv + (size_t)cr0 * co.n, (cr1 - cr0) * co.n);
  __syncthreads();
  // ---- the V-cycle on the block's rows
  bool cur_alt[kMaxTail];            // the level's current vector: x (false) or x2 (true)
  for (int l = 0; l < nlev; ++l) {
    const TailLevel<V, C>& L = lev[l];
    const TailSlice<V, C>& T = S[l];
    const int nr = T.r1 - T.r0, nc = T.c1 - T.c0;
    C* cur = L.x;                    // holds the first sweep from zero
    C* alt = L.x2;
    for (int q = 1; q < nu_pre; ++q) {
      for (int m = threadIdx.x; m < nr; m += nt)
        jacobi_row<V, C, LdL2>(m, T.r0 + m, T.rp, T.ci, T.v, T.dinv, L.b, omega, cur, alt);
      if (!grid_barrier(bar, err, G)) return;
      C* t = cur;
      cur = alt;
      alt = t;
    }
    for (int m = threadIdx.x; m < nr; m += nt)
      residual_row<V, C, LdL2>(m, T.r0 + m, T.rp, T.ci, T.v, L.b, cur, L.r);
    if (!grid_barrier(bar, err, G)) return;
    const bool last = l + 1 == nlev;
    C* nb = last ? co.b : lev[l + 1].b;
    C* nx = last ? nullptr : lev[l + 1].x;
    const C* nd = last ? nullptr : S[l + 1].dinv;
    for (int m = threadIdx.x; m < nc; m += nt)
      restrict_row<V, C, LdL2>(m, T.c0 + m, T.rrp, T.rci, T.rv, L.r, nb, nd, omega, nx);
    if (!grid_barrier(bar, err, G)) return;
    cur_alt[l] = cur != L.x;
  }
  {
    const int lane = threadIdx.x & 31;
    for (int row = cr0 + (threadIdx.x >> 5); row < cr1; row += nt >> 5) {
      const C s = gemv_row<C, LdL2>(ainv_s + (size_t)(row - cr0) * co.n, lane, co.n, co.b);
      if (lane == 0) co.x[row] = s;
    }
    if (!grid_barrier(bar, err, G)) return;
  }
  for (int l = nlev - 1; l >= 0; --l) {
    const TailLevel<V, C>& L = lev[l];
    const TailSlice<V, C>& T = S[l];
    const int nr = T.r1 - T.r0;
    const C* xc = l + 1 < nlev ? lev[l + 1].x : co.x;
    C* cur = cur_alt[l] ? L.x2 : L.x;
    C* target = nu_post % 2 == 0 ? L.x : L.x2;
    for (int m = threadIdx.x; m < nr; m += nt)
      prolong_row<V, C, LdL2>(m, T.r0 + m, T.prp, T.pci, T.pv, xc, cur, target);
    if (!grid_barrier(bar, err, G)) return;
    cur = target;
    C* alt = target == L.x ? L.x2 : L.x;
    for (int q = 0; q < nu_post; ++q) {
      for (int m = threadIdx.x; m < nr; m += nt)
        jacobi_row<V, C, LdL2>(m, T.r0 + m, T.rp, T.ci, T.v, T.dinv, L.b, omega, cur, alt);
      if (!grid_barrier(bar, err, G)) return;
      C* t = cur;
      cur = alt;
      alt = t;
    }
  }
}

template <class C>
__global__ void k_gather_var(int N, int nb, const double* __restrict__ v, int var,
                             C* __restrict__ out, const C* __restrict__ dinv, C omega,
                             C* __restrict__ x1) {
  gather_var_row(blockIdx.x * blockDim.x + threadIdx.x, N, nb, v, var, out, dinv, omega, x1);
}

__global__ void k_scatter_var_zero(int N, int nb, const double* __restrict__ s, int var,
                                   double* __restrict__ out) {
  long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= (long long)N * nb) return;
  int i = (int)(tid / nb), k = (int)(tid % nb);
  out[tid] = k == var ? s[i] : 0.0;
}

template <class C>
__global__ void k_pattern_sub(int N, int nb, const int* __restrict__ rp,
                              const int* __restrict__ ci, const C* __restrict__ vals,
                              const C* __restrict__ x, const double* __restrict__ r, int var,
                              C* __restrict__ out, const C* __restrict__ dinv, C omega,
                              C* __restrict__ x1) {
  pattern_sub_row(blockIdx.x * blockDim.x + threadIdx.x, N, nb, rp, ci, vals, x, r, var, out, dinv,
                  omega, x1);
}

__global__ void k_to_float(long long n, const double* __restrict__ in, float* __restrict__ out) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long stride = (long long)gridDim.x * blockDim.x;
  for (; i < n; i += stride) out[i] = (float)in[i];
}

// round to nearest FP32, then to nearest BF16
__global__ void k_to_bf16(long long n, const double* __restrict__ in,
                          __nv_bfloat16* __restrict__ out) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long stride = (long long)gridDim.x * blockDim.x;
  for (; i < n; i += stride) out[i] = __float2bfloat16_rn((float)in[i]);
}


// pointers of one level for one precision
template <class V, class C>
struct LV {
  int n, nc;
  const int *rp, *ci, *prp, *pci, *rrp, *rci;
  const V *v, *pv, *rv;
  const C* dinv;
  C *x2, *r, *d;
  double lam;
  const int* mcorder;                 // multicolour Gauss-Seidel order (or null)
  const std::vector<int>* cstart;     // its colour boundaries (host)
  const C* dinv2;                     // system AMG: inverse 2 x 2 diagonal blocks
};

LV<double, double> view(Level& L, double*) {
  return {L.n, L.nc, L.rp.p, L.ci.p, L.prp.p, L.pci.p, L.rrp.p, L.rci.p,
          L.v.p, L.pv.p, L.rv.p, L.dinv.p, L.x2.p, L.r.p, L.d.p, L.lam,
          L.mcorder.p, &L.cstart, L.dinv2.p};
}
LV<__nv_bfloat16, float> view(Level& L, float*) {
  return {L.n, L.nc, L.rp.p, L.ci.p, L.prp.p, L.pci.p, L.rrp.p, L.rci.p,
          L.vh.p, L.pvh.p, L.rvh.p, L.dinvf.p, L.x2f.p, L.rf.p, L.df.p, L.lam,
          L.mcorder.p, &L.cstart, L.dinv2f.p};
}
double* level_b(Level& L, double*) { return L.b.p; }
float* level_b(Level& L, float*) { return L.bf.p; }
double* level_x(Level& L, double*) { return L.x.p; }
float* level_x(Level& L, float*) { return L.xf.p; }
const double* coarse_inv(Hierarchy& H, double*) { return H.coarse_inv.p; }
const float* coarse_inv(Hierarchy& H, float*) { return H.coarse_invf.p; }

template <class V, class C>
struct Sweeper {
  Handle* h;
  const LV<V, C>& L;
  const mss_options& o;
  // one smoothing application on (b, x): writes the result to xout; xin and
  // xout must differ
  void jacobi(const C* b, const C* xin, C* xout) {
    k_jacobi<V, C><<<grid_for(L.n, h->tb), h->tb, 0, h->stream>>>(L.n, L.rp, L.ci, L.v, L.dinv, b,
                                                            (C)o.jacobi_omega, xin, xout);
    MSS_LAUNCH_CK("k_jacobi");
  }
  // one damped 2 x 2 block-Jacobi sweep (system AMG); xin and xout differ
  void bjac2(const C* b, const C* xin, C* xout) {
    const int np = L.n / 2;
    k_bjac2<V, C><<<grid_for(np, h->tb), h->tb, 0, h->stream>>>(np, L.rp, L.ci, L.v, L.dinv2, b,
                                                               (C)o.jacobi_omega, xin, xout);
    MSS_LAUNCH_CK("k_bjac2");
  }
  // symmetric multicolour Gauss-Seidel, in place on x: the colours in
  // order, then in reverse. The reverse pass starts with the colour the
  // forward pass ended with, whose recomputation from unchanged neighbours
  // gives the same values, so it is not repeated.
  void mcsgs(const C* b, C* x) {
    const std::vector<int>& cs = *L.cstart;
    const int nc = (int)cs.size() - 1;
    auto colour = [&](int c) {
      const int q0 = cs[c], q1 = cs[c + 1];
      if (q1 <= q0) return;
      k_mcgs<V, C><<<grid_for(q1 - q0, h->tb), h->tb, 0, h->stream>>>(q0, q1, L.mcorder, L.rp,
                                                                       L.ci, L.v, L.dinv, b, x);
      MSS_LAUNCH_CK("k_mcgs");
    };
    for (int c = 0; c < nc; ++c) colour(c);
    for (int c = nc - 2; c >= 0; --c) colour(c);
  }
  // Chebyshev polynomial of degree o.cheb_degree; ping-pongs between x and
  // alt, returns the buffer holding the result
  C* cheb(const C* b, C* x, C* alt) {
    double hi = o.cheb_hi_factor * L.lam, lo = L.lam / o.cheb_lo_ratio;
    double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo);
    double sigma = theta / delta, rho = 1.0 / sigma;
    C* cur = x;
    C* nxt = alt;
    for (int k = 1; k <= o.cheb_degree; ++k) {
      double c1, c2;
      if (k == 1) {
        c1 = 0.0;
        c2 = 1.0 / theta;
      } else {
        double rn = 1.0 / (2.0 * sigma - rho);
        c1 = rn * rho;
        c2 = 2.0 * rn / delta;
        rho = rn;
      }
      k_cheb<V, C><<<grid_for(L.n, h->tb), h->tb, 0, h->stream>>>(L.n, L.rp, L.ci, L.v, L.dinv, b,
                                                            (C)c1, (C)c2, cur, L.d, nxt);
      MSS_LAUNCH_CK("k_cheb");
      C* t = cur;
      cur = nxt;
      nxt = t;
    }
    return cur;
  }
};

// Does the V-cycle on level l start with a Jacobi sweep from zero whose
// result the producer of b can write? (Jacobi smoothing, not the coarsest.)
bool has_sweep0(const Hierarchy& H, const mss_options& o, int l) {
  return H.bs == 1 && o.smoother == MSS_JACOBI && l < (int)H.lev.size() - 1;
}

// V-cycle on level l for right-hand side b; the result goes to out. With
// x_has_sweep0, out already holds the first pre-smoothing sweep from zero,
// omega D^-1 b, written by the kernel that formed b (the restriction on
// coarser levels), so the remaining sweeps are plain Jacobi sweeps; the
// values are those of the sweeps run from zero here.
const unsigned char* tail_desc(Hierarchy& H, double*) { return H.tdesc.p; }
const unsigned char* tail_desc(Hierarchy& H, float*) { return H.tdescf.p; }

// The fused launches of different handles run one after the other on the
// device: a grid with one block per SM cannot share the device with another
// such grid, so each launch waits (on its stream, no host wait) for the
// completion event of the previous one, whichever stream ran it.
std::mutex g_tail_mu;
cudaEvent_t g_tail_done[64] = {};   // per device

template <class V, class C>
void launch_tail(Handle* h, Hierarchy& H) {
  const int nlev = (int)H.lev.size() - 1 - H.tail;
  Level& Cl = H.lev.back();
  TailCoarse<C> co{Cl.n, coarse_inv(H, (C*)nullptr), level_b(Cl, (C*)nullptr),
                   level_x(Cl, (C*)nullptr)};
  const TailLevel<V, C>* lev =
      reinterpret_cast<const TailLevel<V, C>*>(tail_desc(H, (C*)nullptr));
  int nu_pre = h->opt.nu_pre, nu_post = h->opt.nu_post;
  C omega = (C)h->opt.jacobi_omega;
  unsigned* bar = H.tbar.p;
  int* err = H.terr.p;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)H.tail_grid);
  cfg.blockDim = dim3(kTailThreads);
  cfg.dynamicSmemBytes = H.tail_smem;
  cfg.stream = h->stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  std::lock_guard<std::mutex> lk(g_tail_mu);
  if (h->device < 0 || h->device >= 64) fail(MSS_ERR_CUDA, "device index out of range");
  cudaEvent_t& done = g_tail_done[h->device];
  if (!done) MSS_CK(cudaEventCreateWithFlags(&done, cudaEventDisableTiming));
  MSS_CK(cudaStreamWaitEvent(h->stream, done, 0));
  MSS_CK(cudaLaunchKernelEx(&cfg, k_vcycle_tail<V, C>, lev, nlev, co, nu_pre, nu_post, omega, bar,
                            err));
  MSS_LAUNCH_CK("k_vcycle_tail");
  MSS_CK(cudaEventRecord(done, h->stream));
}

template <class V, class C>
void vcycle_level(Handle* h, Hierarchy& H, int l, const C* b, C* out, bool x_has_sweep0) {
  Level& Lev = H.lev[l];
  const LV<V, C> L = view(Lev, (C*)nullptr);
  const mss_options& o = h->opt;
  const int n = L.n;
  if (l == H.tail && x_has_sweep0 && !h->capturing && tail_desc(H, (C*)nullptr)) {
    // b and the first sweep were written by the previous level's restriction
    // into this level's vectors, which the fused launch reads. Launches from
    // the host cost several microseconds each, more than a grid barrier; in
    // a captured graph a launch boundary costs about a microsecond, less
    // than a grid barrier (measured), so graphs keep the per-level kernels.
    launch_tail<V, C>(h, H);
    return;
  }
  if (l == (int)H.lev.size() - 1) {
    k_dense_gemv<C><<<grid_for((long long)n * 32, 256), 256, 0, h->stream>>>(
        n, coarse_inv(H, (C*)nullptr), b, out);
    MSS_LAUNCH_CK("k_dense_gemv");
    return;
  }
  Sweeper<V, C> sw{h, L, o};
  Level& Cl = H.lev[l + 1];
  C* cb = level_b(Cl, (C*)nullptr);
  C* cx = level_x(Cl, (C*)nullptr);
  // ---- pre-smoothing from zero, then the residual
  C* cur = out;
  C* alt = L.x2;
  if (H.bs == 2) {   // system AMG: block Jacobi from zero
    MSS_CK(cudaMemsetAsync(cur, 0, sizeof(C) * (size_t)n, h->stream));
    for (int s = 0; s < o.nu_pre; ++s) {
      sw.bjac2(b, cur, alt);
      std::swap(cur, alt);
    }
    k_residual<V, C><<<grid_for(n, h->tb), h->tb, 0, h->stream>>>(n, L.rp, L.ci, L.v, b, cur, L.r);
    MSS_LAUNCH_CK("k_residual");
  } else if (o.smoother == MSS_JACOBI && x_has_sweep0) {
    for (int s = 1; s < o.nu_pre; ++s) {
      sw.jacobi(b, cur, alt);
      std::swap(cur, alt);
    }
    k_residual<V, C><<<grid_for(n, h->tb), h->tb, 0, h->stream>>>(n, L.rp, L.ci, L.v, b, cur, L.r);
    MSS_LAUNCH_CK("k_residual");
  } else if (o.smoother == MSS_JACOBI && o.nu_pre == 1) {
    k_jacobi0_residual<V, C><<<grid_for(n, h->tb), h->tb, 0, h->stream>>>(
        n, L.rp, L.ci, L.v, L.dinv, b, (C)o.jacobi_omega, out, L.r);
    MSS_LAUNCH_CK("k_jacobi0_residual");
  } else if (o.smoother == MSS_JACOBI) {
    k_jacobi0_twice<V, C><<<grid_for(n, h->tb), h->tb, 0, h->stream>>>(
        n, L.rp, L.ci, L.v, L.dinv, b, (C)o.jacobi_omega, out);
    MSS_LAUNCH_CK("k_jacobi0_twice");
    for (int s = 2; s < o.nu_pre; ++s) {
      sw.jacobi(b, cur, alt);
      std::swap(cur, alt);
    }
    k_residual<V, C><<<grid_for(n, h->tb), h->tb, 0, h->stream>>>(n, L.rp, L.ci, L.v, b, cur, L.r);
    MSS_LAUNCH_CK("k_residual");
  } else if (o.smoother == MSS_MCSGS) {
    MSS_CK(cudaMemsetAsync(cur, 0, sizeof(C) * (size_t)n, h->stream));
    for (int s = 0; s < o.nu_pre; ++s) sw.mcsgs(b, cur);
    k_residual<V, C><<<grid_for(n, h->tb), h->tb, 0, h->stream>>>(n, L.rp, L.ci, L.v, b, cur, L.r);
    MSS_LAUNCH_CK("k_residual");
  } else {
    MSS_CK(cudaMemsetAsync(cur, 0, sizeof(C) * (size_t)n, h->stream));
    for (int s = 0; s < o.nu_pre; ++s) {
      C* res = sw.cheb(b, cur, alt);
      if (res != cur) std::swap(cur, alt);
    }
    k_residual<V, C><<<grid_for(n, h->tb), h->tb, 0, h->stream>>>(n, L.rp, L.ci, L.v, b, cur, L.r);
    MSS_LAUNCH_CK("k_residual");
  }
  // ---- restriction (with the coarse level's first sweep) and the coarse
  // correction
  const bool next0 = has_sweep0(H, o, l + 1);
  const LV<V, C> Lc = view(Cl, (C*)nullptr);
  k_restrict<V, C><<<grid_for(L.nc, h->tb), h->tb, 0, h->stream>>>(
      L.nc, L.rrp, L.rci, L.rv, L.r, cb, Lc.dinv, (C)o.jacobi_omega, next0 ? cx : nullptr);
  MSS_LAUNCH_CK("k_restrict");
  vcycle_level<V, C>(h, H, l + 1, cb, cx, next0);
  // ---- prolongation into the vector from which the post-smoothing sweeps,
  // alternating between the two vectors, end in out
  // (Gauss-Seidel sweeps work in place)
  const int writes = H.bs == 2 ? o.nu_post
                   : o.smoother == MSS_MCSGS
                         ? 0
                         : o.nu_post * (o.smoother == MSS_JACOBI ? 1 : o.cheb_degree);
  C* target = writes % 2 == 0 ? out : L.x2;
  k_prolong<V, C><<<grid_for(n, h->tb), h->tb, 0, h->stream>>>(n, L.prp, L.pci, L.pv, cx, cur,
                                                               target);
  MSS_LAUNCH_CK("k_prolong");
  cur = target;
  alt = target == out ? L.x2 : out;
  // ---- post-smoothing
  for (int s = 0; s < o.nu_post; ++s) {
    if (H.bs == 2) {
      sw.bjac2(b, cur, alt);
      std::swap(cur, alt);
    } else if (o.smoother == MSS_JACOBI) {
      sw.jacobi(b, cur, alt);
      std::swap(cur, alt);
    } else if (o.smoother == MSS_MCSGS) {
      sw.mcsgs(b, cur);
    } else {
      C* res = sw.cheb(b, cur, alt);
      if (res != cur) std::swap(cur, alt);
    }
  }
  if (cur != out) copy_dev(h, out, cur, sizeof(C) * (size_t)n);
}

unsigned stride_grid(long long n) {
  unsigned g = grid_for(n, 256);
  return g > 8192u ? 8192u : g;
}

}  // namespace

static std::mutex g_coop_mu;

// Blocked Gauss-Jordan without pivoting into H.coarse_inv; false when a pivot
// was too small (H.coarse_inv is then to be recomputed with pivoting).
static bool coarse_inverse_blocked(Handle* h, Hierarchy& H) {
  Level& C = H.lev.back();
  const int n = C.n;
  double* M = H.coarse_inv.p;
  MSS_CK(cudaMemsetAsync(M, 0, sizeof(double) * (size_t)n * n, h->stream));
  k_dense_square<<<grid_for(n, 128), 128, 0, h->stream>>>(n, C.rp.p, C.ci.p, C.v.p, M);
  MSS_LAUNCH_CK("k_dense_square");
  DBuf<double> D(h, GB * GB);
  DBuf<int> status(h, 1);
  fill_int(h, status.p, 0, 1);
  const int tiles = (n + GT - 1) / GT;
  const int panels = (n + GP - 1) / GP;
  for (int k0 = 0; k0 < n; k0 += GB) {
    const int kw = n - k0 < GB ? n - k0 : GB;
    k_bgj_diag<<<1, GB * GB, 0, h->stream>>>(n, M, k0, kw, D.p, status.p);
    MSS_LAUNCH_CK("k_bgj_diag");
    k_bgj_row<<<panels, GB * GP, 0, h->stream>>>(n, M, k0, kw, D.p);
    MSS_LAUNCH_CK("k_bgj_row");
    k_bgj_trail<<<dim3(tiles, tiles), 256, 0, h->stream>>>(n, M, k0, kw);
    MSS_LAUNCH_CK("k_bgj_trail");
    k_bgj_col<<<panels, GB * GP, 0, h->stream>>>(n, M, k0, kw, D.p);
    MSS_LAUNCH_CK("k_bgj_col");
    k_bgj_store<<<1, 256, 0, h->stream>>>(n, M, k0, kw, D.p);
    MSS_LAUNCH_CK("k_bgj_store");
  }
  return read_int(h, status.p) == 0;
}

void coarse_inverse(Handle* h, Hierarchy& H) {
  Level& C = H.lev.back();
  const int n = C.n;
  if (n > 8192) fail(MSS_ERR_AMG, "coarsest AMG level has " + std::to_string(n) +
                                      " rows; raise amg_max_levels or amg_max_coarse");
  H.nc = n;
  H.coarse_inv.reset(h, (size_t)n * n);
  {
    static const bool times = std::getenv("MSS_SETUP_TIMES") != nullptr;
    const auto t0 = std::chrono::steady_clock::now();
    const bool ok = coarse_inverse_blocked(h, H);
    if (times)
      std::fprintf(stderr, "mss coarse inverse (blocked): n = %d, %s, %.2f ms\n", n,
                   ok ? "ok" : "small pivot, falling back",
                   std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0)
                       .count());
    if (ok) return;
  }
  DBuf<double> M(h, (size_t)n * 2 * n);
  DBuf<int> piv(h, n), status(h, 1);
  MSS_CK(cudaMemsetAsync(M.p, 0, sizeof(double) * (size_t)n * 2 * n, h->stream));
  fill_int(h, status.p, 0, 1);
  k_dense_from_csr<<<grid_for(n, 128), 128, 0, h->stream>>>(n, C.rp.p, C.ci.p, C.v.p, M.p);
  MSS_LAUNCH_CK("k_dense_from_csr");
  const int threads = 256;
  int per_sm = 0;
  size_t smem = (size_t)n;
  MSS_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gauss_jordan, threads, smem));
  if (per_sm < 1) fail(MSS_ERR_CUDA, "cooperative Gauss-Jordan kernel cannot be resident");
  int want = (n + (threads / 32) - 1) / (threads / 32);
  int blocks = h->num_sms * per_sm;
  if (blocks > want) blocks = want;
  if (blocks < 1) blocks = 1;
  int nn = n;
  double* Mp = M.p;
  int* pp = piv.p;
  int* sp = status.p;
  void* args[] = {&nn, &Mp, &pp, &sp};
  int st;
  {
    // one cooperative grid at a time in the process: the set-up builds two
    // hierarchies on concurrent streams, and two device-filling cooperative
    // grids must not wait on each other's residency
    static const bool times = std::getenv("MSS_SETUP_TIMES") != nullptr;
    const auto t0 = std::chrono::steady_clock::now();
    std::lock_guard<std::mutex> lk(g_coop_mu);
    const auto t1 = std::chrono::steady_clock::now();
    MSS_CK(cudaLaunchCooperativeKernel((const void*)k_gauss_jordan, dim3(blocks),
                                       dim3(threads), args, smem, h->stream));
    count_launch();
    st = read_int(h, status.p);   // synchronises: the grid has finished
    if (times)
      std::fprintf(stderr, "mss coarse inverse: n = %d, waited %.2f ms, ran %.2f ms\n", n,
                   std::chrono::duration<double, std::milli>(t1 - t0).count(),
                   std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t1)
                       .count());
  }
  if (st != 0) fail(MSS_ERR_AMG, "coarsest AMG operator is singular (column " +
                                     std::to_string(st - 1) + ")");
  DBuf<int> slot(h, n);
  k_gj_slots<<<grid_for(n, 256), 256, 0, h->stream>>>(n, piv.p, slot.p);
  MSS_LAUNCH_CK("k_gj_slots");
  k_gj_extract<<<grid_for((long long)n * n, 256), 256, 0, h->stream>>>(n, M.p, piv.p, slot.p,
                                                                       H.coarse_inv.p);
  MSS_LAUNCH_CK("k_gj_extract");
}

void to_float(Handle* h, const double* in, float* out, long long n) {
  if (n <= 0) return;
  k_to_float<<<stride_grid(n), 256, 0, h->stream>>>(n, in, out);
  MSS_LAUNCH_CK("k_to_float");
}

void to_bf16(Handle* h, const double* in, __nv_bfloat16* out, long long n) {
  if (n <= 0) return;
  k_to_bf16<<<stride_grid(n), 256, 0, h->stream>>>(n, in, out);
  MSS_LAUNCH_CK("k_to_bf16");
}

// BF16 copies of A, P, R values, FP32 D^-1, FP32 vectors, FP32 coarse inverse
void pack_hierarchy_mixed(Handle* h, Hierarchy& H) {
  for (size_t l = 0; l < H.lev.size(); ++l) {
    Level& L = H.lev[l];
    const bool last = l + 1 == H.lev.size();
    L.vh.reset(h, L.nnz);
    to_bf16(h, L.v.p, L.vh.p, L.nnz);
    L.dinvf.reset(h, L.n);
    to_float(h, L.dinv.p, L.dinvf.p, L.n);
    if (L.dinv2.p) {
      L.dinv2f.reset(h, L.dinv2.n);
      to_float(h, L.dinv2.p, L.dinv2f.p, (long long)L.dinv2.n);
    }
    if (!last) {
      L.pvh.reset(h, L.nnzP);
      to_bf16(h, L.pv.p, L.pvh.p, L.nnzP);
      L.rvh.reset(h, L.nnzP);
      to_bf16(h, L.rv.p, L.rvh.p, L.nnzP);
    }
    L.bf.reset(h, L.n);
    L.xf.reset(h, L.n);
    L.x2f.reset(h, L.n);
    L.rf.reset(h, L.n);
    L.df.reset(h, L.n);
  }
  H.coarse_invf.reset(h, (size_t)H.nc * H.nc);
  to_float(h, H.coarse_inv.p, H.coarse_invf.p, (long long)H.nc * H.nc);
}

Sweep0<double> sweep0(Handle* h, Hierarchy& H, double* x) {
  if (!has_sweep0(H, h->opt, 0)) return {};
  return {H.lev[0].dinv.p, h->opt.jacobi_omega, x};
}

Sweep0<float> sweep0_mixed(Handle* h, Hierarchy& H, float* x) {
  if (!has_sweep0(H, h->opt, 0)) return {};
  return {H.lev[0].dinvf.p, (float)h->opt.jacobi_omega, x};
}

template <class V, class C>
TailLevel<V, C> tail_level(Level& L) {
  const LV<V, C> w = view(L, (C*)nullptr);
  return {w.n, w.nc, w.rp, w.ci, w.prp, w.pci, w.rrp, w.rci, w.v, w.pv, w.rv, w.dinv,
          level_b(L, (C*)nullptr), level_x(L, (C*)nullptr), w.x2, w.r};
}

template <class V, class C>
void upload_tail(Handle* h, Hierarchy& H, DBuf<unsigned char>& dst) {
  std::vector<TailLevel<V, C>> hv;
  for (int l = H.tail; l + 1 < (int)H.lev.size(); ++l) hv.push_back(tail_level<V, C>(H.lev[l]));
  const size_t bytes = sizeof(TailLevel<V, C>) * hv.size();
  dst.reset(h, bytes);
  MSS_CK(cudaMemcpyAsync(dst.p, hv.data(), bytes, cudaMemcpyHostToDevice, h->stream));
  MSS_CK(cudaStreamSynchronize(h->stream));   // hv lives on this frame
}

// Per-block bytes of the fused launch's shared-memory copies of levels
// l..(coarsest) over G blocks (FP64 storage, the larger of the two forms);
// the row pointers are read back for the levels that can fit at all.
static std::vector<size_t> tail_level_block_bytes(Handle* h, Level& L, int G) {
  std::vector<int> rp((size_t)L.n + 1), prp((size_t)L.n + 1), rrp((size_t)L.nc + 1);
  MSS_CK(cudaMemcpyAsync(rp.data(), L.rp.p, sizeof(int) * rp.size(), cudaMemcpyDeviceToHost,
                         h->stream));
  MSS_CK(cudaMemcpyAsync(prp.data(), L.prp.p, sizeof(int) * prp.size(), cudaMemcpyDeviceToHost,
                         h->stream));
  MSS_CK(cudaMemcpyAsync(rrp.data(), L.rrp.p, sizeof(int) * rrp.size(), cudaMemcpyDeviceToHost,
                         h->stream));
  MSS_CK(cudaStreamSynchronize(h->stream));
  std::vector<size_t> out((size_t)G);
  for (int b = 0; b < G; ++b) {
    int r0, r1, c0, c1;
    tail_rows(L.n, G, b, r0, r1);
    tail_rows(L.nc, G, b, c0, c1);
    out[b] = tail_level_bytes<double, double>(r1 - r0, c1 - c0, rp[r1] - rp[r0], prp[r1] - prp[r0],
                                              rrp[c1] - rrp[c0]);
  }
  return out;
}

void prepare_tail(Handle* h, Hierarchy& H) {
  H.tail = -1;
  H.tdesc.release();
  H.tdescf.release();
  const int nl = (int)H.lev.size();
  if (h->opt.smoother != MSS_JACOBI || H.bs != 1 || nl < 3) return;
  // one block per SM; the first level from which every block's copies fit
  const int G = h->num_sms;
  std::vector<size_t> tot((size_t)G, 0);
  {
    const int nc = H.lev.back().n;
    for (int b = 0; b < G; ++b) {
      int c0, c1;
      tail_rows(nc, G, b, c0, c1);
      tot[b] = al8(sizeof(double) * (size_t)(c1 - c0) * nc);
    }
  }
  int t = -1;
  size_t smem = 0;
  for (int l = nl - 2; l >= 1; --l) {
    Level& L = H.lev[l];
    // a level whose average share is already too large cannot fit
    if ((size_t)L.nnz * 12 / G > kTailSmemCap) break;
    const std::vector<size_t> lb = tail_level_block_bytes(h, L, G);
    size_t mx = 0;
    for (int b = 0; b < G; ++b) mx = std::max(mx, tot[b] + lb[b]);
    if (mx > kTailSmemCap || nl - 1 - l > kMaxTail) break;
    for (int b = 0; b < G; ++b) tot[b] += lb[b];
    t = l;
    smem = mx;
  }
  if (t < 0) return;
  // the kernels' shared-memory limit is process-wide: every handle sets the
  // same cap (never its own size, which would shrink another handle's)
  MSS_CK(cudaFuncSetAttribute(k_vcycle_tail<double, double>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTailSmemCap));
  MSS_CK(cudaFuncSetAttribute(k_vcycle_tail<__nv_bfloat16, float>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTailSmemCap));
  int per_sm = 0;
  MSS_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_vcycle_tail<double, double>,
                                                       kTailThreads, smem));
  if (per_sm < 1) return;
  H.tail_grid = G;
  H.tail_smem = smem;
  H.tail = t;
  H.tbar.reset(h, 1);
  H.terr.reset(h, 1);
  MSS_CK(cudaMemsetAsync(H.tbar.p, 0, sizeof(unsigned), h->stream));
  MSS_CK(cudaMemsetAsync(H.terr.p, 0, sizeof(int), h->stream));
  upload_tail<double, double>(h, H, H.tdesc);
  if (h->opt.precision == MSS_MIXED) upload_tail<__nv_bfloat16, float>(h, H, H.tdescf);
}

int wait_limit_probe(Handle* h) {
  DBuf<unsigned> bar(h, 1);
  DBuf<int> err(h, 1);
  MSS_CK(cudaMemsetAsync(bar.p, 0, sizeof(unsigned), h->stream));
  MSS_CK(cudaMemsetAsync(err.p, 0, sizeof(int), h->stream));
  k_wait_probe<<<1, 32, 0, h->stream>>>(bar.p, err.p);
  MSS_LAUNCH_CK("k_wait_probe");
  return read_int(h, err.p);
}

void check_tail(Handle* h, Hierarchy& H) {
  if (H.tail < 0 || !H.terr.p) return;
  if (read_int(h, H.terr.p) != 0)
    fail(MSS_ERR_CUDA, "a grid barrier of the fused coarse V-cycle levels exceeded its wait limit");
}

void vcycle(Handle* h, Hierarchy& H, const double* b, double* x, bool x_has_sweep0) {
  TraceScope ts(h, TR_VCYCLE);
  vcycle_level<double, double>(h, H, 0, b, x, x_has_sweep0 && has_sweep0(H, h->opt, 0));
}

void vcycle_mixed(Handle* h, Hierarchy& H, const float* b, float* x, bool x_has_sweep0) {
  TraceScope ts(h, TR_VCYCLE);
  vcycle_level<__nv_bfloat16, float>(h, H, 0, b, x, x_has_sweep0 && has_sweep0(H, h->opt, 0));
}

void gather_var(Handle* h, const double* v, int var, double* out, Sweep0<double> s0) {
  k_gather_var<double><<<grid_for(h->N, h->tb), h->tb, 0, h->stream>>>(h->N, h->nb, v, var, out,
                                                                       s0.dinv, s0.omega, s0.x);
  MSS_LAUNCH_CK("k_gather_var");
}

void gather_var(Handle* h, const double* v, int var, float* out, Sweep0<float> s0) {
  k_gather_var<float><<<grid_for(h->N, h->tb), h->tb, 0, h->stream>>>(h->N, h->nb, v, var, out,
                                                                      s0.dinv, s0.omega, s0.x);
  MSS_LAUNCH_CK("k_gather_var");
}

void scatter_var_zero(Handle* h, const double* s, int var, double* out) {
  long long tot = (long long)h->N * h->nb;
  k_scatter_var_zero<<<grid_for(tot, h->tb), h->tb, 0, h->stream>>>(h->N, h->nb, s, var, out);
  MSS_LAUNCH_CK("k_scatter_var_zero");
}

void csr_block_pattern_spmv_sub(Handle* h, const double* vals, const double* x, const double* r,
                                int var, double* out, Sweep0<double> s0) {
  k_pattern_sub<double><<<grid_for(h->N, h->tb), h->tb, 0, h->stream>>>(
      h->N, h->nb, h->rp.p, h->ci.p, vals, x, r, var, out, s0.dinv, s0.omega, s0.x);
  MSS_LAUNCH_CK("k_pattern_sub");
}

void csr_block_pattern_spmv_sub(Handle* h, const float* vals, const float* x, const double* r,
                                int var, float* out, Sweep0<float> s0) {
  k_pattern_sub<float><<<grid_for(h->N, h->tb), h->tb, 0, h->stream>>>(
      h->N, h->nb, h->rp.p, h->ci.p, vals, x, r, var, out, s0.dinv, s0.omega, s0.x);
  MSS_LAUNCH_CK("k_pattern_sub");
}

void gather_pair(Handle* h, const double* v, double* out) {
  k_gather_pair<double><<<grid_for(h->N, h->tb), h->tb, 0, h->stream>>>(h->N, h->nb, v, h->p,
                                                                       h->t, out);
  MSS_LAUNCH_CK("k_gather_pair");
}

void gather_pair(Handle* h, const double* v, float* out) {
  k_gather_pair<float><<<grid_for(h->N, h->tb), h->tb, 0, h->stream>>>(h->N, h->nb, v, h->p,
                                                                      h->t, out);
  MSS_LAUNCH_CK("k_gather_pair");
}

template <class C>
void split_pair(Handle* h, const C* pair, C* vP, C* xT) {
  k_split_pair<C><<<grid_for(h->N, h->tb), h->tb, 0, h->stream>>>(h->N, pair, vP, xT);
  MSS_LAUNCH_CK("k_split_pair");
}
template void split_pair<double>(Handle*, const double*, double*, double*);
template void split_pair<float>(Handle*, const float*, float*, float*);

void scatter_pair_zero(Handle* h, const double* pair, double* out) {
  const long long tot = (long long)h->N * h->nb;
  k_scatter_pair_zero<<<grid_for(tot, h->tb), h->tb, 0, h->stream>>>(h->N, h->nb, pair, h->p,
                                                                     h->t, out);
  MSS_LAUNCH_CK("k_scatter_pair_zero");
}

}  // namespace mss
