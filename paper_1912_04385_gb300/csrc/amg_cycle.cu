// amg_cycle.cu -- AMG V-cycle (Sec. 5.1: one V-cycle, direct coarse solve)
// and the dense inverse of the coarsest operator.
//
// V(nu_pre, nu_post) with damped Jacobi or Chebyshev smoothing from a zero
// initial guess, restriction R = P^T, prolongation P, and the direct coarse
// solve applied as a dense matrix-vector product with the explicit inverse.
#include <cooperative_groups.h>

#include <cmath>
#include <cstring>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace mss {
namespace {

// ---- coarse inverse: Gauss-Jordan with partial pivoting ------------------
// M is the n x 2n augmented matrix [A | I] (row-major). Every block finds
// the pivot of column k itself (same data, same decision); rows are not
// swapped, the pivot row of column k is recorded instead. One grid-wide
// barrier per column.
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
    if (blockIdx.x == 0 && threadIdx.x == 0) pivrow[k] = p;
    const double* prow = M + (size_t)p * ld;
    const double pk = prow[k];
    for (int i = gwarp; i < n; i += nwarps) {
      if (i == p) continue;
      double* row = M + (size_t)i * ld;
      const double f = row[k] / pk;
      if (f == 0.0) continue;
      for (int j = k + 1 + lane; j < ld; j += 32) row[j] = fma(-f, prow[j], row[j]);
    }
    grid.sync();
    __syncthreads();
  }
}

__global__ void k_gj_extract(int n, const double* __restrict__ M, const int* __restrict__ pivrow,
                             double* __restrict__ inv) {
  long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= (long long)n * n) return;
  int k = (int)(tid / n), c = (int)(tid % n);
  int p = pivrow[k];
  inv[tid] = M[(size_t)p * 2 * n + n + c] / M[(size_t)p * 2 * n + k];
}

__global__ void k_dense_from_csr(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                 const double* __restrict__ v, double* __restrict__ M) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double* row = M + (size_t)i * 2 * n;
  for (int k = rp[i]; k < rp[i + 1]; ++k) row[ci[k]] = v[k];
  row[n + i] = 1.0;
}

// ---- V-cycle kernels ----------------------------------------------------
// x = omega D^-1 b (one Jacobi sweep from zero) and r = b - A x
__global__ void k_jacobi0_residual(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                   const double* __restrict__ v, const double* __restrict__ dinv,
                                   const double* __restrict__ b, double omega,
                                   double* __restrict__ x, double* __restrict__ r) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int k = rp[i]; k < rp[i + 1]; ++k) {
    int j = ci[k];
    s += v[k] * (omega * dinv[j] * b[j]);
  }
  x[i] = omega * dinv[i] * b[i];
  r[i] = b[i] - s;
}

// x_out = x_in + omega D^-1 (b - A x_in)
__global__ void k_jacobi(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                         const double* __restrict__ v, const double* __restrict__ dinv,
                         const double* __restrict__ b, double omega,
                         const double* __restrict__ xin, double* __restrict__ xout) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int k = rp[i]; k < rp[i + 1]; ++k) s += v[k] * xin[ci[k]];
  xout[i] = xin[i] + omega * (dinv[i] * (b[i] - s));
}

// Chebyshev step: r = b - A x_in; d = c1 d + c2 D^-1 r; x_out = x_in + d
__global__ void k_cheb(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                       const double* __restrict__ v, const double* __restrict__ dinv,
                       const double* __restrict__ b, double c1, double c2,
                       const double* __restrict__ xin, double* __restrict__ d,
                       double* __restrict__ xout) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int k = rp[i]; k < rp[i + 1]; ++k) s += v[k] * xin[ci[k]];
  double di = c1 * d[i] + c2 * (dinv[i] * (b[i] - s));
  d[i] = di;
  xout[i] = xin[i] + di;
}

__global__ void k_residual(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                           const double* __restrict__ v, const double* __restrict__ b,
                           const double* __restrict__ x, double* __restrict__ r) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int k = rp[i]; k < rp[i + 1]; ++k) s += v[k] * x[ci[k]];
  r[i] = b[i] - s;
}

__global__ void k_csr_spmv(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                           const double* __restrict__ v, const double* __restrict__ x,
                           double* __restrict__ y) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int k = rp[i]; k < rp[i + 1]; ++k) s += v[k] * x[ci[k]];
  y[i] = s;
}

// xout = x + P xc
__global__ void k_prolong(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                          const double* __restrict__ v, const double* __restrict__ xc,
                          const double* __restrict__ x, double* __restrict__ xout) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int k = rp[i]; k < rp[i + 1]; ++k) s += v[k] * xc[ci[k]];
  xout[i] = x[i] + s;
}

// x = Ainv b, one warp per row
__global__ void k_dense_gemv(int n, const double* __restrict__ A, const double* __restrict__ b,
                             double* __restrict__ x) {
  int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (row >= n) return;
  const double* a = A + (size_t)row * n;
  double s = 0.0;
  for (int j = lane; j < n; j += 32) s += a[j] * b[j];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) x[row] = s;
}

__global__ void k_gather_var(int N, int nb, const double* __restrict__ v, int var,
                             double* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) out[i] = v[(size_t)i * nb + var];
}

__global__ void k_scatter_var_zero(int N, int nb, const double* __restrict__ s, int var,
                                   double* __restrict__ out) {
  long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= (long long)N * nb) return;
  int i = (int)(tid / nb), k = (int)(tid % nb);
  out[tid] = k == var ? s[i] : 0.0;
}

// out_i = r[i*nb + var] - sum_j vals_ij x_j over the block pattern
__global__ void k_pattern_sub(int N, int nb, const int* __restrict__ rp,
                              const int* __restrict__ ci, const double* __restrict__ vals,
                              const double* __restrict__ x, const double* __restrict__ r, int var,
                              double* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double s = 0.0;
  for (int k = rp[i]; k < rp[i + 1]; ++k) s += vals[k] * x[ci[k]];
  out[i] = r[(size_t)i * nb + var] - s;
}

constexpr int VT = 256;

struct Sweeper {
  Handle* h;
  Level& L;
  const mss_options& o;
  // one smoothing application on (b, x): writes the result to xout; xin and
  // xout must differ
  void jacobi(const double* b, const double* xin, double* xout) {
    k_jacobi<<<grid_for(L.n, VT), VT, 0, h->stream>>>(L.n, L.rp.p, L.ci.p, L.v.p, L.dinv.p, b,
                                                      o.jacobi_omega, xin, xout);
    MSS_LAUNCH_CK("k_jacobi");
  }
  // Chebyshev polynomial of degree o.cheb_degree; ping-pongs between x and
  // alt, returns the buffer holding the result
  double* cheb(const double* b, double* x, double* alt) {
    double hi = o.cheb_hi_factor * L.lam, lo = L.lam / o.cheb_lo_ratio;
    double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo);
    double sigma = theta / delta, rho = 1.0 / sigma;
    double* cur = x;
    double* nxt = alt;
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
      k_cheb<<<grid_for(L.n, VT), VT, 0, h->stream>>>(L.n, L.rp.p, L.ci.p, L.v.p, L.dinv.p, b, c1,
                                                      c2, cur, L.d.p, nxt);
      MSS_LAUNCH_CK("k_cheb");
      double* t = cur;
      cur = nxt;
      nxt = t;
    }
    return cur;
  }
};

void vcycle_level(Handle* h, Hierarchy& H, int l, const double* b, double* out) {
  Level& L = H.lev[l];
  const mss_options& o = h->opt;
  const int n = L.n;
  if (l == (int)H.lev.size() - 1) {
    k_dense_gemv<<<grid_for((long long)n * 32, 256), 256, 0, h->stream>>>(n, H.coarse_inv.p, b,
                                                                          out);
    MSS_LAUNCH_CK("k_dense_gemv");
    return;
  }
  Sweeper sw{h, L, o};
  Level& C = H.lev[l + 1];
  // ---- pre-smoothing from zero, then the residual
  double* cur = out;
  double* alt = L.x2.p;
  if (o.smoother == MSS_JACOBI && o.nu_pre >= 1) {
    k_jacobi0_residual<<<grid_for(n, VT), VT, 0, h->stream>>>(n, L.rp.p, L.ci.p, L.v.p, L.dinv.p,
                                                              b, o.jacobi_omega, out, L.r.p);
    MSS_LAUNCH_CK("k_jacobi0_residual");
    for (int s = 1; s < o.nu_pre; ++s) {
      sw.jacobi(b, cur, alt);
      std::swap(cur, alt);
    }
    if (o.nu_pre > 1) {
      k_residual<<<grid_for(n, VT), VT, 0, h->stream>>>(n, L.rp.p, L.ci.p, L.v.p, b, cur, L.r.p);
      MSS_LAUNCH_CK("k_residual");
    }
  } else {
    fill_double(h, cur, 0.0, n);
    for (int s = 0; s < o.nu_pre; ++s) {
      double* res = sw.cheb(b, cur, alt);
      if (res != cur) std::swap(cur, alt);
    }
    k_residual<<<grid_for(n, VT), VT, 0, h->stream>>>(n, L.rp.p, L.ci.p, L.v.p, b, cur, L.r.p);
    MSS_LAUNCH_CK("k_residual");
  }
  // ---- restriction and the coarse correction
  k_csr_spmv<<<grid_for(L.nc, VT), VT, 0, h->stream>>>(L.nc, L.rrp.p, L.rci.p, L.rv.p, L.r.p,
                                                       C.b.p);
  MSS_LAUNCH_CK("k_csr_spmv(R)");
  vcycle_level(h, H, l + 1, C.b.p, C.x.p);
  k_prolong<<<grid_for(n, VT), VT, 0, h->stream>>>(n, L.prp.p, L.pci.p, L.pv.p, C.x.p, cur, alt);
  MSS_LAUNCH_CK("k_prolong");
  std::swap(cur, alt);
  // ---- post-smoothing
  for (int s = 0; s < o.nu_post; ++s) {
    if (o.smoother == MSS_JACOBI) {
      sw.jacobi(b, cur, alt);
      std::swap(cur, alt);
    } else {
      double* res = sw.cheb(b, cur, alt);
      if (res != cur) std::swap(cur, alt);
    }
  }
  if (cur != out) copy_dev(h, out, cur, sizeof(double) * (size_t)n);
}

}  // namespace

void coarse_inverse(Handle* h, Hierarchy& H) {
  Level& C = H.lev.back();
  const int n = C.n;
  if (n > 8192) fail(MSS_ERR_AMG, "coarsest AMG level has " + std::to_string(n) +
                                      " rows; raise amg_max_levels or amg_max_coarse");
  H.nc = n;
  H.coarse_inv.reset(h, (size_t)n * n);
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
  MSS_CK(cudaLaunchCooperativeKernel((const void*)k_gauss_jordan, dim3(blocks), dim3(threads),
                                     args, smem, h->stream));
  count_launch();
  int st = read_int(h, status.p);
  if (st != 0) fail(MSS_ERR_AMG, "coarsest AMG operator is singular (column " +
                                     std::to_string(st - 1) + ")");
  k_gj_extract<<<grid_for((long long)n * n, 256), 256, 0, h->stream>>>(n, M.p, piv.p,
                                                                       H.coarse_inv.p);
  MSS_LAUNCH_CK("k_gj_extract");
}

void vcycle(Handle* h, Hierarchy& H, const double* b, double* x) {
  TraceScope ts(h, TR_VCYCLE);
  vcycle_level(h, H, 0, b, x);
}

void gather_var(Handle* h, const double* v, int var, double* out) {
  k_gather_var<<<grid_for(h->N, 256), 256, 0, h->stream>>>(h->N, h->nb, v, var, out);
  MSS_LAUNCH_CK("k_gather_var");
}

void scatter_var_zero(Handle* h, const double* s, int var, double* out) {
  long long tot = (long long)h->N * h->nb;
  k_scatter_var_zero<<<grid_for(tot, 256), 256, 0, h->stream>>>(h->N, h->nb, s, var, out);
  MSS_LAUNCH_CK("k_scatter_var_zero");
}

void csr_block_pattern_spmv_sub(Handle* h, const double* vals, const double* x, const double* r,
                                int var, double* out) {
  k_pattern_sub<<<grid_for(h->N, 256), 256, 0, h->stream>>>(h->N, h->nb, h->rp.p, h->ci.p, vals,
                                                            x, r, var, out);
  MSS_LAUNCH_CK("k_pattern_sub");
}

}  // namespace mss
