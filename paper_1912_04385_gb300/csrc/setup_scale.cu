// setup_scale.cu -- pattern validation, left scaling N^{-1} (Sec. 4, Eqs.
// CPR, CPTR31, CPTR32) and subsystem extraction.
//
// This translation unit is compiled with -fmad=false: every product and sum
// rounds separately, in the order written, so the scaled matrix feeds the
// AMG set-up (whose strength tests turn floating point into index decisions)
// with values that do not depend on instruction selection.
#include "common.cuh"
#include "vec_rows.cuh"

namespace mss {
namespace {

// error codes written to the flag (first error wins through atomicMin)
enum { VAL_OK = 0x7fffffff, VAL_ROWPTR = 1, VAL_COLS = 2, VAL_NODIAG = 3, VAL_ASYM = 4 };

__global__ void k_validate(const int* __restrict__ rp, const int* __restrict__ ci, int N,
                           int nnzb, int* __restrict__ diag, int* __restrict__ flag) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  int b = rp[i], e = rp[i + 1];
  if ((i == 0 && b != 0) || (i == N - 1 && e != nnzb) || e < b || b < 0 || e > nnzb) {
    atomicMin(flag, VAL_ROWPTR);
    diag[i] = -1;
    return;
  }
  int d = -1;
  for (int k = b; k < e; ++k) {
    int j = ci[k];
    if (j < 0 || j >= N || (k > b && j <= ci[k - 1])) {
      atomicMin(flag, VAL_COLS);
      diag[i] = -1;
      return;
    }
    if (j == i) d = k;
  }
  diag[i] = d;
  if (d < 0) {
    atomicMin(flag, VAL_NODIAG);
    return;
  }
  // structural symmetry: i must appear in every neighbour's row
  for (int k = b; k < e; ++k) {
    int j = ci[k];
    if (j == i) continue;
    int lo = rp[j], hi = rp[j + 1] - 1;
    if (lo < 0 || hi >= nnzb) {
      atomicMin(flag, VAL_ROWPTR);
      return;
    }
    bool found = false;
    while (lo <= hi) {
      int mid = (lo + hi) >> 1;
      int c = ci[mid];
      if (c == i) { found = true; break; }
      if (c < i) lo = mid + 1; else hi = mid - 1;
    }
    if (!found) {
      atomicMin(flag, VAL_ASYM);
      return;
    }
  }
}

// W = N^{-1} restricted to one cell, built from the cell's diagonal block D
// (read through src): only rows p and t differ from the identity, stored as
// wrows[i][0][:] (row p) and wrows[i][1][:] (row t).
// scheme: 0 CPTR3 (Eq. CPTR31 then Eq. CPTR32), 1 CPR (Eq. CPR), 2 none,
// 3 CPTR (Eq. CPTR1: the N1 of Eq. CPTR31 alone).
//
// The inverse of the sub-block D_xx (x = s for CPTR3/CPTR, h = all but p for
// CPR) is formed by Gauss-Jordan without pivoting on the whole NB x NB block
// with the rows and columns outside x replaced by the identity: pivoting
// only on the x positions, in ascending order, performs on the x-by-x part
// exactly the operations, in the same order, of the elimination on the
// compacted sub-block (the other entries are zero and never enter it), while
// every array index is a compile-time constant, so the work stays in
// registers. One division per pivot (the row is scaled by its reciprocal),
// updates as fused multiply-adds; the same
// arithmetic as the FP64 definition, so the scaled blocks match it bit for
// bit.
template <int NB>
__device__ bool build_w_cell(const double* src, bool col_major, int p, int t, int scheme,
                             double (&wp)[NB], double (&wt)[NB]) {
  auto D = [&](int r, int c) { return col_major ? src[c * NB + r] : src[r * NB + c]; };
#pragma unroll
  for (int k = 0; k < NB; ++k) {
    wp[k] = (k == p) ? 1.0 : 0.0;
    wt[k] = (k == t) ? 1.0 : 0.0;
  }
  if (scheme == 2) return true;
  // x: the eliminated unknowns
  auto in_x = [&](int k) { return scheme == 1 ? k != p : (k != p && k != t); };
  double a[NB][NB], inv[NB][NB];
  // the elimination fully unrolled (register arrays) up to 8 unknowns; larger
  // blocks run the same operations in loops (fast compilation, same values)
  constexpr int U = NB <= 8 ? NB : 1;
#pragma unroll
  for (int r = 0; r < NB; ++r)
#pragma unroll
    for (int c = 0; c < NB; ++c) {
      a[r][c] = (in_x(r) && in_x(c)) ? D(r, c) : (r == c ? 1.0 : 0.0);
      inv[r][c] = r == c ? 1.0 : 0.0;
    }
#pragma unroll U
  for (int k = 0; k < NB; ++k) {
    if (!in_x(k)) continue;
    const double piv = a[k][k];
    if (piv == 0.0 || !isfinite(piv)) return false;
    const double rpiv = 1.0 / piv;     // the pivot row scaled by the reciprocal
#pragma unroll U
    for (int j = 0; j < NB; ++j) {
      if (!in_x(j)) continue;
      a[k][j] = a[k][j] * rpiv;
      inv[k][j] = inv[k][j] * rpiv;
    }
#pragma unroll U
    for (int i = 0; i < NB; ++i) {
      if (i == k || !in_x(i)) continue;
      const double f = a[i][k];
#pragma unroll U
      for (int j = 0; j < NB; ++j) {
        if (!in_x(j)) continue;
        a[i][j] = fma(-f, a[k][j], a[i][j]);
        inv[i][j] = fma(-f, inv[k][j], inv[i][j]);
      }
    }
  }
  // w = -D_e,x D_xx^{-1} for the scaled rows e (p; and t for CPTR3 / CPTR)
#pragma unroll U
  for (int c = 0; c < NB; ++c) {
    if (!in_x(c)) continue;
    double vp = 0.0, vt = 0.0;
#pragma unroll U
    for (int r = 0; r < NB; ++r) {
      if (!in_x(r)) continue;
      vp = fma(D(p, r), inv[r][c], vp);
      if (scheme != 1) vt = fma(D(t, r), inv[r][c], vt);
    }
    wp[c] = -vp;
    if (scheme != 1) wt[c] = -vt;
  }
  if (scheme == 0) {
    // once-scaled entries B_PP and B_Tp of N1^{-1} D, then the N2 factor
    double bpp = 0.0, btp = 0.0;
#pragma unroll
    for (int k = 0; k < NB; ++k) {
      bpp = fma(wp[k], D(k, p), bpp);
      btp = fma(wt[k], D(k, p), btp);
    }
    if (bpp == 0.0 || !isfinite(bpp)) return false;
    const double cc = btp / bpp;
#pragma unroll
    for (int k = 0; k < NB; ++k) wt[k] = fma(-cc, wp[k], wt[k]);
  }
  return true;
}

// One thread per cell: W_i from the diagonal block (see build_w_cell).
template <int NB>
__global__ void k_build_w(const double* __restrict__ vals, const int* __restrict__ diag, int N,
                          int p, int t, int scheme, int col_major, double* __restrict__ wrows,
                          int* __restrict__ flag, double* __restrict__ dcopy) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double* src = vals + (size_t)diag[i] * NB * NB;
  if (dcopy) {   // the block as stored, for k_apply_w (host-resident values are read once)
    for (int k = 0; k < NB * NB; ++k) dcopy[(size_t)i * NB * NB + k] = src[k];
    src = dcopy + (size_t)i * NB * NB;
  }
  double wp[NB], wt[NB];
  if (!build_w_cell<NB>(src, col_major != 0, p, t, scheme, wp, wt)) {
    atomicMin(flag, i);
    return;
  }
  double* out = wrows + (size_t)i * 2 * NB;
#pragma unroll
  for (int k = 0; k < NB; ++k) {
    out[k] = wp[k];
    out[NB + k] = wt[k];
  }
}

// block -> block row map
__global__ void k_block_rows(int N, const int* __restrict__ rp, int* __restrict__ brow) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  for (int e = rp[i]; e < rp[i + 1]; ++e) brow[e] = i;
}

// One thread per block column (block e, column c): the rows of W that are
// not unit vectors (p, and t for CPTR3) give Abar_ij[r][c] = sum_k W_i[r][k]
// J_ij[k][c] (ascending k); the other rows are copied. Every lane of a warp
// does the same FP64 work (FP64 issue is the bound of this kernel on GB300).
// The threads of columns p and t also write the entries of the scalar
// subsystems (Extract), so no later pass reads one entry per 8 nb^2 bytes.
template <int NB>
__global__ void k_apply_w(const double* __restrict__ vals, const int* __restrict__ brow,
                          long long nnzb, int p, int t, int scheme, int col_major,
                          const double* __restrict__ wrows, double* __restrict__ abar,
                          const int* __restrict__ diag, const double* __restrict__ dcopy,
                          Extract ex) {
  constexpr int B2 = NB * NB;
  long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= nnzb * NB) return;
  const long long e = tid / NB;
  const int c = (int)(tid - e * NB);
  const double* src = vals + (size_t)e * B2;
  if (dcopy) {   // diagonal blocks from the device copy k_build_w made
    const int i = brow[e];
    if (diag[i] == e) src = dcopy + (size_t)i * B2;
  }
  double col[NB];
#pragma unroll
  for (int k = 0; k < NB; ++k) col[k] = col_major ? src[c * NB + k] : src[k * NB + c];
  double* dst = abar + (size_t)e * B2 + c;
#pragma unroll
  for (int r = 0; r < NB; ++r) dst[r * NB] = col[r];
  double rowp = col[p], rowt = col[t];   // the final entries (p, c) and (t, c)
  if (scheme != 2) {
    const double* w = wrows + (size_t)brow[e] * 2 * NB;
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < NB; ++k) acc = fma(w[k], col[k], acc);
    dst[p * NB] = acc;
    rowp = acc;
    if (scheme == 0 || scheme == 3) {
      double acc2 = 0.0;
#pragma unroll
      for (int k = 0; k < NB; ++k) acc2 = fma(w[NB + k], col[k], acc2);
      dst[t * NB] = acc2;
      rowt = acc2;
    }
  }
  if (c == p) {
    if (ex.pp) ex.pp[e] = rowp;
    if (ex.tp) ex.tp[e] = rowt;
  }
  if (c == t) {
    if (ex.tt) ex.tt[e] = rowt;
    if (ex.pt) ex.pt[e] = rowp;
  }
}

template <int NB>
__global__ void k_scale_vec(const double* __restrict__ b, int N, int p, int t, int scheme,
                            const double* __restrict__ wrows, double* __restrict__ out) {
  dev::scale_vec_entry<NB>((long long)blockIdx.x * blockDim.x + threadIdx.x, b, N, p, t, scheme,
                           wrows, out);
}


// B_ee of CPTR: out[4e + 2k + l] = Abar_e[e_k][e_l], e = (p, t)
__global__ void k_extract_pair(const double* __restrict__ abar, int nnzb, int nb, int p, int t,
                               double* __restrict__ out) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nnzb) return;
  const double* a = abar + (size_t)e * nb * nb;
  out[(size_t)4 * e + 0] = a[p * nb + p];
  out[(size_t)4 * e + 1] = a[p * nb + t];
  out[(size_t)4 * e + 2] = a[t * nb + p];
  out[(size_t)4 * e + 3] = a[t * nb + t];
}

template <int NB>
void build_scaling_nb(Handle* h, const double* vals, bool col_major, const Extract& ex) {
  int N = h->N;
  int scheme = h->opt.scheme;
  DBuf<int> flag(h, 1);
  fill_int(h, flag.p, 0x7fffffff, 1);
  // values in host memory are read over the host link: k_build_w keeps a
  // device copy of the diagonal blocks so that k_apply_w reads each block once
  DBuf<double> dcopy;
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, vals) == cudaSuccess && at.type == cudaMemoryTypeHost)
    dcopy.reset(h, (size_t)N * NB * NB);
  else
    cudaGetLastError();
  k_build_w<NB><<<grid_for(N, 128), 128, 0, h->stream>>>(vals, h->diag.p, N, h->p, h->t, scheme,
                                                         col_major, h->wrows.p, flag.p, dcopy.p);
  MSS_LAUNCH_CK("k_build_w");
  int bad = read_int(h, flag.p);
  if (bad != 0x7fffffff)
    fail(MSS_ERR_SINGULAR_BLOCK,
         "cell " + std::to_string(bad) + ": diagonal block needs pivoting (zero pivot)");
  DBuf<int> brow(h, h->nnzb);
  k_block_rows<<<grid_for(N, 256), 256, 0, h->stream>>>(N, h->rp.p, brow.p);
  MSS_LAUNCH_CK("k_block_rows");
  long long tot = (long long)h->nnzb * NB;
  k_apply_w<NB><<<grid_for(tot, 256), 256, 0, h->stream>>>(vals, brow.p, h->nnzb, h->p, h->t,
                                                           scheme, col_major, h->wrows.p,
                                                           h->abar.p, h->diag.p, dcopy.p, ex);
  MSS_LAUNCH_CK("k_apply_w");
}

template <int NB>
void scale_vector_nb(Handle* h, const double* b, double* bbar) {
  long long tot = (long long)h->N * NB;
  k_scale_vec<NB><<<grid_for(tot, 256), 256, 0, h->stream>>>(b, h->N, h->p, h->t,
                                                             h->opt.scheme, h->wrows.p, bbar);
  MSS_LAUNCH_CK("k_scale_vec");
}

}  // namespace

void validate_pattern(Handle* h, const int* rp, const int* ci, int N, int nnzb, int* diag) {
  DBuf<int> flag(h, 1);
  fill_int(h, flag.p, VAL_OK, 1);
  k_validate<<<grid_for(N, 256), 256, 0, h->stream>>>(rp, ci, N, nnzb, diag, flag.p);
  MSS_LAUNCH_CK("k_validate");
  int f = read_int(h, flag.p);
  switch (f) {
    case VAL_OK: return;
    case VAL_ROWPTR: fail(MSS_ERR_INVALID_ARG, "row_ptr is not a valid offset array");
    case VAL_COLS: fail(MSS_ERR_INVALID_ARG, "col_idx out of range or not strictly ascending");
    case VAL_NODIAG: fail(MSS_ERR_INVALID_ARG, "a row has no diagonal block");
    default: fail(MSS_ERR_INVALID_ARG, "block pattern is not structurally symmetric");
  }
}

void build_scaling(Handle* h, const double* vals, bool col_major, const Extract& ex) {
  MSS_NB_DISPATCH(h->nb, build_scaling_nb<NB>(h, vals, col_major, ex));
}

void scale_vector(Handle* h, const double* b, double* bbar) {
  MSS_NB_DISPATCH(h->nb, scale_vector_nb<NB>(h, b, bbar));
}

void extract_pair(Handle* h, double* out) {
  k_extract_pair<<<grid_for(h->nnzb, 256), 256, 0, h->stream>>>(h->abar.p, h->nnzb, h->nb, h->p,
                                                                 h->t, out);
  MSS_LAUNCH_CK("k_extract_pair");
}

}  // namespace mss
