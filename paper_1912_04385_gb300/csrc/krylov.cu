// krylov.cu -- preconditioner orchestration (Algorithms 1 and 2) and
// right-preconditioned restarted FGMRES (Sec. 5.1).
//
// Arnoldi uses classical Gram-Schmidt, once (CGS1, default) or twice (CGS2):
// every pass is one streaming sweep over the basis that computes all
// projections at once; CGS2 fuses its second projections into the first
// update, and the last update carries the norm. The FP64 work per element is
// 2(j+1) FMAs for CGS1 and 4(j+1) for CGS2. All
// reductions are two-stage with a fixed block count and a fixed summation
// order, so results are identical from run to run.
//
// The solve state (step j, counts, norms, status) lives in device memory and
// every kernel reads j from it, so one fixed sequence of launches performs any
// Arnoldi step. Two drivers run that sequence: a host loop that reads the
// state back after each step, or one CUDA graph holding the whole restarted
// solve, whose two nested while-loop conditional nodes (restart cycles,
// Arnoldi steps) are continued or ended by the control kernels. Both run the
// same kernels in the same order and give the same bits.
#include <cmath>
#include <vector>

#include "common.cuh"

namespace mss {
namespace {

constexpr int KT = 256;   // threads per block of the streaming kernels

__device__ __forceinline__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  __syncthreads();
  return s;   // valid in thread 0
}


// Device solve state. Written by the control kernels only (single thread).
struct GState {
  int j;          // Arnoldi step of the current cycle (0-based)
  int k;          // steps completed in the current cycle
  int total;      // inner iterations in total
  int restarts;   // completed restart cycles
  int status;     // MSS_OK, or MSS_ERR_NOT_CONVERGED / MSS_ERR_BREAKDOWN
  int go_inner;   // 1 while the current cycle takes another step
  int go_outer;   // 1 while another cycle is needed
  int maxit;
  int rhs_bad;    // ||bbar|| is not finite
  int done;       // the solve has ended
  double tol, bnorm, beta, rel_impl, rel_true;
};
static_assert(sizeof(GState) <= 16 * sizeof(double), "GState fits its buffer");

// Sets a while-loop condition when the kernel runs inside the solve graph.
__device__ __forceinline__ void set_cond(cudaGraphConditionalHandle c, int use, int v) {
  if (use) cudaGraphSetConditional(c, v ? 1u : 0u);
}

// Sum of v over the warp (the lanes' tree of block_sum).
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;   // valid in lane 0
}

constexpr int kMaxRows = 128;   // projections per block: restart + 1 <= 121, and the norm

// Projections of w on the block's chunk, rows i0 <= i < nv, four at a time:
// the warps' sums go to tab[row][warp]; the block sums are formed after one
// barrier (warp by warp, as in block_sum).
__device__ __forceinline__ void chunk_projections(const double* __restrict__ V, long long ld,
                                                  const double* __restrict__ w, long long s0,
                                                  long long s1, int nv, double* tab) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  constexpr int NW = KT / 32;
  int i = 0;
  for (; i + 4 <= nv; i += 4) {
    const double* v0 = V + (size_t)i * ld;
    double a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    for (long long e = s0 + threadIdx.x; e < s1; e += KT) {
      double we = w[e];
      a0 += v0[e] * we;
      a1 += v0[ld + e] * we;
      a2 += v0[2 * ld + e] * we;
      a3 += v0[3 * ld + e] * we;
    }
    a0 = warp_sum(a0);
    a1 = warp_sum(a1);
    a2 = warp_sum(a2);
    a3 = warp_sum(a3);
    if (lane == 0) {
      tab[i * NW + wid] = a0;
      tab[(i + 1) * NW + wid] = a1;
      tab[(i + 2) * NW + wid] = a2;
      tab[(i + 3) * NW + wid] = a3;
    }
  }
  for (; i < nv; ++i) {
    const double* v0 = V + (size_t)i * ld;
    double a0 = 0;
    for (long long e = s0 + threadIdx.x; e < s1; e += KT) a0 += v0[e] * w[e];
    a0 = warp_sum(a0);
    if (lane == 0) tab[i * NW + wid] = a0;
  }
}

// partial[row * G + b] = sum over the warps of tab[row], rows < nrows
__device__ __forceinline__ void store_rows(const double* tab, int nrows, double* partial) {
  constexpr int NW = KT / 32;
  __syncthreads();
  const int G = gridDim.x;
  for (int t = threadIdx.x; t < nrows; t += KT) {
    double s = 0.0;
    for (int wv = 0; wv < NW; ++wv) s += tab[t * NW + wv];
    partial[(size_t)t * G + blockIdx.x] = s;
  }
}

// partial[i * G + b] = sum over block b's chunk of V_i . w, i <= j;
// with wnorm, partial[(j + 1) * G + b] = chunk sum of w . w
__global__ void k_mdot(long long n, long long chunk, const double* __restrict__ V, long long ld,
                       const GState* __restrict__ st, const double* __restrict__ w, int wnorm,
                       double* __restrict__ partial) {
  __shared__ double tab[kMaxRows * (KT / 32)];
  const int nv = st->j + 1;
  const long long s0 = (long long)blockIdx.x * chunk;
  const long long s1 = s0 + chunk < n ? s0 + chunk : n;
  chunk_projections(V, ld, w, s0, s1, nv, tab);
  if (wnorm) {
    double a0 = 0;
    for (long long e = s0 + threadIdx.x; e < s1; e += KT) a0 += w[e] * w[e];
    a0 = warp_sum(a0);
    if ((threadIdx.x & 31) == 0) tab[nv * (KT / 32) + (threadIdx.x >> 5)] = a0;
  }
  store_rows(tab, nv + (wnorm ? 1 : 0), partial);
}

// w -= sum_{i<=j} h_i V_i on the block's chunk, then either the projections
// of the updated w (mode 0) or its squared norm (mode 1)
__global__ void k_update(long long n, long long chunk, const double* __restrict__ V, long long ld,
                         const GState* __restrict__ st, const double* __restrict__ hcoef,
                         double* __restrict__ w, int mode, double* __restrict__ partial) {
  __shared__ double hs[128];
  __shared__ double red[KT / 32];
  const int nv = st->j + 1;
  for (int i = threadIdx.x; i < nv; i += KT) hs[i] = hcoef[i];
  __syncthreads();
  const long long s0 = (long long)blockIdx.x * chunk;
  const long long s1 = s0 + chunk < n ? s0 + chunk : n;
  double nrm = 0.0;
  for (long long e = s0 + threadIdx.x; e < s1; e += KT) {
    double acc = w[e];
    for (int i = 0; i < nv; ++i) acc -= hs[i] * V[(size_t)i * ld + e];
    w[e] = acc;
    nrm += acc * acc;
  }
  if (mode == 1) {
    nrm = block_sum(nrm, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = nrm;
    return;
  }
  // projections of the updated chunk (each thread re-reads its own elements)
  __shared__ double tab[kMaxRows * (KT / 32)];
  __syncthreads();
  chunk_projections(V, ld, w, s0, s1, nv, tab);
  store_rows(tab, nv, partial);
}

// out[i] = sum_b partial[row_i * G + b] in a fixed order. mode 0: rows
// i <= j (launched with m + 1 blocks, the others return); mode 1: the single
// row j + 1; mode 2: the single row 0.
__global__ void k_reduce(int G, const double* __restrict__ partial, double* __restrict__ out,
                         const GState* __restrict__ st, int mode) {
  int row = blockIdx.x, o = blockIdx.x;
  if (mode == 0) {
    if (row > st->j) return;
  } else {
    row = mode == 1 ? st->j + 1 : 0;
    o = 0;
  }
  __shared__ double red[KT / 32];
  double s = 0.0;
  for (int b = threadIdx.x; b < G; b += KT) s += partial[(size_t)row * G + b];
  s = block_sum(s, red);
  if (threadIdx.x == 0) out[o] = s;
}

// device scalars of the recurrence (kscal): 0 hn, 1 rel. residual estimate,
// 2 happy-breakdown flag, 3 non-finite flag, 4 ||w0||, 6 ||r||^2, 7 ||bbar||^2
enum { KS_HN = 0, KS_REL = 1, KS_HAPPY = 2, KS_BAD = 3, KS_W0 = 4 };

__global__ void k_arnoldi_finish(int m, const double* __restrict__ h1,
                                 const double* __restrict__ h2, const double* __restrict__ sq,
                                 double* __restrict__ H, double* __restrict__ cs,
                                 double* __restrict__ sn, double* __restrict__ g,
                                 double* __restrict__ ks, const GState* __restrict__ st) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int j = st->j;
  const double bnorm = st->bnorm;
  // sq[0] = ||w0||^2 (before projection), sq[1] = ||w||^2 after the update
  double w0 = sqrt(sq[0]);
  double hn = sqrt(sq[1]);
  for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = h2 ? h1[i] + h2[i] : h1[i];
  H[(size_t)(j + 1) * m + j] = hn;
  int happy = hn <= 1e-14 * w0;
  for (int i = 0; i < j; ++i) {
    double a = H[(size_t)i * m + j], b = H[(size_t)(i + 1) * m + j];
    H[(size_t)i * m + j] = cs[i] * a + sn[i] * b;
    H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * b;
  }
  double a = H[(size_t)j * m + j], b = H[(size_t)(j + 1) * m + j];
  double den = hypot(a, b);
  int bad = !(den > 0.0) || !isfinite(den);
  double c = bad ? 1.0 : a / den, s = bad ? 0.0 : b / den;
  cs[j] = c;
  sn[j] = s;
  H[(size_t)j * m + j] = den;
  H[(size_t)(j + 1) * m + j] = 0.0;
  g[j + 1] = -s * g[j];
  g[j] = c * g[j];
  ks[KS_HN] = hn;
  ks[KS_REL] = fabs(g[j + 1]) / bnorm;
  ks[KS_HAPPY] = happy;
  ks[KS_BAD] = bad;
  ks[KS_W0] = w0;
}

// V_{j+1} = w / h_{j+1,j}, also into the next step's input vector
__global__ void k_normalize_store(long long n, const double* __restrict__ w,
                                  const double* __restrict__ ks, double* __restrict__ V,
                                  long long ld, const GState* __restrict__ st,
                                  double* __restrict__ vnext) {
  if (ks[KS_HAPPY] != 0.0) return;
  const double inv = 1.0 / ks[KS_HN];
  double* out = V + (size_t)(st->j + 1) * ld;
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long stride = (long long)gridDim.x * blockDim.x;
  for (; e < n; e += stride) {
    const double v = w[e] * inv;
    out[e] = v;
    vnext[e] = v;
  }
}

// Z_j = z (the flexible basis keeps every preconditioned vector)
__global__ void k_store_z(long long n, const double* __restrict__ z, double* __restrict__ Z,
                          long long ld, const GState* __restrict__ st) {
  double* out = Z + (size_t)st->j * ld;
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long stride = (long long)gridDim.x * blockDim.x;
  for (; e < n; e += stride) out[e] = z[e];
}

// cycle start: V_0 = r / beta (also the first step's input), g = beta e_1,
// j = k = 0; the cycle takes a step unless maxit is already reached
__global__ void k_cycle_head(long long n, const double* __restrict__ r, double* __restrict__ V,
                             double* __restrict__ vnext, GState* __restrict__ st) {
  const double s = 1.0 / st->beta;
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long stride = (long long)gridDim.x * blockDim.x;
  for (; e < n; e += stride) {
    const double v = r[e] * s;
    V[e] = v;
    vnext[e] = v;
  }
}

__global__ void k_init_g(int m, double* __restrict__ g, GState* __restrict__ st,
                         cudaGraphConditionalHandle inner, int use) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i <= m) g[i] = i == 0 ? st->beta : 0.0;
  if (i == 0) {
    st->j = 0;
    st->k = 0;
    st->go_inner = st->total < st->maxit;
    set_cond(inner, use, st->go_inner);
  }
}

// after an Arnoldi step: count it, stop the cycle on convergence of the
// implicit residual, a happy breakdown, a full basis or maxit
__global__ void k_step_control(int m, const double* __restrict__ ks, GState* __restrict__ st,
                               cudaGraphConditionalHandle inner, int use) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  st->total += 1;
  st->k = st->j + 1;
  st->rel_impl = ks[KS_REL];
  int go;
  if (ks[KS_BAD] != 0.0 || !isfinite(ks[KS_REL])) {
    st->status = MSS_ERR_BREAKDOWN;
    go = 0;
  } else {
    const bool stop = ks[KS_REL] <= st->tol || ks[KS_HAPPY] != 0.0 || st->k >= m ||
                      st->total >= st->maxit;
    go = !stop;
    if (go) st->j += 1;
  }
  st->go_inner = go;
  set_cond(inner, use, go);
}

// y = H_k^{-1} g_k (upper triangular), single thread; nothing after a breakdown
__global__ void k_backsolve(int m, const double* __restrict__ H, const double* __restrict__ g,
                            double* __restrict__ y, const GState* __restrict__ st) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int k = st->status == MSS_ERR_BREAKDOWN ? 0 : st->k;
  for (int i = k - 1; i >= 0; --i) {
    double s = g[i];
    for (int q = i + 1; q < k; ++q) s -= H[(size_t)i * m + q] * y[q];
    y[i] = s / H[(size_t)i * m + i];
  }
}

// x += sum_{q<k} y_q Z_q
__global__ void k_xupdate(long long n, const double* __restrict__ Z, long long ld,
                          const double* __restrict__ y, double* __restrict__ x,
                          const GState* __restrict__ st) {
  __shared__ double ys[128];
  const int k = st->status == MSS_ERR_BREAKDOWN ? 0 : st->k;
  if (k == 0) return;
  for (int i = threadIdx.x; i < k; i += blockDim.x) ys[i] = y[i];
  __syncthreads();
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long stride = (long long)gridDim.x * blockDim.x;
  for (; e < n; e += stride) {
    double acc = x[e];
    for (int q = 0; q < k; ++q) acc += ys[q] * Z[(size_t)q * ld + e];
    x[e] = acc;
  }
}

// r = b - Ax (in place of Ax), partial sums of ||r||^2
__global__ void k_resid_norm(long long n, long long chunk, const double* __restrict__ b,
                             double* __restrict__ r, double* __restrict__ partial) {
  __shared__ double red[KT / 32];
  const long long s0 = (long long)blockIdx.x * chunk;
  const long long s1 = s0 + chunk < n ? s0 + chunk : n;
  double s = 0.0;
  for (long long e = s0 + threadIdx.x; e < s1; e += KT) {
    double v = b[e] - r[e];
    r[e] = v;
    s += v * v;
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void k_sqnorm(long long n, long long chunk, const double* __restrict__ a,
                         double* __restrict__ partial) {
  __shared__ double red[KT / 32];
  const long long s0 = (long long)blockIdx.x * chunk;
  const long long s1 = s0 + chunk < n ? s0 + chunk : n;
  double s = 0.0;
  for (long long e = s0 + threadIdx.x; e < s1; e += KT) s += a[e] * a[e];
  s = block_sum(s, red);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// end of a cycle: true residual check (Sec. 5.1), then stop or restart
__global__ void k_cycle_control(const double* __restrict__ ks, GState* __restrict__ st,
                                cudaGraphConditionalHandle outer, int use) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int go = 0;
  if (st->status != MSS_ERR_BREAKDOWN) {
    const double beta = sqrt(ks[6]);
    st->beta = beta;
    st->rel_true = beta / st->bnorm;
    if (!isfinite(beta)) {
      st->status = MSS_ERR_BREAKDOWN;
    } else if (st->rel_true <= st->tol) {
      st->status = MSS_OK;
    } else if (st->total >= st->maxit || st->k == 0) {
      st->status = MSS_ERR_NOT_CONVERGED;
    } else {
      st->restarts += 1;
      go = 1;
    }
  }
  st->go_outer = go;
  st->done = !go;
  set_cond(outer, use, go);
}

// solve start: ||bbar||; nothing to do for a zero right-hand side
__global__ void k_solve_init(const double* __restrict__ ks, GState* __restrict__ st,
                             cudaGraphConditionalHandle outer, int use) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double bnorm = sqrt(ks[7]);
  st->bnorm = bnorm;
  st->beta = bnorm;
  st->j = st->k = st->total = st->restarts = 0;
  st->status = MSS_OK;
  st->rel_impl = st->rel_true = 0.0;
  st->rhs_bad = !isfinite(bnorm);
  int go = 1;
  if (st->rhs_bad) {
    st->status = MSS_ERR_BREAKDOWN;
    go = 0;
  } else if (bnorm == 0.0) {
    go = 0;
  }
  st->go_outer = go;
  st->done = !go;
  set_cond(outer, use, go);
}

struct Red {
  int G;
  long long chunk;
};

Red reduction_shape(Handle* h, long long n) {
  Red r;
  long long g = (n + 4095) / 4096;
  long long cap = 4LL * h->num_sms;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  r.G = (int)g;
  r.chunk = (n + g - 1) / g;
  r.chunk = (r.chunk + 31) / 32 * 32;
  return r;
}

// Pointers and shapes of one solve's Krylov workspace.
struct Krylov {
  long long n, ld;
  int m;
  Red rs;
  unsigned sgrid;
  double *H, *cs, *sn, *g, *yv, *h1, *h2, *sq, *ks, *part, *V, *Z;
  double *rfix, *zfix, *wfix;
  GState* st;
};

Krylov workspace(Handle* h) {
  Krylov K;
  K.n = (long long)h->N * h->nb;
  K.m = h->opt.restart;
  K.ld = (K.n + 31) / 32 * 32;
  const int m = K.m;
  auto drop_graph = [&] {   // the solve graph holds pointers into the workspace
    if (h->sgraph) cudaGraphExecDestroy(h->sgraph);
    h->sgraph = nullptr;
  };
  if (h->m != m || h->V.n < (size_t)(m + 1) * K.ld) {
    drop_graph();
    h->m = m;
    h->V.reset(h, (size_t)(m + 1) * K.ld);
    h->Z.reset(h, (size_t)m * K.ld);
    h->bbar.reset(h, K.ld);
    h->res.reset(h, K.ld);
    // hbuf: H (m+1)m | cs m | sn m | g m+1 | y m | h1 m+1 | h2 m+1 | sq 2
    h->hbuf.reset(h, (size_t)(m + 1) * m + 7 * (size_t)(m + 2));
    h->kscal.reset(h, 8);
    h->gst.reset(h, 16);
    h->rfix.reset(h, K.ld);
    h->zfix.reset(h, K.ld);
    h->wfix.reset(h, K.ld);
  }
  K.rs = reduction_shape(h, K.n);
  if (h->part.n < (size_t)(m + 2) * K.rs.G) {
    drop_graph();
    h->part.reset(h, (size_t)(m + 2) * K.rs.G);
  }
  K.sgrid = grid_for(K.n, 256) > 4096 ? 4096 : grid_for(K.n, 256);
  K.H = h->hbuf.p;
  K.cs = K.H + (size_t)(m + 1) * m;
  K.sn = K.cs + (m + 2);
  K.g = K.sn + (m + 2);
  K.yv = K.g + (m + 2);
  K.h1 = K.yv + (m + 2);
  K.h2 = K.h1 + (m + 2);
  K.sq = K.h2 + (m + 2);
  K.ks = h->kscal.p;
  K.part = h->part.p;
  K.V = h->V.p;
  K.Z = h->Z.p;
  K.rfix = h->rfix.p;
  K.zfix = h->zfix.p;
  K.wfix = h->wfix.p;
  K.st = reinterpret_cast<GState*>(h->gst.p);
  return K;
}

// ---- the four launch sequences of a solve ----------------------------------
// bbar = N^{-1} b, x = 0, ||bbar||, r = bbar
void seq_init(Handle* h, const Krylov& K, const double* b, double* x,
              cudaGraphConditionalHandle outer, int use) {
  scale_vector(h, b, h->bbar.p);
  fill_double(h, x, 0.0, K.n);
  k_sqnorm<<<K.rs.G, KT, 0, h->stream>>>(K.n, K.rs.chunk, h->bbar.p, K.part);
  MSS_LAUNCH_CK("k_sqnorm");
  k_reduce<<<1, KT, 0, h->stream>>>(K.rs.G, K.part, K.ks + 7, K.st, 2);
  MSS_LAUNCH_CK("k_reduce");
  k_solve_init<<<1, 32, 0, h->stream>>>(K.ks, K.st, outer, use);
  MSS_LAUNCH_CK("k_solve_init");
  copy_dev(h, h->res.p, h->bbar.p, sizeof(double) * (size_t)K.n);
}

void seq_head(Handle* h, const Krylov& K, cudaGraphConditionalHandle inner, int use) {
  k_cycle_head<<<K.sgrid, 256, 0, h->stream>>>(K.n, h->res.p, K.V, K.rfix, K.st);
  MSS_LAUNCH_CK("k_cycle_head");
  k_init_g<<<1, 128, 0, h->stream>>>(K.m, K.g, K.st, inner, use);   // restart <= 120
  MSS_LAUNCH_CK("k_init_g");
}

// one Arnoldi step j: z_j = M^{-1} v_j, w = Abar z_j, orthogonalise, normalise
void seq_step(Handle* h, const Krylov& K, cudaGraphConditionalHandle inner, int use) {
  const long long n = K.n;
  const Red rs = K.rs;
  precond_apply(h, K.rfix, K.zfix);
  k_store_z<<<K.sgrid, 256, 0, h->stream>>>(n, K.zfix, K.Z, K.ld, K.st);
  MSS_LAUNCH_CK("k_store_z");
  bsr_spmv(h, K.zfix, K.wfix);
  TraceScope ts(h, TR_ORTHO);
  const bool cgs2 = h->opt.orthog == MSS_CGS2;
  // CGS pass 1: h1 = V^T w and ||w0||^2
  k_mdot<<<rs.G, KT, 0, h->stream>>>(n, rs.chunk, K.V, K.ld, K.st, K.wfix, 1, K.part);
  MSS_LAUNCH_CK("k_mdot");
  k_reduce<<<K.m + 1, KT, 0, h->stream>>>(rs.G, K.part, K.h1, K.st, 0);
  MSS_LAUNCH_CK("k_reduce");
  k_reduce<<<1, KT, 0, h->stream>>>(rs.G, K.part, K.sq, K.st, 1);
  MSS_LAUNCH_CK("k_reduce");
  if (cgs2) {
    // update with h1, fused pass-2 projections h2
    k_update<<<rs.G, KT, 0, h->stream>>>(n, rs.chunk, K.V, K.ld, K.st, K.h1, K.wfix, 0, K.part);
    MSS_LAUNCH_CK("k_update");
    k_reduce<<<K.m + 1, KT, 0, h->stream>>>(rs.G, K.part, K.h2, K.st, 0);
    MSS_LAUNCH_CK("k_reduce");
  }
  // update (with h2 after CGS2, with h1 after CGS1) and the norm
  k_update<<<rs.G, KT, 0, h->stream>>>(n, rs.chunk, K.V, K.ld, K.st, cgs2 ? K.h2 : K.h1, K.wfix,
                                       1, K.part);
  MSS_LAUNCH_CK("k_update");
  k_reduce<<<1, KT, 0, h->stream>>>(rs.G, K.part, K.sq + 1, K.st, 2);
  MSS_LAUNCH_CK("k_reduce");
  k_arnoldi_finish<<<1, 32, 0, h->stream>>>(K.m, K.h1, cgs2 ? K.h2 : nullptr, K.sq, K.H, K.cs,
                                            K.sn, K.g, K.ks, K.st);
  MSS_LAUNCH_CK("k_arnoldi_finish");
  k_normalize_store<<<K.sgrid, 256, 0, h->stream>>>(n, K.wfix, K.ks, K.V, K.ld, K.st, K.rfix);
  MSS_LAUNCH_CK("k_normalize_store");
  k_step_control<<<1, 32, 0, h->stream>>>(K.m, K.ks, K.st, inner, use);
  MSS_LAUNCH_CK("k_step_control");
}

// end of a cycle: x += Z_k y_k, true residual, stop or restart
void seq_tail(Handle* h, const Krylov& K, double* x, cudaGraphConditionalHandle outer, int use) {
  k_backsolve<<<1, 32, 0, h->stream>>>(K.m, K.H, K.g, K.yv, K.st);
  MSS_LAUNCH_CK("k_backsolve");
  k_xupdate<<<K.sgrid, 256, 0, h->stream>>>(K.n, K.Z, K.ld, K.yv, x, K.st);
  MSS_LAUNCH_CK("k_xupdate");
  bsr_spmv(h, x, h->res.p);
  k_resid_norm<<<K.rs.G, KT, 0, h->stream>>>(K.n, K.rs.chunk, h->bbar.p, h->res.p, K.part);
  MSS_LAUNCH_CK("k_resid_norm");
  k_reduce<<<1, KT, 0, h->stream>>>(K.rs.G, K.part, K.ks + 6, K.st, 2);
  MSS_LAUNCH_CK("k_reduce");
  k_cycle_control<<<1, 32, 0, h->stream>>>(K.ks, K.st, outer, use);
  MSS_LAUNCH_CK("k_cycle_control");
}

GState read_state(Handle* h, const Krylov& K) {
  GState s;
  read_back(h, &s, K.st, sizeof(GState));
  return s;
}

void write_params(Handle* h, const Krylov& K, double tol, int maxit) {
  GState s{};
  s.tol = tol;
  s.maxit = maxit;
  write_to_device(h, K.st, &s, sizeof(GState));
}

int finish(const GState& s, mss_result* out) {
  mss_result res{};
  res.iters = s.total;
  res.restarts = s.restarts;
  res.status = s.status;
  res.rel_res_implicit = s.rel_impl;
  res.rel_res_true = s.rel_true;
  if (out) *out = res;
  if (s.rhs_bad) fail(MSS_ERR_BREAKDOWN, "right-hand side is not finite");
  if (s.status == MSS_ERR_BREAKDOWN)
    fail(MSS_ERR_BREAKDOWN, "non-finite value or zero Givens denominator in the Arnoldi process");
  return s.status;
}

// Host-driven: the state is read back after every step and every cycle.
int fgmres_host(Handle* h, const Krylov& K, const double* b, double* x, double tol, int maxit,
                mss_result* out) {
  const cudaGraphConditionalHandle none = 0;
  write_params(h, K, tol, maxit);
  seq_init(h, K, b, x, none, 0);
  GState s = read_state(h, K);
  while (s.go_outer) {
    seq_head(h, K, none, 0);
    bool go = s.total < maxit;
    while (go) {
      seq_step(h, K, none, 0);
      s = read_state(h, K);
      if (s.status == MSS_ERR_BREAKDOWN) return finish(s, out);
      go = s.go_inner;
    }
    seq_tail(h, K, x, none, 0);
    s = read_state(h, K);
  }
  return finish(s, out);
}

// Captures what fn enqueues on the handle's stream into graph g after the
// nodes deps; returns the single node the next work must follow.
template <class F>
cudaGraphNode_t capture_into(Handle* h, cudaGraph_t g, const cudaGraphNode_t* deps, size_t nd,
                             long long* launches, F&& fn) {
  MSS_CK(cudaStreamBeginCaptureToGraph(h->stream, g, deps, nullptr, nd,
                                       cudaStreamCaptureModeThreadLocal));
  *launches = 0;
  capture_count(launches);
  h->capturing = true;
  try {
    fn();
  } catch (...) {
    capture_count(nullptr);
    h->capturing = false;
    cudaGraph_t dummy = nullptr;
    cudaStreamEndCapture(h->stream, &dummy);
    throw;
  }
  capture_count(nullptr);
  h->capturing = false;
  cudaStreamCaptureStatus cst;
  const cudaGraphNode_t* tail = nullptr;
  size_t nt = 0;
  MSS_CK(cudaStreamGetCaptureInfo(h->stream, &cst, nullptr, nullptr, &tail, nullptr, &nt));
  std::vector<cudaGraphNode_t> last(tail, tail + nt);
  cudaGraph_t same = nullptr;
  MSS_CK(cudaStreamEndCapture(h->stream, &same));
  if (last.size() == 1) return last[0];
  cudaGraphNode_t join;
  MSS_CK(cudaGraphAddEmptyNode(&join, g, last.data(), last.size()));
  return join;
}

cudaGraph_t add_while(cudaGraph_t g, cudaGraphNode_t dep, cudaGraphConditionalHandle c,
                      cudaGraphNode_t* node) {
  cudaGraphNodeParams prm = {};
  prm.type = cudaGraphNodeTypeConditional;
  prm.conditional.handle = c;
  prm.conditional.type = cudaGraphCondTypeWhile;
  prm.conditional.size = 1;
  MSS_CK(cudaGraphAddNode(node, g, &dep, nullptr, 1, &prm));
  return prm.conditional.phGraph_out[0];
}

// init -> while (cycle) { head -> while (step) { step } -> tail }
void build_solve_graph(Handle* h, const Krylov& K) {
  if (h->sgraph) {
    cudaGraphExecDestroy(h->sgraph);
    h->sgraph = nullptr;
  }
  h->gb.reset(h, K.ld);
  h->gx.reset(h, K.ld);
  // capture on a private non-blocking stream (the handle's stream may be the
  // legacy default stream, which cannot be captured); launched on h->stream
  MSS_CK(cudaStreamSynchronize(h->stream));
  cudaStream_t cap = nullptr;
  MSS_CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  const cudaStream_t saved = h->stream;
  h->stream = cap;
  cudaGraph_t top = nullptr;
  auto restore = [&] {
    h->stream = saved;
    cudaStreamDestroy(cap);
    if (top) cudaGraphDestroy(top);
  };
  MSS_CK(cudaGraphCreate(&top, 0));
  try {
    cudaGraphConditionalHandle outer, inner;
    MSS_CK(cudaGraphConditionalHandleCreate(&outer, top, 0, cudaGraphCondAssignDefault));
    cudaGraphNode_t n0 = capture_into(h, top, nullptr, 0, &h->sg_launch[0],
                                      [&] { seq_init(h, K, h->gb.p, h->gx.p, outer, 1); });
    cudaGraphNode_t wo;
    cudaGraph_t ob = add_while(top, n0, outer, &wo);
    MSS_CK(cudaGraphConditionalHandleCreate(&inner, ob, 0, cudaGraphCondAssignDefault));
    cudaGraphNode_t n1 = capture_into(h, ob, nullptr, 0, &h->sg_launch[1],
                                      [&] { seq_head(h, K, inner, 1); });
    cudaGraphNode_t wi;
    cudaGraph_t ib = add_while(ob, n1, inner, &wi);
    capture_into(h, ib, nullptr, 0, &h->sg_launch[2], [&] { seq_step(h, K, inner, 1); });
    capture_into(h, ob, &wi, 1, &h->sg_launch[3], [&] { seq_tail(h, K, h->gx.p, outer, 1); });
    MSS_CK(cudaGraphInstantiate(&h->sgraph, top, 0));
  } catch (...) {
    restore();
    throw;
  }
  restore();
  h->sg_m = K.m;
  h->sg_n = K.n;
}

// Device-driven: one graph launch per solve, one read-back at the end.
int fgmres_graph(Handle* h, const Krylov& K, const double* b, double* x, double tol, int maxit,
                 mss_result* out) {
  if (!h->sgraph || h->sg_m != K.m || h->sg_n != K.n) build_solve_graph(h, K);
  write_params(h, K, tol, maxit);
  copy_dev(h, h->gb.p, b, sizeof(double) * (size_t)K.n);
  MSS_CK(cudaGraphLaunch(h->sgraph, h->stream));
  copy_dev(h, x, h->gx.p, sizeof(double) * (size_t)K.n);
  GState s = read_state(h, K);
  const long long cycles = (s.rhs_bad || s.bnorm == 0.0) ? 0 : s.restarts + 1;
  add_launches(h->sg_launch[0] + cycles * (h->sg_launch[1] + h->sg_launch[3]) +
               (long long)s.total * h->sg_launch[2]);
  return finish(s, out);
}

}  // namespace

// Mixed form of the same stages: BF16 operator blocks and factors, FP32
// vectors and arithmetic; r and y stay FP64 (the Krylov vectors).
static void precond_apply_mixed(Handle* h, const double* r, double* y) {
  const int scheme = h->opt.scheme;
  if (scheme == MSS_ILU0) {
    last_stage_apply(h, r, (const float*)nullptr, (const float*)nullptr, y);
    return;
  }
  // each kernel that forms a V-cycle's right-hand side also writes its first
  // Jacobi sweep from zero into the V-cycle's output vector
  if (scheme == MSS_CPR) {
    gather_var(h, r, h->p, h->rTf.p, sweep0_mixed(h, h->amgP, h->vPf.p));
    vcycle_mixed(h, h->amgP, h->rTf.p, h->vPf.p, true);
    last_stage_apply(h, r, (const float*)nullptr, h->vPf.p, y);
    return;
  }
  if (scheme == MSS_CPTR) {
    gather_pair(h, r, h->rEf.p);
    vcycle_mixed(h, h->amgP, h->rEf.p, h->xEf.p);
    split_pair(h, (const float*)h->xEf.p, h->vPf.p, h->xTf.p);
    last_stage_apply(h, r, h->xTf.p, h->vPf.p, y);
    return;
  }
  if (h->opt.stage_order == MSS_STAGE_T_FIRST) {
    gather_var(h, r, h->t, h->rTf.p, sweep0_mixed(h, h->amgT, h->xTf.p));
    vcycle_mixed(h, h->amgT, h->rTf.p, h->xTf.p, true);
    csr_block_pattern_spmv_sub(h, h->aptf.p, h->xTf.p, r, h->p, h->zPf.p,
                               sweep0_mixed(h, h->amgP, h->vPf.p));
    vcycle_mixed(h, h->amgP, h->zPf.p, h->vPf.p, true);
  } else {
    gather_var(h, r, h->p, h->rTf.p, sweep0_mixed(h, h->amgP, h->vPf.p));
    vcycle_mixed(h, h->amgP, h->rTf.p, h->vPf.p, true);
    csr_block_pattern_spmv_sub(h, h->atpf.p, h->vPf.p, r, h->t, h->zPf.p,
                               sweep0_mixed(h, h->amgT, h->xTf.p));
    vcycle_mixed(h, h->amgT, h->zPf.p, h->xTf.p, true);
  }
  last_stage_apply(h, r, h->xTf.p, h->vPf.p, y);
}

// y = M^{-1} r: Algorithm 2 (CPTR3), Algorithm 1 (CPR), its CPTR form, or the
// last stage only
void precond_apply(Handle* h, const double* r, double* y) {
  TraceScope ts(h, TR_APPLY);
  if (h->opt.precision == MSS_MIXED) {
    precond_apply_mixed(h, r, y);
    return;
  }
  const int scheme = h->opt.scheme;
  if (scheme == MSS_ILU0) {
    last_stage_apply(h, r, (const double*)nullptr, (const double*)nullptr, y);
    return;
  }
  // each kernel that forms a V-cycle's right-hand side also writes its first
  // Jacobi sweep from zero into the V-cycle's output vector
  if (scheme == MSS_CPR) {
    gather_var(h, r, h->p, h->rT.p, sweep0(h, h->amgP, h->vP.p));
    vcycle(h, h->amgP, h->rT.p, h->vP.p, true);            // x = M1 r (pressure)
    last_stage_apply(h, r, (const double*)nullptr, h->vP.p, y);          // y = x + M2 (r - Abar x)
    return;
  }
  if (scheme == MSS_CPTR) {
    // Sec. 4.2: x_e = M_ee^{-1} r_e by the system AMG on (P, T) (Eq. CPTRM1),
    // then y = x + ilu(Abar)^{-1} (r - Abar x) with x = x_e at (p, t)
    gather_pair(h, r, h->rE.p);
    vcycle(h, h->amgP, h->rE.p, h->xE.p);
    split_pair(h, (const double*)h->xE.p, h->vP.p, h->xT.p);
    last_stage_apply(h, r, h->xT.p, h->vP.p, y);
    return;
  }
  if (h->opt.stage_order == MSS_STAGE_T_FIRST) {
    gather_var(h, r, h->t, h->rT.p, sweep0(h, h->amgT, h->xT.p));
    vcycle(h, h->amgT, h->rT.p, h->xT.p, true);            // x = M1 r (temperature)
    csr_block_pattern_spmv_sub(h, h->apt.p, h->xT.p, r, h->p, h->zP.p,    // z_P
                               sweep0(h, h->amgP, h->vP.p));
    vcycle(h, h->amgP, h->zP.p, h->vP.p, true);            // v = M2 z (pressure)
  } else {
    gather_var(h, r, h->p, h->rT.p, sweep0(h, h->amgP, h->vP.p));
    vcycle(h, h->amgP, h->rT.p, h->vP.p, true);            // x = M1 r (pressure)
    csr_block_pattern_spmv_sub(h, h->atp.p, h->vP.p, r, h->t, h->zP.p,    // z_T
                               sweep0(h, h->amgT, h->xT.p));
    vcycle(h, h->amgT, h->zP.p, h->xT.p, true);            // v = M2 z (temperature)
  }
  last_stage_apply(h, r, h->xT.p, h->vP.p, y);             // y = x + v + M3 u
}


int fgmres(Handle* h, const double* b, double* x, double tol, int maxit, mss_result* out) {
  Krylov K = workspace(h);
  const int st = h->opt.driver == MSS_DRIVER_GRAPH ? fgmres_graph(h, K, b, x, tol, maxit, out)
                                                   : fgmres_host(h, K, b, x, tol, maxit, out);
  check_tail(h, h->amgT);
  check_tail(h, h->amgP);
  return st;
}

}  // namespace mss
