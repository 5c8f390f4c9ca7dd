// krylov_kernels.cuh -- device bodies of the FGMRES kernels (Sec. 5.1).
//
// Each body takes the block index vb and the grid size G of its launch as
// arguments instead of reading blockIdx.x and gridDim.x, so that the same code
// runs as a kernel of one system (krylov.cu: vb = blockIdx.x, G = gridDim.x)
// and inside the multi-system tile walker of the batched solve (fused.cu: vb
// and G of the system's own launch shape). Either way every system computes
// the same values in the same order.
#pragma once

#include <vector>

#include "common.cuh"

namespace mss {

constexpr int KT = 256;         // threads per block of the streaming kernels
constexpr int kMaxRows = 128;   // projections per block: restart + 1 <= 121, and the norm

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

// device scalars of the recurrence (kscal): 0 hn, 1 rel. residual estimate,
// 2 happy-breakdown flag, 3 non-finite flag, 4 ||w0||, 6 ||r||^2, 7 ||bbar||^2
enum { KS_HN = 0, KS_REL = 1, KS_HAPPY = 2, KS_BAD = 3, KS_W0 = 4 };

namespace dev {

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

// Sets a while-loop condition when the kernel runs inside the solve graph.
__device__ __forceinline__ void set_cond(cudaGraphConditionalHandle c, int use, int v) {
  if (use) cudaGraphSetConditional(c, v ? 1u : 0u);
}

// Sum of v over the warp (the lanes' tree of block_sum).
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;   // valid in lane 0
}

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

// partial[row * G + vb] = sum over the warps of tab[row], rows < nrows
__device__ __forceinline__ void store_rows(const double* tab, int nrows, double* partial, int vb,
                                           int G) {
  constexpr int NW = KT / 32;
  __syncthreads();
  for (int t = threadIdx.x; t < nrows; t += KT) {
    double s = 0.0;
    for (int wv = 0; wv < NW; ++wv) s += tab[t * NW + wv];
    partial[(size_t)t * G + vb] = s;
  }
}

// partial[i * G + vb] = sum over block vb's chunk of V_i . w, i <= j;
// with wnorm, partial[(j + 1) * G + vb] = chunk sum of w . w
__device__ __forceinline__ void mdot(long long n, long long chunk, const double* __restrict__ V,
                                     long long ld, const GState* __restrict__ st,
                                     const double* __restrict__ w, int wnorm,
                                     double* __restrict__ partial, int vb, int G) {
  __shared__ double tab[kMaxRows * (KT / 32)];
  const int nv = st->j + 1;
  const long long s0 = (long long)vb * chunk;
  const long long s1 = s0 + chunk < n ? s0 + chunk : n;
  chunk_projections(V, ld, w, s0, s1, nv, tab);
  if (wnorm) {
    double a0 = 0;
    for (long long e = s0 + threadIdx.x; e < s1; e += KT) a0 += w[e] * w[e];
    a0 = warp_sum(a0);
    if ((threadIdx.x & 31) == 0) tab[nv * (KT / 32) + (threadIdx.x >> 5)] = a0;
  }
  store_rows(tab, nv + (wnorm ? 1 : 0), partial, vb, G);
}

// w -= sum_{i<=j} h_i V_i on the block's chunk, then either the projections
// of the updated w (mode 0) or its squared norm (mode 1)
__device__ __forceinline__ void update(long long n, long long chunk, const double* __restrict__ V,
                                       long long ld, const GState* __restrict__ st,
                                       const double* __restrict__ hcoef, double* __restrict__ w,
                                       int mode, double* __restrict__ partial, int vb, int G) {
  __shared__ double hs[128];
  __shared__ double red[KT / 32];
  const int nv = st->j + 1;
  for (int i = threadIdx.x; i < nv; i += KT) hs[i] = hcoef[i];
  __syncthreads();
  const long long s0 = (long long)vb * chunk;
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
    if (threadIdx.x == 0) partial[vb] = nrm;
    return;
  }
  // projections of the updated chunk (each thread re-reads its own elements)
  __shared__ double tab[kMaxRows * (KT / 32)];
  __syncthreads();
  chunk_projections(V, ld, w, s0, s1, nv, tab);
  store_rows(tab, nv, partial, vb, G);
}

// out[i] = sum_b partial[row_i * G + b] in a fixed order. mode 0: rows
// i <= j (launched with m + 1 blocks, the others return); mode 1: the single
// row j + 1; mode 2: the single row 0.
__device__ __forceinline__ void reduce(int G, const double* __restrict__ partial,
                                       double* __restrict__ out, const GState* __restrict__ st,
                                       int mode, int vb) {
  int row = vb, o = vb;
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

__device__ __forceinline__ void arnoldi_finish(int m, const double* __restrict__ h1,
                                               const double* __restrict__ h2,
                                               const double* __restrict__ sq,
                                               double* __restrict__ H, double* __restrict__ cs,
                                               double* __restrict__ sn, double* __restrict__ g,
                                               double* __restrict__ ks,
                                               const GState* __restrict__ st) {
  if (threadIdx.x != 0) return;
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
__device__ __forceinline__ void normalize_store(long long n, const double* __restrict__ w,
                                                const double* __restrict__ ks,
                                                double* __restrict__ V, long long ld,
                                                const GState* __restrict__ st,
                                                double* __restrict__ vnext, int vb, int G) {
  if (ks[KS_HAPPY] != 0.0) return;
  const double inv = 1.0 / ks[KS_HN];
  double* out = V + (size_t)(st->j + 1) * ld;
  long long e = (long long)vb * blockDim.x + threadIdx.x;
  const long long stride = (long long)G * blockDim.x;
  for (; e < n; e += stride) {
    const double v = w[e] * inv;
    out[e] = v;
    vnext[e] = v;
  }
}

// Z_j = z (the flexible basis keeps every preconditioned vector)
__device__ __forceinline__ void store_z(long long n, const double* __restrict__ z,
                                        double* __restrict__ Z, long long ld,
                                        const GState* __restrict__ st, int vb, int G) {
  double* out = Z + (size_t)st->j * ld;
  long long e = (long long)vb * blockDim.x + threadIdx.x;
  const long long stride = (long long)G * blockDim.x;
  for (; e < n; e += stride) out[e] = z[e];
}

// cycle start: V_0 = r / beta (also the first step's input)
__device__ __forceinline__ void cycle_head(long long n, const double* __restrict__ r,
                                           double* __restrict__ V, double* __restrict__ vnext,
                                           const GState* __restrict__ st, int vb, int G) {
  const double s = 1.0 / st->beta;
  long long e = (long long)vb * blockDim.x + threadIdx.x;
  const long long stride = (long long)G * blockDim.x;
  for (; e < n; e += stride) {
    const double v = r[e] * s;
    V[e] = v;
    vnext[e] = v;
  }
}

// g = beta e_1, j = k = 0; the cycle takes a step unless maxit is reached
__device__ __forceinline__ void init_g(int m, double* __restrict__ g, GState* __restrict__ st,
                                       cudaGraphConditionalHandle inner, int use, int vb) {
  int i = vb * blockDim.x + threadIdx.x;
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
__device__ __forceinline__ void step_control(int m, const double* __restrict__ ks,
                                             GState* __restrict__ st,
                                             cudaGraphConditionalHandle inner, int use) {
  if (threadIdx.x != 0) return;
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
__device__ __forceinline__ void backsolve(int m, const double* __restrict__ H,
                                          const double* __restrict__ g, double* __restrict__ y,
                                          const GState* __restrict__ st) {
  if (threadIdx.x != 0) return;
  const int k = st->status == MSS_ERR_BREAKDOWN ? 0 : st->k;
  for (int i = k - 1; i >= 0; --i) {
    double s = g[i];
    for (int q = i + 1; q < k; ++q) s -= H[(size_t)i * m + q] * y[q];
    y[i] = s / H[(size_t)i * m + i];
  }
}

// x += sum_{q<k} y_q Z_q
__device__ __forceinline__ void xupdate(long long n, const double* __restrict__ Z, long long ld,
                                        const double* __restrict__ y, double* __restrict__ x,
                                        const GState* __restrict__ st, int vb, int G) {
  __shared__ double ys[128];
  const int k = st->status == MSS_ERR_BREAKDOWN ? 0 : st->k;
  if (k == 0) return;
  for (int i = threadIdx.x; i < k; i += blockDim.x) ys[i] = y[i];
  __syncthreads();
  long long e = (long long)vb * blockDim.x + threadIdx.x;
  const long long stride = (long long)G * blockDim.x;
  for (; e < n; e += stride) {
    double acc = x[e];
    for (int q = 0; q < k; ++q) acc += ys[q] * Z[(size_t)q * ld + e];
    x[e] = acc;
  }
}

// r = b - Ax (in place of Ax), partial sums of ||r||^2
__device__ __forceinline__ void resid_norm(long long n, long long chunk,
                                           const double* __restrict__ b, double* __restrict__ r,
                                           double* __restrict__ partial, int vb) {
  __shared__ double red[KT / 32];
  const long long s0 = (long long)vb * chunk;
  const long long s1 = s0 + chunk < n ? s0 + chunk : n;
  double s = 0.0;
  for (long long e = s0 + threadIdx.x; e < s1; e += KT) {
    double v = b[e] - r[e];
    r[e] = v;
    s += v * v;
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0) partial[vb] = s;
}

__device__ __forceinline__ void sqnorm(long long n, long long chunk, const double* __restrict__ a,
                                       double* __restrict__ partial, int vb) {
  __shared__ double red[KT / 32];
  const long long s0 = (long long)vb * chunk;
  const long long s1 = s0 + chunk < n ? s0 + chunk : n;
  double s = 0.0;
  for (long long e = s0 + threadIdx.x; e < s1; e += KT) s += a[e] * a[e];
  s = block_sum(s, red);
  if (threadIdx.x == 0) partial[vb] = s;
}

// end of a cycle: true residual check (Sec. 5.1), then stop or restart
__device__ __forceinline__ void cycle_control(const double* __restrict__ ks,
                                              GState* __restrict__ st,
                                              cudaGraphConditionalHandle outer, int use) {
  if (threadIdx.x != 0) return;
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
__device__ __forceinline__ void solve_init(const double* __restrict__ ks, GState* __restrict__ st,
                                           cudaGraphConditionalHandle outer, int use) {
  if (threadIdx.x != 0) return;
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

}  // namespace dev

// Reduction shape of a vector of n entries: G blocks of chunk entries each.
struct Red {
  int G;
  long long chunk;
};

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

// Captures what fn enqueues on the handle's stream into graph g after the
// nodes deps; returns the single node the next work must follow.
template <class F>
inline cudaGraphNode_t capture_into(Handle* h, cudaGraph_t g, const cudaGraphNode_t* deps,
                                    size_t nd, long long* launches, F&& fn) {
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

inline cudaGraph_t add_while(cudaGraph_t g, cudaGraphNode_t dep, cudaGraphConditionalHandle c,
                             cudaGraphNode_t* node) {
  cudaGraphNodeParams prm = {};
  prm.type = cudaGraphNodeTypeConditional;
  prm.conditional.handle = c;
  prm.conditional.type = cudaGraphCondTypeWhile;
  prm.conditional.size = 1;
  MSS_CK(cudaGraphAddNode(node, g, &dep, nullptr, 1, &prm));
  return prm.conditional.phGraph_out[0];
}

// krylov.cu: allocates (or keeps) the handle's Krylov workspace for its
// current restart length and returns its pointers
Krylov workspace(Handle* h);

}  // namespace mss
