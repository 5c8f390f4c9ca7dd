// krylov.cu -- BSR matrix-vector product, preconditioner orchestration
// (Algorithms 1 and 2) and right-preconditioned restarted FGMRES (Sec. 5.1).
//
// Arnoldi uses classical Gram-Schmidt, once (CGS1, default) or twice (CGS2):
// every pass is one streaming sweep over the basis that computes all
// projections at once; CGS2 fuses its second projections into the first
// update, and the last update carries the norm. The FP64 work per element is
// 2(j+1) FMAs for CGS1 and 4(j+1) for CGS2. All
// reductions are two-stage with a fixed block count and a fixed summation
// order, so results are identical from run to run.
#include <cmath>
#include <vector>

#include "common.cuh"

namespace mss {
namespace {

constexpr int KT = 256;   // threads per block of the streaming kernels

// y = Abar x, NB lanes per block row (lane c produces component c)
template <int NB>
__global__ void k_bsr_spmv(int N, const int* __restrict__ rp, const int* __restrict__ ci,
                           const double* __restrict__ vals, const double* __restrict__ x,
                           double* __restrict__ y) {
  constexpr int RPW = 32 / NB;
  constexpr int B2 = NB * NB;
  const int lane = threadIdx.x & 31;
  const int sub = lane / NB, comp = lane - sub * NB;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long ii = warp * RPW + sub;
  if (sub >= RPW || ii >= N) return;
  const int i = (int)ii;
  double acc = 0.0;
  for (int e = rp[i]; e < rp[i + 1]; ++e) {
    const double* a = vals + (size_t)e * B2 + comp * NB;
    const double* xj = x + (size_t)ci[e] * NB;
#pragma unroll
    for (int c = 0; c < NB; ++c) acc += a[c] * xj[c];
  }
  y[(size_t)i * NB + comp] = acc;
}

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

// partial[i * G + b] = sum over block b's chunk of V_i . w, i < nv;
// with wnorm, partial[nv * G + b] = chunk sum of w . w
__global__ void k_mdot(long long n, long long chunk, const double* __restrict__ V, long long ld,
                       int nv, const double* __restrict__ w, int wnorm,
                       double* __restrict__ partial) {
  __shared__ double red[KT / 32];
  const long long s0 = (long long)blockIdx.x * chunk;
  const long long s1 = s0 + chunk < n ? s0 + chunk : n;
  const int G = gridDim.x;
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
    a0 = block_sum(a0, red);
    a1 = block_sum(a1, red);
    a2 = block_sum(a2, red);
    a3 = block_sum(a3, red);
    if (threadIdx.x == 0) {
      partial[(size_t)i * G + blockIdx.x] = a0;
      partial[(size_t)(i + 1) * G + blockIdx.x] = a1;
      partial[(size_t)(i + 2) * G + blockIdx.x] = a2;
      partial[(size_t)(i + 3) * G + blockIdx.x] = a3;
    }
  }
  for (; i < nv; ++i) {
    const double* v0 = V + (size_t)i * ld;
    double a0 = 0;
    for (long long e = s0 + threadIdx.x; e < s1; e += KT) a0 += v0[e] * w[e];
    a0 = block_sum(a0, red);
    if (threadIdx.x == 0) partial[(size_t)i * G + blockIdx.x] = a0;
  }
  if (wnorm) {
    double a0 = 0;
    for (long long e = s0 + threadIdx.x; e < s1; e += KT) a0 += w[e] * w[e];
    a0 = block_sum(a0, red);
    if (threadIdx.x == 0) partial[(size_t)nv * G + blockIdx.x] = a0;
  }
}

// w -= sum_i h_i V_i on the block's chunk, then either the projections of
// the updated w (mode 0) or its squared norm (mode 1)
__global__ void k_update(long long n, long long chunk, const double* __restrict__ V, long long ld,
                         int nv, const double* __restrict__ hcoef, double* __restrict__ w,
                         int mode, double* __restrict__ partial) {
  __shared__ double hs[128];
  __shared__ double red[KT / 32];
  for (int i = threadIdx.x; i < nv; i += KT) hs[i] = hcoef[i];
  __syncthreads();
  const long long s0 = (long long)blockIdx.x * chunk;
  const long long s1 = s0 + chunk < n ? s0 + chunk : n;
  const int G = gridDim.x;
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
  __syncthreads();
  // projections of the updated chunk (each thread re-reads its own elements)
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
    a0 = block_sum(a0, red);
    a1 = block_sum(a1, red);
    a2 = block_sum(a2, red);
    a3 = block_sum(a3, red);
    if (threadIdx.x == 0) {
      partial[(size_t)i * G + blockIdx.x] = a0;
      partial[(size_t)(i + 1) * G + blockIdx.x] = a1;
      partial[(size_t)(i + 2) * G + blockIdx.x] = a2;
      partial[(size_t)(i + 3) * G + blockIdx.x] = a3;
    }
  }
  for (; i < nv; ++i) {
    const double* v0 = V + (size_t)i * ld;
    double a0 = 0;
    for (long long e = s0 + threadIdx.x; e < s1; e += KT) a0 += v0[e] * w[e];
    a0 = block_sum(a0, red);
    if (threadIdx.x == 0) partial[(size_t)i * G + blockIdx.x] = a0;
  }
}

// out[i] = sum_b partial[i * G + b], fixed order
__global__ void k_reduce(int nv, int G, const double* __restrict__ partial,
                         double* __restrict__ out) {
  const int i = blockIdx.x;
  __shared__ double red[KT / 32];
  double s = 0.0;
  for (int b = threadIdx.x; b < G; b += KT) s += partial[(size_t)i * G + b];
  s = block_sum(s, red);
  if (threadIdx.x == 0) out[i] = s;
}

// device scalars of the recurrence (kscal): 0 hn, 1 rel. residual estimate,
// 2 happy-breakdown flag, 3 non-finite flag, 4 ||w0||
enum { KS_HN = 0, KS_REL = 1, KS_HAPPY = 2, KS_BAD = 3, KS_W0 = 4 };

// Hessenberg column j = h1 + h2, norm, Givens rotations, residual estimate
__global__ void k_arnoldi_finish(int j, int m, const double* __restrict__ h1,
                                 const double* __restrict__ h2, const double* __restrict__ sq,
                                 double* __restrict__ H, double* __restrict__ cs,
                                 double* __restrict__ sn, double* __restrict__ g, double bnorm,
                                 double* __restrict__ ks) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  // sq[0] = ||w0||^2 (before projection), sq[1] = ||w||^2 after CGS2
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

__global__ void k_normalize(long long n, double* __restrict__ w, const double* __restrict__ ks) {
  if (ks[KS_HAPPY] != 0.0) return;
  const double inv = 1.0 / ks[KS_HN];
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long stride = (long long)gridDim.x * blockDim.x;
  for (; e < n; e += stride) w[e] = w[e] * inv;
}

__global__ void k_scale(long long n, const double* __restrict__ src, double s,
                        double* __restrict__ dst) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long stride = (long long)gridDim.x * blockDim.x;
  for (; e < n; e += stride) dst[e] = src[e] * s;
}

__global__ void k_init_g(int m, double beta, double* __restrict__ g) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i <= m) g[i] = i == 0 ? beta : 0.0;
}

// y = H_k^{-1} g_k (upper triangular), single thread
__global__ void k_backsolve(int k, int m, const double* __restrict__ H,
                            const double* __restrict__ g, double* __restrict__ y) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = k - 1; i >= 0; --i) {
    double s = g[i];
    for (int q = i + 1; q < k; ++q) s -= H[(size_t)i * m + q] * y[q];
    y[i] = s / H[(size_t)i * m + i];
  }
}

// x += sum_q y_q Z_q
__global__ void k_xupdate(long long n, const double* __restrict__ Z, long long ld, int k,
                          const double* __restrict__ y, double* __restrict__ x) {
  __shared__ double ys[128];
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

template <int NB>
void spmv_nb(Handle* h, const double* x, double* y) {
  constexpr int RPW = 32 / NB;
  long long warps = (h->N + RPW - 1) / RPW;
  k_bsr_spmv<NB><<<grid_for(warps * 32, 256), 256, 0, h->stream>>>(h->N, h->rp.p, h->ci.p,
                                                                   h->abar.p, x, y);
  MSS_LAUNCH_CK("k_bsr_spmv");
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

double device_norm(Handle* h, const double* a, long long n, double* part, double* out) {
  Red rs = reduction_shape(h, n);
  k_sqnorm<<<rs.G, KT, 0, h->stream>>>(n, rs.chunk, a, part);
  MSS_LAUNCH_CK("k_sqnorm");
  k_reduce<<<1, KT, 0, h->stream>>>(1, rs.G, part, out);
  MSS_LAUNCH_CK("k_reduce");
  return std::sqrt(read_double(h, out));
}

}  // namespace

void bsr_spmv(Handle* h, const double* x, double* y) {
  TraceScope ts(h, TR_SPMV);
  MSS_NB_DISPATCH(h->nb, spmv_nb<NB>(h, x, y));
}

// y = M^{-1} r: Algorithm 2 (CPTR3), Algorithm 1 (CPR) or the last stage only
// Mixed form of the same stages: BF16 operator blocks and factors, FP32
// vectors and arithmetic; r and y stay FP64 (the Krylov vectors).
static void precond_apply_mixed(Handle* h, const double* r, double* y) {
  const int scheme = h->opt.scheme;
  if (scheme == MSS_ILU0) {
    last_stage_apply(h, r, (const float*)nullptr, (const float*)nullptr, y);
    return;
  }
  if (scheme == MSS_CPR) {
    gather_var(h, r, h->p, h->rTf.p);
    vcycle_mixed(h, h->amgP, h->rTf.p, h->vPf.p);
    last_stage_apply(h, r, (const float*)nullptr, h->vPf.p, y);
    return;
  }
  if (h->opt.stage_order == MSS_STAGE_T_FIRST) {
    gather_var(h, r, h->t, h->rTf.p);
    vcycle_mixed(h, h->amgT, h->rTf.p, h->xTf.p);
    csr_block_pattern_spmv_sub(h, h->aptf.p, h->xTf.p, r, h->p, h->zPf.p);
    vcycle_mixed(h, h->amgP, h->zPf.p, h->vPf.p);
  } else {
    gather_var(h, r, h->p, h->rTf.p);
    vcycle_mixed(h, h->amgP, h->rTf.p, h->vPf.p);
    csr_block_pattern_spmv_sub(h, h->atpf.p, h->vPf.p, r, h->t, h->zPf.p);
    vcycle_mixed(h, h->amgT, h->zPf.p, h->xTf.p);
  }
  last_stage_apply(h, r, h->xTf.p, h->vPf.p, y);
}

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
  if (scheme == MSS_CPR) {
    gather_var(h, r, h->p, h->rT.p);
    vcycle(h, h->amgP, h->rT.p, h->vP.p);                  // x = M1 r (pressure)
    last_stage_apply(h, r, (const double*)nullptr, h->vP.p, y);          // y = x + M2 (r - Abar x)
    return;
  }
  if (h->opt.stage_order == MSS_STAGE_T_FIRST) {
    gather_var(h, r, h->t, h->rT.p);
    vcycle(h, h->amgT, h->rT.p, h->xT.p);                  // x = M1 r (temperature)
    csr_block_pattern_spmv_sub(h, h->apt.p, h->xT.p, r, h->p, h->zP.p);   // z_P
    vcycle(h, h->amgP, h->zP.p, h->vP.p);                  // v = M2 z (pressure)
  } else {
    gather_var(h, r, h->p, h->rT.p);
    vcycle(h, h->amgP, h->rT.p, h->vP.p);                  // x = M1 r (pressure)
    csr_block_pattern_spmv_sub(h, h->atp.p, h->vP.p, r, h->t, h->zP.p);   // z_T
    vcycle(h, h->amgT, h->zP.p, h->xT.p);                  // v = M2 z (temperature)
  }
  last_stage_apply(h, r, h->xT.p, h->vP.p, y);             // y = x + v + M3 u
}

int fgmres(Handle* h, const double* b, double* x, double tol, int maxit, mss_result* out) {
  const long long n = (long long)h->N * h->nb;
  const int m = h->opt.restart;
  const long long ld = (n + 31) / 32 * 32;
  if (h->m != m || h->V.n < (size_t)(m + 1) * ld) {
    h->m = m;
    h->V.reset(h, (size_t)(m + 1) * ld);
    h->Z.reset(h, (size_t)m * ld);
    h->bbar.reset(h, ld);
    h->res.reset(h, ld);
    // hbuf: H (m+1)m | cs m | sn m | g m+1 | y m | h1 m+1 | h2 m+1 | sq 2
    h->hbuf.reset(h, (size_t)(m + 1) * m + 7 * (size_t)(m + 2));
    h->kscal.reset(h, 8);
  }
  Red rs = reduction_shape(h, n);
  if (h->part.n < (size_t)(m + 2) * rs.G) h->part.reset(h, (size_t)(m + 2) * rs.G);
  double* H = h->hbuf.p;
  double* cs = H + (size_t)(m + 1) * m;
  double* sn = cs + (m + 2);
  double* g = sn + (m + 2);
  double* yv = g + (m + 2);
  double* h1 = yv + (m + 2);
  double* h2 = h1 + (m + 2);
  double* sq = h2 + (m + 2);
  double* ks = h->kscal.p;
  double* part = h->part.p;
  double* V = h->V.p;
  double* Z = h->Z.p;

  mss_result res{};
  res.status = MSS_OK;
  scale_vector(h, b, h->bbar.p);
  fill_double(h, x, 0.0, n);
  double bnorm = device_norm(h, h->bbar.p, n, part, ks + 7);
  if (!std::isfinite(bnorm)) fail(MSS_ERR_BREAKDOWN, "right-hand side is not finite");
  if (bnorm == 0.0) {
    if (out) *out = res;
    return MSS_OK;
  }
  copy_dev(h, h->res.p, h->bbar.p, sizeof(double) * (size_t)n);
  double beta = bnorm;
  int total = 0;
  const unsigned sgrid = grid_for(n, 256) > 4096 ? 4096 : grid_for(n, 256);
  for (;;) {
    k_scale<<<sgrid, 256, 0, h->stream>>>(n, h->res.p, 1.0 / beta, V);
    MSS_LAUNCH_CK("k_scale");
    k_init_g<<<1, 128, 0, h->stream>>>(m, beta, g);   // restart <= 120
    MSS_LAUNCH_CK("k_init_g");
    int k = 0;
    bool happy = false;
    for (int j = 0; j < m; ++j) {
      if (total >= maxit) break;
      double* vj = V + (size_t)j * ld;
      double* zj = Z + (size_t)j * ld;
      double* w = V + (size_t)(j + 1) * ld;
      precond_apply(h, vj, zj);
      bsr_spmv(h, zj, w);
      const int nv = j + 1;
      {
        TraceScope ts(h, TR_ORTHO);
        // CGS pass 1: h1 = V^T w and ||w0||^2
        k_mdot<<<rs.G, KT, 0, h->stream>>>(n, rs.chunk, V, ld, nv, w, 1, part);
        MSS_LAUNCH_CK("k_mdot");
        k_reduce<<<nv, KT, 0, h->stream>>>(nv, rs.G, part, h1);
        MSS_LAUNCH_CK("k_reduce");
        k_reduce<<<1, KT, 0, h->stream>>>(1, rs.G, part + (size_t)nv * rs.G, sq);
        MSS_LAUNCH_CK("k_reduce");
        const bool cgs2 = h->opt.orthog == MSS_CGS2;
        if (cgs2) {
          // update with h1, fused pass-2 projections h2
          k_update<<<rs.G, KT, 0, h->stream>>>(n, rs.chunk, V, ld, nv, h1, w, 0, part);
          MSS_LAUNCH_CK("k_update");
          k_reduce<<<nv, KT, 0, h->stream>>>(nv, rs.G, part, h2);
          MSS_LAUNCH_CK("k_reduce");
        }
        // update (with h2 after CGS2, with h1 after CGS1) and the norm
        k_update<<<rs.G, KT, 0, h->stream>>>(n, rs.chunk, V, ld, nv, cgs2 ? h2 : h1, w, 1, part);
        MSS_LAUNCH_CK("k_update");
        k_reduce<<<1, KT, 0, h->stream>>>(1, rs.G, part, sq + 1);
        MSS_LAUNCH_CK("k_reduce");
        k_arnoldi_finish<<<1, 32, 0, h->stream>>>(j, m, h1, cgs2 ? h2 : nullptr, sq, H, cs, sn,
                                                  g, bnorm, ks);
        MSS_LAUNCH_CK("k_arnoldi_finish");
        k_normalize<<<sgrid, 256, 0, h->stream>>>(n, w, ks);
        MSS_LAUNCH_CK("k_normalize");
      }
      double hks[5];
      MSS_CK(cudaMemcpyAsync(hks, ks, sizeof(hks), cudaMemcpyDeviceToHost, h->stream));
      MSS_CK(cudaStreamSynchronize(h->stream));
      ++total;
      k = j + 1;
      res.rel_res_implicit = hks[KS_REL];
      if (hks[KS_BAD] != 0.0 || !std::isfinite(hks[KS_REL])) {
        res.iters = total;
        res.status = MSS_ERR_BREAKDOWN;
        if (out) *out = res;
        fail(MSS_ERR_BREAKDOWN, "non-finite or zero Givens denominator");
      }
      happy = hks[KS_HAPPY] != 0.0;
      if (hks[KS_REL] <= tol || happy) break;
    }
    if (k > 0) {
      k_backsolve<<<1, 32, 0, h->stream>>>(k, m, H, g, yv);
      MSS_LAUNCH_CK("k_backsolve");
      k_xupdate<<<sgrid, 256, 0, h->stream>>>(n, Z, ld, k, yv, x);
      MSS_LAUNCH_CK("k_xupdate");
    }
    bsr_spmv(h, x, h->res.p);
    k_resid_norm<<<rs.G, KT, 0, h->stream>>>(n, rs.chunk, h->bbar.p, h->res.p, part);
    MSS_LAUNCH_CK("k_resid_norm");
    k_reduce<<<1, KT, 0, h->stream>>>(1, rs.G, part, ks + 6);
    MSS_LAUNCH_CK("k_reduce");
    beta = std::sqrt(read_double(h, ks + 6));
    res.rel_res_true = beta / bnorm;
    res.iters = total;
    if (!std::isfinite(beta)) {
      res.status = MSS_ERR_BREAKDOWN;
      break;
    }
    if (res.rel_res_true <= tol) break;
    if (total >= maxit || k == 0) {
      res.status = MSS_ERR_NOT_CONVERGED;
      break;
    }
    res.restarts++;
  }
  if (out) *out = res;
  return res.status;
}

}  // namespace mss
