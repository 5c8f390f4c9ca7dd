// bilu.cu -- last stage of the multi-stage preconditioner: block ILU(0) of
// the scaled matrix (Eq. CPTR3M3; the CPR second stage) in a multicolour
// ordering, or block Jacobi, plus the fused stage arithmetic around it.
//
// Ordering: Jones-Plassmann colouring with SplitMix64 priorities; cells are
// renumbered colour-major (ascending cell index inside a colour), so that
// every colour is a contiguous range of "positions" and the factor blocks
// of a colour are contiguous in memory. The factorisation and both
// triangular sweeps then run one launch per colour; cells of one colour are
// never adjacent, so each launch is fully parallel.
//
// Apply (Algorithm 2, fused): the forward sweep forms
//   u = r - Abar[:,t] x_T - Abar[:,p] v_P
// on the fly from per-block column slices, and the backward sweep writes
//   y = x + v + M3 u
// directly, so u, z and the intermediate stage vectors are never stored.
// Sweeps use NB lanes per cell row (lane c owns component c), so a row's
// nb x nb blocks are read as contiguous rows by adjacent lanes.
#include <algorithm>

#include "common.cuh"

namespace mss {
namespace {

// ---- colouring ------------------------------------------------------------
__global__ void k_jp_pick(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                          uint64_t seed, const int* __restrict__ colour, int* __restrict__ pick) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int chosen = -1;
  if (colour[i] < 0) {
    uint64_t pi = splitmix64(seed, (0xFFFFULL << 32) | (uint64_t)(unsigned)i);
    bool best = true;
    for (int k = rp[i]; k < rp[i + 1] && best; ++k) {
      int j = ci[k];
      if (j == i || colour[j] >= 0) continue;
      uint64_t pj = splitmix64(seed, (0xFFFFULL << 32) | (uint64_t)(unsigned)j);
      if (pj > pi || (pj == pi && j > i)) best = false;
    }
    if (best) {
      int c = 0;
      for (;;) {
        bool used = false;
        for (int k = rp[i]; k < rp[i + 1]; ++k)
          if (ci[k] != i && colour[ci[k]] == c) { used = true; break; }
        if (!used) break;
        ++c;
      }
      chosen = c;
    }
  }
  pick[i] = chosen;
}

__global__ void k_jp_commit(int n, const int* __restrict__ pick, int* __restrict__ colour,
                            int* __restrict__ left, int* __restrict__ maxcol) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (pick[i] >= 0) {
    colour[i] = pick[i];
    atomicMax(maxcol, pick[i]);
  } else if (colour[i] < 0) {
    atomicAdd(left, 1);
  }
}

__global__ void k_flag_colour(int n, const int* __restrict__ colour, int c, int* __restrict__ f) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) f[i] = colour[i] == c ? 1 : 0;
}

__global__ void k_place_colour(int n, const int* __restrict__ colour, int c, int base,
                               const int* __restrict__ rank, int* __restrict__ iperm,
                               int* __restrict__ perm) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || colour[i] != c) return;
  int q = base + rank[i];
  iperm[i] = q;
  perm[q] = i;
}

__global__ void k_perm_rowlen(int n, const int* __restrict__ perm, const int* __restrict__ rp,
                              int* __restrict__ len) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) len[q] = rp[perm[q] + 1] - rp[perm[q]];
}

// factor pattern of row q (cell perm[q]) sorted by column position; copies
// the scaled blocks and the column slices [Abar[:, t] | Abar[:, p]]
template <int NB>
__global__ void k_fill_factor(int n, const int* __restrict__ perm, const int* __restrict__ iperm,
                              const int* __restrict__ rp, const int* __restrict__ ci,
                              const double* __restrict__ abar, int p, int t,
                              const int* __restrict__ frp, int* __restrict__ fpos,
                              int* __restrict__ fcell, int* __restrict__ fdp,
                              double* __restrict__ fv, double* __restrict__ fcs) {
  constexpr int B2 = NB * NB;
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  int i = perm[q];
  int b = rp[i], len = rp[i + 1] - b, base = frp[q];
  // insertion sort of (position, source block) pairs
  for (int a = 0; a < len; ++a) {
    int e = b + a;
    int pc = iperm[ci[e]];
    int k = a - 1;
    while (k >= 0 && fpos[base + k] > pc) {
      fpos[base + k + 1] = fpos[base + k];
      fcell[base + k + 1] = fcell[base + k];
      --k;
    }
    fpos[base + k + 1] = pc;
    fcell[base + k + 1] = ci[e];
  }
  int d = -1;
  for (int a = 0; a < len; ++a) {
    int f = base + a;
    int j = fcell[f];
    if (j == i) d = f;
    // source block: binary search of column j in row i
    int lo = b, hi = b + len - 1, e = -1;
    while (lo <= hi) {
      int mid = (lo + hi) >> 1;
      if (ci[mid] == j) { e = mid; break; }
      if (ci[mid] < j) lo = mid + 1; else hi = mid - 1;
    }
    const double* src = abar + (size_t)e * B2;
    double* dst = fv + (size_t)f * B2;
    for (int k = 0; k < B2; ++k) dst[k] = src[k];
    double* cs = fcs + (size_t)f * 2 * NB;
    for (int r = 0; r < NB; ++r) {
      cs[r] = src[r * NB + t];
      cs[NB + r] = src[r * NB + p];
    }
  }
  fdp[q] = d;
}

template <int NB>
__device__ bool gj_inverse_nb(const double* a_in, double* inv) {
  double a[NB * NB];
#pragma unroll
  for (int k = 0; k < NB * NB; ++k) a[k] = a_in[k];
#pragma unroll
  for (int i = 0; i < NB; ++i)
#pragma unroll
    for (int j = 0; j < NB; ++j) inv[i * NB + j] = (i == j) ? 1.0 : 0.0;
#pragma unroll
  for (int k = 0; k < NB; ++k) {
    double piv = a[k * NB + k];
    if (piv == 0.0 || !isfinite(piv)) return false;
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      a[k * NB + j] = a[k * NB + j] / piv;
      inv[k * NB + j] = inv[k * NB + j] / piv;
    }
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      if (i == k) continue;
      double f = a[i * NB + k];
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        a[i * NB + j] = a[i * NB + j] - f * a[k * NB + j];
        inv[i * NB + j] = inv[i * NB + j] - f * inv[k * NB + j];
      }
    }
  }
  return true;
}

// IKJ block ILU(0) for the rows of one colour. Lower neighbours of a row
// belong to earlier colours and are final; their U^{-1} diagonal blocks are
// in fdinv. diag_only: block Jacobi (invert the diagonal block only).
template <int NB>
__global__ void k_bilu_factor(int q0, int q1, const int* __restrict__ frp,
                              const int* __restrict__ fdp, const int* __restrict__ fpos,
                              double* __restrict__ fv, double* __restrict__ fdinv, int diag_only,
                              int* __restrict__ bad) {
  constexpr int B2 = NB * NB;
  int q = q0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= q1) return;
  const int b = frp[q], e = frp[q + 1], d = fdp[q];
  if (!diag_only) {
    for (int f = b; f < d; ++f) {
      const int kk = fpos[f];
      double L[B2];
      const double* W = fv + (size_t)f * B2;
      const double* Ui = fdinv + (size_t)kk * B2;
#pragma unroll
      for (int r = 0; r < NB; ++r)
#pragma unroll
        for (int c = 0; c < NB; ++c) {
          double s = 0.0;
#pragma unroll
          for (int k = 0; k < NB; ++k) s += W[r * NB + k] * Ui[k * NB + c];
          L[r * NB + c] = s;
        }
      double* Wf = fv + (size_t)f * B2;
#pragma unroll
      for (int k = 0; k < B2; ++k) Wf[k] = L[k];
      for (int g = fdp[kk] + 1; g < frp[kk + 1]; ++g) {
        const int j = fpos[g];
        int hit = -1;
        for (int h2 = b; h2 < e; ++h2)
          if (fpos[h2] == j) { hit = h2; break; }
        if (hit < 0) continue;
        double* Wq = fv + (size_t)hit * B2;
        const double* U = fv + (size_t)g * B2;
#pragma unroll
        for (int r = 0; r < NB; ++r)
#pragma unroll
          for (int c = 0; c < NB; ++c) {
            double s = 0.0;
#pragma unroll
            for (int k = 0; k < NB; ++k) s += L[r * NB + k] * U[k * NB + c];
            Wq[r * NB + c] -= s;
          }
      }
    }
  }
  double inv[B2];
  if (!gj_inverse_nb<NB>(fv + (size_t)d * B2, inv)) {
    atomicMin(bad, q);
    return;
  }
  double* out = fdinv + (size_t)q * B2;
#pragma unroll
  for (int k = 0; k < B2; ++k) out[k] = inv[k];
}

// ---- sweeps (NB lanes per row) -------------------------------------------
// MODE bit 1: subtract Abar[:, t] x_T; bit 2: subtract Abar[:, p] v_P
template <int NB, int MODE>
__global__ void k_bilu_fwd(int q0, int q1, const int* __restrict__ perm,
                           const int* __restrict__ frp, const int* __restrict__ fdp,
                           const int* __restrict__ fpos, const int* __restrict__ fcell,
                           const double* __restrict__ fv, const double* __restrict__ fcs,
                           const double* __restrict__ r, const double* __restrict__ xT,
                           const double* __restrict__ vP, double* __restrict__ w, int lower) {
  constexpr int RPW = 32 / NB;
  constexpr int B2 = NB * NB;
  const int lane = threadIdx.x & 31;
  const int sub = lane / NB, comp = lane - sub * NB;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long qq = q0 + warp * RPW + sub;
  if (sub >= RPW || qq >= q1) return;
  const int q = (int)qq;
  const int cell = perm[q];
  double acc = r[(size_t)cell * NB + comp];
  const int b = frp[q], e = frp[q + 1];
  if (MODE) {
    for (int f = b; f < e; ++f) {
      const int j = fcell[f];
      const double* cs = fcs + (size_t)f * 2 * NB;
      if (MODE & 1) acc -= cs[comp] * xT[j];
      if (MODE & 2) acc -= cs[NB + comp] * vP[j];
    }
  }
  if (lower) {
    const int d = fdp[q];
    for (int f = b; f < d; ++f) {
      const double* Lr = fv + (size_t)f * B2 + comp * NB;
      const double* wk = w + (size_t)fpos[f] * NB;
#pragma unroll
      for (int c = 0; c < NB; ++c) acc -= Lr[c] * wk[c];
    }
  }
  w[(size_t)q * NB + comp] = acc;
}

// backward sweep: x_q = U_qq^{-1} (w_q - sum_{upper} U_qj x_j); writes x_q
// back into w (read by earlier colours) and y = x + stage corrections
template <int NB, int MODE>
__global__ void k_bilu_bwd(int q0, int q1, const int* __restrict__ perm,
                           const int* __restrict__ frp, const int* __restrict__ fdp,
                           const int* __restrict__ fpos, const double* __restrict__ fv,
                           const double* __restrict__ fdinv, const double* __restrict__ xT,
                           const double* __restrict__ vP, int p, int t, double* __restrict__ w,
                           double* __restrict__ y, int upper) {
  constexpr int RPW = 32 / NB;
  constexpr int B2 = NB * NB;
  const int lane = threadIdx.x & 31;
  const int sub = lane / NB, comp = lane - sub * NB;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long qq = q0 + warp * RPW + sub;
  const bool active = sub < RPW && qq < q1;
  const int q = active ? (int)qq : 0;
  double tv = 0.0;
  if (active) {
    tv = w[(size_t)q * NB + comp];
    if (upper) {
      const int d = fdp[q], e = frp[q + 1];
      for (int g = d + 1; g < e; ++g) {
        const double* Ur = fv + (size_t)g * B2 + comp * NB;
        const double* xj = w + (size_t)fpos[g] * NB;
#pragma unroll
        for (int c = 0; c < NB; ++c) tv -= Ur[c] * xj[c];
      }
    }
  }
  const int base = sub * NB;
  const double* Ui = fdinv + (size_t)q * B2 + comp * NB;
  double x = 0.0;
#pragma unroll
  for (int c = 0; c < NB; ++c) {
    double tc = __shfl_sync(0xffffffffu, tv, (base + c) & 31);
    if (active) x += Ui[c] * tc;
  }
  if (!active) return;
  w[(size_t)q * NB + comp] = x;
  const int cell = perm[q];
  double out = x;
  if ((MODE & 1) && comp == t) out += xT[cell];
  if ((MODE & 2) && comp == p) out += vP[cell];
  y[(size_t)cell * NB + comp] = out;
}

template <int NB>
void bilu_setup_nb(Handle* h) {
  const int N = h->N;
  const int nnzb = h->nnzb;
  const bool bjac = h->opt.stage3 == MSS_BLOCK_JACOBI;
  h->colour.reset(h, N);
  h->perm.reset(h, N);
  h->iperm.reset(h, N);
  // ---- colouring (block Jacobi needs no order: a single colour)
  if (bjac) {
    fill_int(h, h->colour.p, 0, N);
    h->ncol = 1;
  } else {
    fill_int(h, h->colour.p, -1, N);
    DBuf<int> pick(h, N), left(h, 1), maxcol(h, 1);
    fill_int(h, maxcol.p, -1, 1);
    int remaining = N, rounds = 0;
    while (remaining > 0) {
      if (++rounds > N + 1) fail(MSS_ERR_CUDA, "colouring did not terminate");
      k_jp_pick<<<grid_for(N, 256), 256, 0, h->stream>>>(N, h->rp.p, h->ci.p, h->opt.seed,
                                                         h->colour.p, pick.p);
      MSS_LAUNCH_CK("k_jp_pick");
      fill_int(h, left.p, 0, 1);
      k_jp_commit<<<grid_for(N, 256), 256, 0, h->stream>>>(N, pick.p, h->colour.p, left.p,
                                                           maxcol.p);
      MSS_LAUNCH_CK("k_jp_commit");
      remaining = read_int(h, left.p);
    }
    h->ncol = read_int(h, maxcol.p) + 1;
  }
  // ---- colour-major positions
  h->cstart.assign(h->ncol + 1, 0);
  {
    DBuf<int> flag(h, N), rank(h, N + 1);
    int base = 0;
    for (int c = 0; c < h->ncol; ++c) {
      k_flag_colour<<<grid_for(N, 256), 256, 0, h->stream>>>(N, h->colour.p, c, flag.p);
      MSS_LAUNCH_CK("k_flag_colour");
      exclusive_scan(h, flag.p, rank.p, N);
      int cnt = read_int(h, rank.p + N);
      k_place_colour<<<grid_for(N, 256), 256, 0, h->stream>>>(N, h->colour.p, c, base, rank.p,
                                                              h->iperm.p, h->perm.p);
      MSS_LAUNCH_CK("k_place_colour");
      h->cstart[c] = base;
      base += cnt;
    }
    h->cstart[h->ncol] = base;
    if (base != N) fail(MSS_ERR_CUDA, "colour classes do not cover every cell");
  }
  // ---- factor pattern and values
  {
    DBuf<int> len(h, N);
    k_perm_rowlen<<<grid_for(N, 256), 256, 0, h->stream>>>(N, h->perm.p, h->rp.p, len.p);
    MSS_LAUNCH_CK("k_perm_rowlen");
    h->frp.reset(h, N + 1);
    exclusive_scan(h, len.p, h->frp.p, N);
  }
  h->fpos.reset(h, nnzb);
  h->fcell.reset(h, nnzb);
  h->fdp.reset(h, N);
  h->fv.reset(h, (size_t)nnzb * NB * NB);
  h->fcs.reset(h, (size_t)nnzb * 2 * NB);
  h->fdinv.reset(h, (size_t)N * NB * NB);
  k_fill_factor<NB><<<grid_for(N, 128), 128, 0, h->stream>>>(
      N, h->perm.p, h->iperm.p, h->rp.p, h->ci.p, h->abar.p, h->p, h->t, h->frp.p, h->fpos.p,
      h->fcell.p, h->fdp.p, h->fv.p, h->fcs.p);
  MSS_LAUNCH_CK("k_fill_factor");
  // ---- factorisation, colour by colour
  DBuf<int> bad(h, 1);
  fill_int(h, bad.p, 0x7fffffff, 1);
  for (int c = 0; c < h->ncol; ++c) {
    int q0 = h->cstart[c], q1 = h->cstart[c + 1];
    if (q1 <= q0) continue;
    k_bilu_factor<NB><<<grid_for(q1 - q0, 128), 128, 0, h->stream>>>(
        q0, q1, h->frp.p, h->fdp.p, h->fpos.p, h->fv.p, h->fdinv.p, bjac ? 1 : 0, bad.p);
    MSS_LAUNCH_CK("k_bilu_factor");
  }
  int badq = read_int(h, bad.p);
  if (badq != 0x7fffffff)
    fail(MSS_ERR_SINGULAR_BLOCK, "block ILU(0): zero pivot in the diagonal block at position " +
                                     std::to_string(badq));
}

template <int NB, int MODE>
void sweeps(Handle* h, const double* r, const double* xT, const double* vP, double* y) {
  constexpr int RPW = 32 / NB;
  const bool bjac = h->opt.stage3 == MSS_BLOCK_JACOBI;
  const int T = 256;
  for (int c = 0; c < h->ncol; ++c) {
    int q0 = h->cstart[c], q1 = h->cstart[c + 1];
    if (q1 <= q0) continue;
    long long warps = (q1 - q0 + RPW - 1) / RPW;
    TraceScope ts(h, TR_BILU_FWD);
    k_bilu_fwd<NB, MODE><<<grid_for(warps * 32, T), T, 0, h->stream>>>(
        q0, q1, h->perm.p, h->frp.p, h->fdp.p, h->fpos.p, h->fcell.p, h->fv.p, h->fcs.p, r, xT, vP,
        h->w.p, bjac ? 0 : 1);
    MSS_LAUNCH_CK("k_bilu_fwd");
  }
  for (int c = h->ncol - 1; c >= 0; --c) {
    int q0 = h->cstart[c], q1 = h->cstart[c + 1];
    if (q1 <= q0) continue;
    long long warps = (q1 - q0 + RPW - 1) / RPW;
    TraceScope ts(h, TR_BILU_BWD);
    k_bilu_bwd<NB, MODE><<<grid_for(warps * 32, T), T, 0, h->stream>>>(
        q0, q1, h->perm.p, h->frp.p, h->fdp.p, h->fpos.p, h->fv.p, h->fdinv.p, xT, vP, h->p, h->t,
        h->w.p, y, bjac ? 0 : 1);
    MSS_LAUNCH_CK("k_bilu_bwd");
  }
}

template <int NB>
void last_stage_nb(Handle* h, const double* r, const double* xT, const double* vP, double* y) {
  int mode = (xT ? 1 : 0) | (vP ? 2 : 0);
  switch (mode) {
    case 0: sweeps<NB, 0>(h, r, xT, vP, y); break;
    case 1: sweeps<NB, 1>(h, r, xT, vP, y); break;
    case 2: sweeps<NB, 2>(h, r, xT, vP, y); break;
    default: sweeps<NB, 3>(h, r, xT, vP, y); break;
  }
}

}  // namespace

void bilu_setup(Handle* h) {
  TraceScope ts(h, TR_SETUP_BILU);
  MSS_NB_DISPATCH(h->nb, bilu_setup_nb<NB>(h));
}

void last_stage_apply(Handle* h, const double* r, const double* xT, const double* vP, double* y) {
  MSS_NB_DISPATCH(h->nb, last_stage_nb<NB>(h, r, xT, vP, y));
}

}  // namespace mss
