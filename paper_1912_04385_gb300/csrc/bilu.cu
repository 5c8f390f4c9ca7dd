// bilu.cu -- last stage of the multi-stage preconditioner: block ILU(0) of
// the scaled matrix (Eq. CPTR3M3; the CPR second stage), or block Jacobi,
// plus the fused stage arithmetic around it.
//
// Ordering. Cells are grouped into strips of `ilu_strip` consecutive cells
// (or single cells for the point-multicolour order) and the strips are
// coloured by Jones-Plassmann with SplitMix64 priorities. Cells are then
// renumbered colour-major with ascending cell index inside a colour, so a
// colour is a contiguous range of positions made of whole strips, and each
// strip keeps its natural order. Strips of one colour are never coupled, so
// they are factored and swept in parallel; inside a strip the rows are
// processed in order. Natural order inside strips keeps the upwind chains of
// the advection operators that a point colouring cuts at every cell.
//
// Apply (Algorithm 2, fused): the forward sweep forms
//   u = r - Abar[:,t] x_T - Abar[:,p] v_P
// on the fly from per-block column slices, and the backward sweep writes
//   y = x + v + M3 u
// directly. A strip is swept by NB lanes (lane c owns component c), so a
// row's nb x nb blocks are read as contiguous rows by adjacent lanes; the
// factorisation uses the same layout (lane r holds row r of each block).
#include <algorithm>

#include "common.cuh"
#include "bilu_sweeps.cuh"

namespace mss {
namespace {

using namespace dev;

constexpr uint64_t KEY_CELL = 0xFFFFULL << 32;    // priorities of single cells
constexpr uint64_t KEY_STRIP = 0xFFFEULL << 32;   // priorities of strips

// ---- Jones-Plassmann colouring of strips of S consecutive cells -----------
// (S = 1 with the cell key is the point-multicolour order). One warp per
// strip, the lanes over the strip's cells: an uncoloured strip whose
// priority beats every uncoloured neighbour strip picks the smallest colour
// no neighbour strip has.
__global__ void k_jp_pick(int ns, int S, int n, const int* __restrict__ rp,
                          const int* __restrict__ ci, uint64_t seed, uint64_t key,
                          const int* __restrict__ scol, int* __restrict__ pick,
                          int* __restrict__ left) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *left = 0;   // the round's count (k_jp_commit)
  const int lane = threadIdx.x & 31;
  const long long a = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (a >= ns) return;                     // uniform per warp
  int chosen = -1;
  if (scol[a] < 0) {
    const int lo = (int)a * S, hi = min(lo + S, n);
    const uint64_t pa = splitmix64(seed, key | (uint64_t)(unsigned)a);
    bool best = true;
    for (int i = lo + lane; i < hi && best; i += 32)
      for (int k = rp[i]; k < rp[i + 1] && best; ++k) {
        const int b = ci[k] / S;
        if (b == a || scol[b] >= 0) continue;
        const uint64_t pb = splitmix64(seed, key | (uint64_t)(unsigned)b);
        if (pb > pa || (pb == pa && b > a)) best = false;
      }
    if (__all_sync(0xffffffffu, best)) {
      // colours of the neighbour strips below 64 as a bit set, then the
      // smallest free one (a search past 64 when all of those are taken)
      unsigned long long used = 0;
      for (int i = lo + lane; i < hi; i += 32)
        for (int k = rp[i]; k < rp[i + 1]; ++k) {
          const int b = ci[k] / S;
          const int cb = b != a ? scol[b] : -1;
          if (cb >= 0 && cb < 64) used |= 1ULL << cb;
        }
      for (int o = 16; o > 0; o >>= 1) used |= __shfl_xor_sync(0xffffffffu, used, o);
      if (~used != 0ULL) {
        chosen = __ffsll((long long)~used) - 1;
      } else {
        for (int c = 64;; ++c) {
          bool hit = false;
          for (int i = lo + lane; i < hi && !hit; i += 32)
            for (int k = rp[i]; k < rp[i + 1]; ++k) {
              const int b = ci[k] / S;
              if (b != a && scol[b] == c) { hit = true; break; }
            }
          if (!__any_sync(0xffffffffu, hit)) { chosen = c; break; }
        }
      }
    }
  }
  if (lane == 0) pick[a] = chosen;
}

__global__ void k_jp_commit(int ns, const int* __restrict__ pick, int* __restrict__ scol,
                            int* __restrict__ left, int* __restrict__ maxcol) {
  int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= ns) return;
  if (pick[a] >= 0) {
    scol[a] = pick[a];
    atomicMax(maxcol, pick[a]);
  } else if (scol[a] < 0) {
    atomicAdd(left, 1);
  }
}

// First-fit colouring of strips needs, per strip, its distinct lower-index
// adjacent strips; up to kStripNbrs of them are listed (cnt = -1: more)
constexpr int kStripNbrs = 32;

__global__ void k_strip_lower(int ns, int S, int n, const int* __restrict__ rp,
                              const int* __restrict__ ci, int* __restrict__ nbr,
                              int* __restrict__ cnt) {
  int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= ns) return;
  int* out = nbr + (size_t)a * kStripNbrs;
  int m = 0;
  const int lo = a * S, hi = min(lo + S, n);
  for (int i = lo; i < hi && m >= 0; ++i)
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
      const int b = ci[k] / S;
      if (b >= a) continue;
      bool seen = false;
      for (int t = 0; t < m && !seen; ++t) seen = out[t] == b;
      if (seen) continue;
      if (m == kStripNbrs) {
        m = -1;
        break;
      }
      out[m++] = b;
    }
  cnt[a] = m;
}

__global__ void k_cell_colour(int n, int S, const int* __restrict__ scol, int* __restrict__ col) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) col[i] = scol[i / S];
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

__global__ void k_place_strips(int ns, int S, int n, const int* __restrict__ scol, int c,
                               int base, const int* __restrict__ rank,
                               const int* __restrict__ iperm, int* __restrict__ st_first,
                               int* __restrict__ st_len) {
  int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= ns || scol[a] != c) return;
  int k = base + rank[a];
  st_first[k] = iperm[a * S];
  st_len[k] = min(S, n - a * S);
}

__global__ void k_perm_rowlen(int n, const int* __restrict__ perm, const int* __restrict__ rp,
                              int* __restrict__ len) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) len[q] = rp[perm[q] + 1] - rp[perm[q]];
}

// position range [qlo, qhi) of the strip that holds each position
__global__ void k_strip_ranges(int ns, const int* __restrict__ st_first,
                               const int* __restrict__ st_len, int* __restrict__ qlo,
                               int* __restrict__ qhi) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= ns) return;
  const int f = st_first[k], e = f + st_len[k];
  for (int q = f; q < e; ++q) {
    qlo[q] = f;
    qhi[q] = e;
  }
}

// factor pattern of row q (cell perm[q]) sorted by column position, and the
// split of the row into other-strip lower | in-strip lower | diagonal |
// in-strip upper | other-strip upper entries
__global__ void k_factor_pattern(int n, const int* __restrict__ perm,
                                 const int* __restrict__ iperm, const int* __restrict__ rp,
                                 const int* __restrict__ ci, const int* __restrict__ frp,
                                 const int* __restrict__ qlo, const int* __restrict__ qhi,
                                 int* __restrict__ fpos, int* __restrict__ fcell,
                                 int* __restrict__ fsrc, int* __restrict__ fdp,
                                 int* __restrict__ fslo, int* __restrict__ fshi) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const int i = perm[q];
  const int b = rp[i], len = rp[i + 1] - b, base = frp[q];
  int d = -1;
  for (int a = 0; a < len; ++a) {
    const int e = b + a;
    const int pc = iperm[ci[e]];
    int k = a - 1;
    while (k >= 0 && fpos[base + k] > pc) {
      fpos[base + k + 1] = fpos[base + k];
      fcell[base + k + 1] = fcell[base + k];
      fsrc[base + k + 1] = fsrc[base + k];
      --k;
    }
    fpos[base + k + 1] = pc;
    fcell[base + k + 1] = ci[e];
    fsrc[base + k + 1] = e;
  }
  const int lo = qlo[q], hi = qhi[q];
  int slo = base + len, shi = base;
  for (int a = 0; a < len; ++a) {
    const int pc = fpos[base + a];
    if (pc == q) d = base + a;
    if (pc >= lo && pc < q && base + a < slo) slo = base + a;
    if (pc > q && pc < hi) shi = base + a + 1;
  }
  fdp[q] = d;
  fslo[q] = slo < d ? slo : d;
  fshi[q] = shi > d + 1 ? shi : d + 1;
}

// factor blocks (copies of Abar) and column slices [Abar[:, t] | Abar[:, p]]
template <int NB>
__global__ void k_factor_values(long long nnzb, const int* __restrict__ fsrc,
                                const double* __restrict__ abar, int p, int t,
                                double* __restrict__ fv, double* __restrict__ fcs) {
  constexpr int B2 = NB * NB;
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long stride = (long long)gridDim.x * blockDim.x;
  for (; idx < nnzb * B2; idx += stride) {
    long long f = idx / B2;
    int k = (int)(idx - f * B2);
    fv[idx] = abar[(size_t)fsrc[f] * B2 + k];
  }
  idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (; idx < nnzb * 2 * NB; idx += stride) {
    long long f = idx / (2 * NB);
    int k = (int)(idx - f * 2 * NB);
    int r = k < NB ? k : k - NB;
    int col = k < NB ? t : p;
    fcs[idx] = abar[(size_t)fsrc[f] * B2 + r * NB + col];
  }
}

// Row r of an nb x nb row-major block (16-byte loads and stores when the rows
// are whole 16-byte units: the blocks start 256-byte aligned).
template <int NB>
__device__ __forceinline__ void ld_row(const double* p, double (&x)[NB]) {
  if constexpr (NB % 2 == 0) {
    const double2* p2 = reinterpret_cast<const double2*>(p);
#pragma unroll
    for (int i = 0; i < NB / 2; ++i) {
      const double2 v = p2[i];
      x[2 * i] = v.x;
      x[2 * i + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < NB; ++i) x[i] = p[i];
  }
}
template <int NB>
__device__ __forceinline__ void st_row(double* p, const double (&x)[NB]) {
  if constexpr (NB % 2 == 0) {
    double2* p2 = reinterpret_cast<double2*>(p);
#pragma unroll
    for (int i = 0; i < NB / 2; ++i) p2[i] = make_double2(x[2 * i], x[2 * i + 1]);
  } else {
#pragma unroll
    for (int i = 0; i < NB; ++i) p[i] = x[i];
  }
}

// Block ILU(0) of one colour with a whole warp per strip (the operations of
// k_bilu_factor below, in the same order): the block products and the
// Gauss-Jordan elimination on [U_qq | I] are spread over the 32 lanes. Fewer
// instructions per row than NB lanes per strip, so it is the faster form for
// colours too small to fill the SMs, where the row-by-row latency of each
// strip decides the time.
// warps per CTA of the warp-per-strip factorisation: its shared work blocks
// (3 nb x nb per warp) stay under the 48 KB static limit
template <int NB>
constexpr int factor_warps() { return NB <= 12 ? 8 : 4; }

template <int NB>
__global__ void __launch_bounds__(32 * factor_warps<NB>())
k_bilu_factor_warp(int s0, int s1, const int* __restrict__ st_first, const int* __restrict__ st_len,
              const int* __restrict__ frp, const int* __restrict__ fdp,
              const int* __restrict__ fpos, double* __restrict__ fv,
              double* __restrict__ fdinv, int diag_only, int* __restrict__ bad) {
  constexpr int B2 = NB * NB;
  constexpr int W2 = 2 * NB;
  __shared__ double smem[factor_warps<NB>()][3 * B2];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const long long k = s0 + (((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (k >= s1) return;                       // uniform per warp
  double* L = smem[wib];
  double* aug = L + B2;                      // NB x 2NB augmented matrix
  const int first = st_first[k], len = st_len[k];
  for (int q = first; q < first + len; ++q) {
    const int b = frp[q], e = frp[q + 1], d = fdp[q];
    if (!diag_only) {
      for (int f = b; f < d; ++f) {
        const int kk = fpos[f];
        const double* W = fv + (size_t)f * B2;
        const double* Ui = fdinv + (size_t)kk * B2;
        for (int idx = lane; idx < B2; idx += 32) {
          const int r = idx / NB, c = idx - r * NB;
          double s = 0.0;
#pragma unroll
          for (int m = 0; m < NB; ++m) s += W[r * NB + m] * Ui[m * NB + c];
          L[idx] = s;
        }
        __syncwarp();
        for (int idx = lane; idx < B2; idx += 32) fv[(size_t)f * B2 + idx] = L[idx];
        for (int g = fdp[kk] + 1; g < frp[kk + 1]; ++g) {
          const int j = fpos[g];
          int hit = -1;
          for (int h2 = b; h2 < e; ++h2)
            if (fpos[h2] == j) { hit = h2; break; }
          if (hit < 0) continue;
          double* Wq = fv + (size_t)hit * B2;
          const double* U = fv + (size_t)g * B2;
          for (int idx = lane; idx < B2; idx += 32) {
            const int r = idx / NB, c = idx - r * NB;
            double s = 0.0;
#pragma unroll
            for (int m = 0; m < NB; ++m) s += L[r * NB + m] * U[m * NB + c];
            Wq[idx] -= s;
          }
        }
        __syncwarp();
      }
    }
    // Gauss-Jordan inverse of the pivot block, no pivoting
    for (int idx = lane; idx < NB * W2; idx += 32) {
      const int r = idx / W2, c = idx - r * W2;
      aug[idx] = c < NB ? fv[(size_t)d * B2 + r * NB + c] : (c - NB == r ? 1.0 : 0.0);
    }
    __syncwarp();
    bool ok = true;
    for (int ks = 0; ks < NB; ++ks) {
      const double piv = aug[ks * W2 + ks];
      if (piv == 0.0 || !isfinite(piv)) { ok = false; break; }   // same value in all lanes
      const double rpiv = 1.0 / piv;          // one division per pivot
      __syncwarp();
      if (lane < W2) aug[ks * W2 + lane] = aug[ks * W2 + lane] * rpiv;
      __syncwarp();
      double fr[(NB * W2 + 31) / 32];
      int tt = 0;
      for (int idx = lane; idx < NB * W2; idx += 32, ++tt) fr[tt] = aug[(idx / W2) * W2 + ks];
      __syncwarp();
      tt = 0;
      for (int idx = lane; idx < NB * W2; idx += 32, ++tt) {
        const int i = idx / W2, j = idx - i * W2;
        if (i != ks) aug[idx] = aug[idx] - fr[tt] * aug[ks * W2 + j];
      }
      __syncwarp();
    }
    if (!ok) {
      if (lane == 0) atomicMin(bad, q);
      return;
    }
    for (int idx = lane; idx < B2; idx += 32) {
      const int r = idx / NB, c = idx - r * NB;
      fdinv[(size_t)q * B2 + idx] = aug[r * W2 + NB + c];
    }
    __syncwarp();
  }
}


// IKJ block ILU(0) of one colour's strips, each strip's rows in order. A strip
// is owned by NB lanes (32 / NB strips per warp) and lane r holds row r of
// every block of the current row, so each FP64 instruction does useful work
// on almost every lane. Lower neighbours belong to earlier colours or to
// earlier rows of the same strip and are final; their U^{-1} diagonal blocks
// are in fdinv. For each lower entry k of row q:
//   L_qk = A_qk U_kk^{-1},  A_qj -= L_qk U_kj  for every j > k in both rows,
// then U_qq (kept in registers) is inverted by Gauss-Jordan without pivoting,
// in place, the pivot row passed between the NB lanes by shuffles (the same
// operations, in the same order, as elimination on [U_qq | I]). A zero or
// non-finite pivot stops the strip and records the smallest such position
// in *bad. diag_only: block Jacobi (no lower entries are used).
constexpr int kRowCols = 8;       // columns of the current row held in registers
// A colour with fewer than kSmallColour x (32 / NB) strips per SM is factored
// with a whole warp per strip (k_bilu_factor_warp).
constexpr int kSmallColour = 4;

template <int NB>
__global__ void __launch_bounds__(32, 16)
k_bilu_factor(int s0, int s1, const int* __restrict__ st_first, const int* __restrict__ st_len,
              const int* __restrict__ frp, const int* __restrict__ fdp,
              const int* __restrict__ fpos, double* __restrict__ fv,
              double* __restrict__ fdinv, int diag_only, int* __restrict__ bad) {
  constexpr int B2 = NB * NB;
  constexpr int G = 32 / NB;                 // strips per warp
  const int lane = threadIdx.x & 31;
  const int sub = lane / NB, r = lane - sub * NB, base = sub * NB;
  const long long k = s0 + ((long long)blockIdx.x * blockDim.x + threadIdx.x) / 32 * G + sub;
  const bool own = sub < G && k < s1;
  const int first = own ? st_first[k] : 0;
  const int len = own ? st_len[k] : 0;
  const int maxlen = warp_max(len);
  bool alive = own;
  for (int t = 0; t < maxlen; ++t) {
    const bool act = alive && t < len;
    const int q = first + t;
    int b = 0, d = 0, e = 0;
    double dq[NB];
#pragma unroll
    for (int c = 0; c < NB; ++c) dq[c] = 0.0;
    if (act) {
      b = frp[q];
      e = frp[q + 1];
      d = fdp[q];
      ld_row<NB>(fv + (size_t)d * B2 + r * NB, dq);
    }
    int cols[kRowCols];                    // row q's first columns, -1 past its end
#pragma unroll
    for (int i = 0; i < kRowCols; ++i) cols[i] = b + i < e ? fpos[b + i] : -1;
    if (!diag_only) {
      for (int f = b; f < d; ++f) {        // no lane exchange inside: may diverge
        const int kk = fpos[f];
        const double* Ui = fdinv + (size_t)kk * B2;
        double w[NB], l[NB], u[NB];
        ld_row<NB>(fv + (size_t)f * B2 + r * NB, w);
#pragma unroll
        for (int c = 0; c < NB; ++c) l[c] = 0.0;
#pragma unroll
        for (int m = 0; m < NB; ++m) {
          ld_row<NB>(Ui + m * NB, u);
#pragma unroll
          for (int c = 0; c < NB; ++c) l[c] += w[m] * u[c];
        }
        st_row<NB>(fv + (size_t)f * B2 + r * NB, l);
        const int g1 = frp[kk + 1];
        for (int g = fdp[kk] + 1; g < g1; ++g) {
          const int j = fpos[g];
          int hit = -1;
#pragma unroll
          for (int i = 0; i < kRowCols; ++i)
            if (cols[i] == j) hit = b + i;
          if (hit < 0)
            for (int h2 = b + kRowCols; h2 < e; ++h2)
              if (fpos[h2] == j) {
                hit = h2;
                break;
              }
          if (hit < 0) continue;
          const double* U = fv + (size_t)g * B2;
          double sacc[NB];
#pragma unroll
          for (int c = 0; c < NB; ++c) sacc[c] = 0.0;
#pragma unroll
          for (int m = 0; m < NB; ++m) {
            ld_row<NB>(U + m * NB, u);
#pragma unroll
            for (int c = 0; c < NB; ++c) sacc[c] += l[m] * u[c];
          }
          if (hit == d) {
#pragma unroll
            for (int c = 0; c < NB; ++c) dq[c] -= sacc[c];
          } else {
            double* X = fv + (size_t)hit * B2 + r * NB;
            double x[NB];
            ld_row<NB>(X, x);
#pragma unroll
            for (int c = 0; c < NB; ++c) x[c] -= sacc[c];
            st_row<NB>(X, x);
          }
        }
      }
    }
    if (act) st_row<NB>(fv + (size_t)d * B2 + r * NB, dq);   // U_qq
    // Gauss-Jordan, in place: after pivot ks, columns < ks of dq hold the
    // inverse's columns and columns > ks the reduced matrix.
    bool ok = true;
#pragma unroll
    for (int ks = 0; ks < NB; ++ks) {
      double pn[NB];
#pragma unroll
      for (int j = 0; j < NB; ++j) pn[j] = __shfl_sync(0xffffffffu, dq[j], (base + ks) & 31);
      const double piv = pn[ks];
      ok = ok && piv != 0.0 && isfinite(piv);
      const double rpiv = 1.0 / piv;
#pragma unroll
      for (int j = 0; j < NB; ++j) pn[j] = j == ks ? rpiv : pn[j] * rpiv;
      const double fr = dq[ks];
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        const double x = j == ks ? 0.0 : dq[j];
        dq[j] = r == ks ? pn[j] : x - fr * pn[j];
      }
    }
    if (act) {
      if (ok) {
        st_row<NB>(fdinv + (size_t)q * B2 + r * NB, dq);
      } else {
        if (r == 0) atomicMin(bad, q);
        alive = false;
      }
    }
    __syncwarp();     // row q's blocks, written lane by lane, are read whole by row q + 1
  }
}

// ---- sweeps ----------------------------------------------------------------
// The kernels of the sweeps run the bodies of bilu_sweeps.cuh (the parallel
// and chain passes of each colour) with the warp index of this launch.
template <int NB, int MODE, class V, class C>
__global__ void k_bilu_fwd_par(int q0, int q1, const int* __restrict__ perm,
                               const int* __restrict__ frp, const int* __restrict__ fslo,
                               const int* __restrict__ fpos, const int* __restrict__ fcell,
                               const V* __restrict__ fv, const C* __restrict__ fcs,
                               const double* __restrict__ r, const C* __restrict__ xT,
                               const C* __restrict__ vP, C* __restrict__ w, int lower,
                               int wait_first) {
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  fwd_par<NB, MODE, V, C>(warp, q0, q1, perm, frp, fslo, fpos, fcell, fv, fcs, r, xT, vP, w,
                          lower, wait_first);
}

template <int NB, class V, class C>
__global__ void k_bilu_fwd_chain(int s0, int s1, const int* __restrict__ st_first,
                                 const int* __restrict__ st_len, const int* __restrict__ fslo,
                                 const int* __restrict__ fdp, const int* __restrict__ fpos,
                                 const V* __restrict__ fv, const V* __restrict__ cL,
                                 const int* __restrict__ cflag, C* __restrict__ w) {
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  fwd_chain<NB, V, C>(warp, s0, s1, st_first, st_len, fslo, fdp, fpos, fv, cL, cflag, w);
}

// After the factorisation, every in-strip upper block U_qj becomes
// G_qj = U_qq^{-1} U_qj, so that the backward chain reads
//   x_q = s_q - sum_{in-strip upper} G_qj x_j,  s_q = U_qq^{-1} t_q,
// with s_q formed in the parallel pass (the same operator, written as a
// product of the already inverted pivot block).
template <int NB>
__global__ void k_strip_upper_scale(int n, const int* __restrict__ fdp,
                                    const int* __restrict__ fshi,
                                    const double* __restrict__ fdinv, double* __restrict__ fv) {
  // NB lanes per row q (32 / NB rows per warp), lane r forms row r of
  // U_qq^{-1} U_qj with the sums in ascending m; a block is read by all lanes
  // of its row before any of them writes
  constexpr int B2 = NB * NB;
  constexpr int RPW = 32 / NB;
  const int lane = threadIdx.x & 31;
  const int sub = lane / NB, r = lane - sub * NB;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long qq = warp * RPW + sub;
  const bool active = sub < RPW && qq < n;
  const int q = active ? (int)qq : 0;
  int g0 = 0, cnt = 0;
  double ui[NB];
#pragma unroll
  for (int m = 0; m < NB; ++m) ui[m] = 0.0;
  if (active) {
    g0 = fdp[q] + 1;
    cnt = fshi[q] - g0;
#pragma unroll
    for (int m = 0; m < NB; ++m) ui[m] = fdinv[(size_t)q * B2 + r * NB + m];
  }
  const int maxc = warp_max(cnt);
  for (int it = 0; it < maxc; ++it) {
    const bool on = it < cnt;
    double out[NB];
    if (on) {
      const double* U = fv + (size_t)(g0 + it) * B2;
#pragma unroll
      for (int c = 0; c < NB; ++c) {
        double s = 0.0;
#pragma unroll
        for (int m = 0; m < NB; ++m) s += ui[m] * U[m * NB + c];
        out[c] = s;
      }
    }
    __syncwarp();
    if (on) {
#pragma unroll
      for (int c = 0; c < NB; ++c) fv[(size_t)(g0 + it) * B2 + r * NB + c] = out[c];
    }
    __syncwarp();
  }
}

// Dense per-position copies of the chain couplings: cL[q] = L_{q,q-1} when
// the only in-strip lower neighbour of q is q-1, cG[q] = G_{q,q+1} when the
// only in-strip upper neighbour is q+1, zero blocks when there is none; any
// other in-strip coupling sets cflag (bit 0 lower, bit 1 upper) and is then
// taken from the factor rows instead.
template <int NB>
__global__ void k_chain_blocks(long long N, const int* __restrict__ fslo,
                               const int* __restrict__ fdp, const int* __restrict__ fshi,
                               const int* __restrict__ fpos, const double* __restrict__ fv,
                               double* __restrict__ cL, double* __restrict__ cG,
                               int* __restrict__ cflag) {
  constexpr int B2 = NB * NB;
  long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= N * B2) return;
  const int q = (int)(tid / B2);
  const int k = (int)(tid - (long long)q * B2);
  const int lo = fslo[q], d = fdp[q], hi = fshi[q];
  const bool one_lo = d - lo == 1 && fpos[lo] == q - 1;
  const bool one_hi = hi - d == 2 && fpos[d + 1] == q + 1;
  cL[tid] = one_lo ? fv[(size_t)lo * B2 + k] : 0.0;
  cG[tid] = one_hi ? fv[(size_t)(d + 1) * B2 + k] : 0.0;
  if (k == 0) cflag[q] = ((d > lo && !one_lo) ? 1 : 0) | ((hi > d + 1 && !one_hi) ? 2 : 0);
}

template <int NB, class V, class C>
__global__ void k_bilu_bwd_par(int q0, int q1, const int* __restrict__ frp,
                               const int* __restrict__ fshi, const int* __restrict__ fpos,
                               const V* __restrict__ fv, const V* __restrict__ fdinv,
                               C* __restrict__ w) {
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  bwd_par<NB, V, C>(warp, q0, q1, frp, fshi, fpos, fv, fdinv, w);
}

template <int NB, class V, class C>
__global__ void k_bilu_bwd_chain(int s0, int s1, const int* __restrict__ st_first,
                                 const int* __restrict__ st_len, const int* __restrict__ fdp,
                                 const int* __restrict__ fshi, const int* __restrict__ fpos,
                                 const V* __restrict__ fv, const V* __restrict__ fdinv,
                                 const V* __restrict__ cG, const int* __restrict__ cflag,
                                 C* __restrict__ w, int upper, const int* __restrict__ perm,
                                 const C* __restrict__ xT, const C* __restrict__ vP, int p,
                                 int t, double* __restrict__ y) {
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  bwd_chain<NB, V, C>(warp, s0, s1, st_first, st_len, fdp, fshi, fpos, fv, fdinv, cG, cflag, w,
                      upper, perm, xT, vP, p, t, y);
}

template <int NB>
void bilu_setup_nb(Handle* h) {
  const int N = h->N;
  const int nnzb = h->nnzb;
  const bool bjac = h->opt.stage3 == MSS_BLOCK_JACOBI;
  const bool strips = !bjac && (h->opt.ilu_order == MSS_STRIPS || h->opt.ilu_order == MSS_STRIPS_JP);
  const int S = strips ? h->opt.ilu_strip : 1;
  const int ns = (N + S - 1) / S;
  DBuf<int> scol(h, ns);
  h->colour.reset(h, N);
  h->perm.reset(h, N);
  h->iperm.reset(h, N);
  // ---- colouring of strips (block Jacobi needs no order: one colour)
  if (bjac) {
    fill_int(h, scol.p, 0, ns);
    h->ncol = 1;
  } else if (strips && h->opt.ilu_order == MSS_STRIPS) {
    // first-fit in strip order: each strip takes the smallest colour none of
    // its lower-index adjacent strips has (two colours on a structured
    // grid). The device lists the neighbours; the host walks the strips.
    DBuf<int> nbr(h, (size_t)ns * kStripNbrs), cnt(h, ns);
    k_strip_lower<<<grid_for(ns, 128), 128, 0, h->stream>>>(ns, S, N, h->rp.p, h->ci.p, nbr.p,
                                                            cnt.p);
    MSS_LAUNCH_CK("k_strip_lower");
    std::vector<int> hn((size_t)ns * kStripNbrs), hc(ns), sc(ns);
    MSS_CK(cudaMemcpyAsync(hn.data(), nbr.p, sizeof(int) * hn.size(), cudaMemcpyDeviceToHost,
                           h->stream));
    MSS_CK(cudaMemcpyAsync(hc.data(), cnt.p, sizeof(int) * hc.size(), cudaMemcpyDeviceToHost,
                           h->stream));
    MSS_CK(cudaStreamSynchronize(h->stream));
    std::vector<int> hrp, hci;               // the cell pattern, only for long lists
    std::vector<unsigned char> used;
    int ncol = 0;
    for (int a = 0; a < ns; ++a) {
      used.assign((size_t)ncol + 1, 0);
      if (hc[a] >= 0) {
        for (int t = 0; t < hc[a]; ++t) used[sc[hn[(size_t)a * kStripNbrs + t]]] = 1;
      } else {
        if (hrp.empty()) {
          hrp.resize((size_t)N + 1);
          hci.resize((size_t)nnzb);
          MSS_CK(cudaMemcpy(hrp.data(), h->rp.p, sizeof(int) * hrp.size(),
                            cudaMemcpyDeviceToHost));
          MSS_CK(cudaMemcpy(hci.data(), h->ci.p, sizeof(int) * hci.size(),
                            cudaMemcpyDeviceToHost));
        }
        const int lo = a * S, hi = std::min(lo + S, N);
        for (int i = lo; i < hi; ++i)
          for (int k = hrp[i]; k < hrp[i + 1]; ++k) {
            const int b = hci[k] / S;
            if (b < a) used[sc[b]] = 1;
          }
      }
      int c = 0;
      while (c <= ncol && used[c]) ++c;
      sc[a] = c;
      if (c + 1 > ncol) ncol = c + 1;
    }
    MSS_CK(cudaMemcpyAsync(scol.p, sc.data(), sizeof(int) * ns, cudaMemcpyHostToDevice,
                           h->stream));
    MSS_CK(cudaStreamSynchronize(h->stream));   // sc lives on this frame
    h->ncol = ncol;
  } else {
    fill_int(h, scol.p, -1, ns);
    DBuf<int> pick(h, ns), left(h, 1), maxcol(h, 1);
    fill_int(h, maxcol.p, -1, 1);
    const uint64_t key = strips ? KEY_STRIP : KEY_CELL;
    int remaining = ns, rounds = 0;
    while (remaining > 0) {
      // three rounds per read-back: once every strip is coloured a round
      // picks nothing, so the colouring is the round-by-round one
      for (int r = 0; r < 3; ++r) {
        if (++rounds > ns + 3) fail(MSS_ERR_CUDA, "colouring did not terminate");
        k_jp_pick<<<grid_for((long long)ns * 32, 128), 128, 0, h->stream>>>(
            ns, S, N, h->rp.p, h->ci.p, h->opt.seed, key, scol.p, pick.p, left.p);
        MSS_LAUNCH_CK("k_jp_pick");
        k_jp_commit<<<grid_for(ns, 256), 256, 0, h->stream>>>(ns, pick.p, scol.p, left.p,
                                                              maxcol.p);
        MSS_LAUNCH_CK("k_jp_commit");
      }
      remaining = read_int(h, left.p);
    }
    h->ncol = read_int(h, maxcol.p) + 1;
  }
  k_cell_colour<<<grid_for(N, 256), 256, 0, h->stream>>>(N, S, scol.p, h->colour.p);
  MSS_LAUNCH_CK("k_cell_colour");
  // ---- colour-major positions and the strip list
  h->cstart.assign(h->ncol + 1, 0);
  h->sc_start.assign(h->ncol + 1, 0);
  h->st_first.reset(h, ns);
  h->st_len.reset(h, ns);
  {
    DBuf<int> flag(h, std::max(N, ns)), rank(h, std::max(N, ns) + 1);
    int base = 0, sbase = 0;
    for (int c = 0; c < h->ncol; ++c) {
      k_flag_colour<<<grid_for(N, 256), 256, 0, h->stream>>>(N, h->colour.p, c, flag.p);
      MSS_LAUNCH_CK("k_flag_colour");
      exclusive_scan(h, flag.p, rank.p, N);
      const int cnt = read_int(h, rank.p + N);
      k_place_colour<<<grid_for(N, 256), 256, 0, h->stream>>>(N, h->colour.p, c, base, rank.p,
                                                              h->iperm.p, h->perm.p);
      MSS_LAUNCH_CK("k_place_colour");
      h->cstart[c] = base;
      base += cnt;
      k_flag_colour<<<grid_for(ns, 256), 256, 0, h->stream>>>(ns, scol.p, c, flag.p);
      MSS_LAUNCH_CK("k_flag_colour");
      exclusive_scan(h, flag.p, rank.p, ns);
      const int scnt = read_int(h, rank.p + ns);
      k_place_strips<<<grid_for(ns, 256), 256, 0, h->stream>>>(ns, S, N, scol.p, c, sbase,
                                                               rank.p, h->iperm.p,
                                                               h->st_first.p, h->st_len.p);
      MSS_LAUNCH_CK("k_place_strips");
      h->sc_start[c] = sbase;
      sbase += scnt;
    }
    h->cstart[h->ncol] = base;
    h->sc_start[h->ncol] = sbase;
    if (base != N || sbase != ns) fail(MSS_ERR_CUDA, "colour classes do not cover every cell");
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
  h->fsrc.reset(h, nnzb);
  h->fdp.reset(h, N);
  h->fslo.reset(h, N);
  h->fshi.reset(h, N);
  h->fv.reset(h, (size_t)nnzb * NB * NB);
  h->fcs.reset(h, (size_t)nnzb * 2 * NB);
  h->fdinv.reset(h, (size_t)N * NB * NB);
  {
    DBuf<int> qlo(h, N), qhi(h, N);
    k_strip_ranges<<<grid_for(ns, 256), 256, 0, h->stream>>>(ns, h->st_first.p, h->st_len.p,
                                                             qlo.p, qhi.p);
    MSS_LAUNCH_CK("k_strip_ranges");
    k_factor_pattern<<<grid_for(N, 128), 128, 0, h->stream>>>(
        N, h->perm.p, h->iperm.p, h->rp.p, h->ci.p, h->frp.p, qlo.p, qhi.p, h->fpos.p,
        h->fcell.p, h->fsrc.p, h->fdp.p, h->fslo.p, h->fshi.p);
    MSS_LAUNCH_CK("k_factor_pattern");
  }
}

// Numeric part of the last stage on the symbolic set-up above (ordering,
// strips, factor pattern): factor values and column slices from Abar, the
// factorisation colour by colour, the in-strip upper scaling and the chain
// blocks. Run again alone when only the values change.
template <int NB>
void bilu_numeric_nb(Handle* h) {
  const int N = h->N;
  const int nnzb = h->nnzb;
  const bool bjac = h->opt.stage3 == MSS_BLOCK_JACOBI;
  const bool strips = !bjac && (h->opt.ilu_order == MSS_STRIPS || h->opt.ilu_order == MSS_STRIPS_JP);
  const int S = strips ? h->opt.ilu_strip : 1;
  {
    long long tot = (long long)nnzb * NB * NB;
    unsigned g = grid_for(tot, 256);
    if (g > 8u * h->num_sms * 8) g = 8u * h->num_sms * 8;
    k_factor_values<NB><<<g, 256, 0, h->stream>>>(nnzb, h->fsrc.p, h->abar.p, h->p, h->t,
                                                  h->fv.p, h->fcs.p);
    MSS_LAUNCH_CK("k_factor_values");
  }
  // ---- factorisation, colour by colour (NB lanes per strip, one-warp CTAs so
  // that small colours spread over the SMs)
  DBuf<int> bad(h, 1);
  fill_int(h, bad.p, 0x7fffffff, 1);
  for (int c = 0; c < h->ncol; ++c) {
    const int s0 = h->sc_start[c], s1 = h->sc_start[c + 1];
    if (s1 <= s0) continue;
    constexpr int G = 32 / NB;
    const int form = h->opt.factor_form;
    const bool warp_form =
        form == MSS_FACTOR_WARP ||
        (form == MSS_FACTOR_AUTO && (long long)(s1 - s0) < (long long)kSmallColour * G * h->num_sms);
    if (warp_form) {
      constexpr int FT = 32 * factor_warps<NB>();
      k_bilu_factor_warp<NB><<<grid_for((long long)(s1 - s0) * 32, FT), FT, 0, h->stream>>>(
          s0, s1, h->st_first.p, h->st_len.p, h->frp.p, h->fdp.p, h->fpos.p, h->fv.p,
          h->fdinv.p, bjac ? 1 : 0, bad.p);
      MSS_LAUNCH_CK("k_bilu_factor_warp");
    } else {
      k_bilu_factor<NB><<<(unsigned)((s1 - s0 + G - 1) / G), 32, 0, h->stream>>>(
          s0, s1, h->st_first.p, h->st_len.p, h->frp.p, h->fdp.p, h->fpos.p, h->fv.p,
          h->fdinv.p, bjac ? 1 : 0, bad.p);
      MSS_LAUNCH_CK("k_bilu_factor");
    }
  }
  const int badq = read_int(h, bad.p);
  if (badq != 0x7fffffff)
    fail(MSS_ERR_SINGULAR_BLOCK, "block ILU(0): zero pivot in the diagonal block at position " +
                                     std::to_string(badq));
  if (!bjac) {
    if (strips && S > 1) {
      constexpr int RPW = 32 / NB;
      k_strip_upper_scale<NB><<<grid_for(((long long)N + RPW - 1) / RPW * 32, 256), 256, 0,
                                 h->stream>>>(N, h->fdp.p, h->fshi.p, h->fdinv.p, h->fv.p);
      MSS_LAUNCH_CK("k_strip_upper_scale");
    }
    // chain blocks (zero blocks and no flags when strips are single cells)
    h->cL.reset(h, (size_t)N * NB * NB);
    h->cG.reset(h, (size_t)N * NB * NB);
    h->cflag.reset(h, N);
    k_chain_blocks<NB><<<grid_for((long long)N * NB * NB, 256), 256, 0, h->stream>>>(
        N, h->fslo.p, h->fdp.p, h->fshi.p, h->fpos.p, h->fv.p, h->cL.p, h->cG.p, h->cflag.p);
    MSS_LAUNCH_CK("k_chain_blocks");
  }
}

// Factor data in one storage type V with vectors in compute type C: FP64 / FP64,
// or BF16 blocks with FP32 vectors in the mixed form.
template <class V, class C>
struct Factors {
  const V *fv, *fdinv, *cL, *cG;
  const C* fcs;
  C* w;
};

Factors<double, double> factors(Handle* h, const double*) {
  return {h->fv.p, h->fdinv.p, h->cL.p, h->cG.p, h->fcs.p, h->w.p};
}
Factors<__nv_bfloat16, float> factors(Handle* h, const float*) {
  return {h->fvh.p, h->fdinvh.p, h->cLh.p, h->cGh.p, h->fcsf.p, h->wf.p};
}

// The sweep kernels follow one another on the handle's stream with
// programmatic serialization: each may be scheduled once its predecessor has
// passed its own wait, loads what does not depend on that predecessor (factor
// data, chain blocks, the stage terms of later colours) and then waits for it
// (bilu_sweeps.cuh), so one launch's ramp overlaps the drain of the one
// before. The first sweep kernel is launched without the attribute.
template <class... P, class... A>
void launch_sweep(void (*k)(P...), unsigned grid, unsigned block, cudaStream_t s, bool pdl,
                  A... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  MSS_CK(cudaLaunchKernelEx(&cfg, k, ((P)args)...));
}

template <int NB, int MODE, class V, class C>
void sweeps(Handle* h, const Factors<V, C>& F, const double* r, const C* xT, const C* vP,
            double* y) {
  constexpr int RPW = 32 / NB;
  const bool bjac = h->opt.stage3 == MSS_BLOCK_JACOBI;
  // strips longer than one cell carry in-strip couplings (chain passes)
  const bool chains = !bjac &&
                      (h->opt.ilu_order == MSS_STRIPS || h->opt.ilu_order == MSS_STRIPS_JP) &&
                      h->opt.ilu_strip > 1;
  const int T = h->tb;   // any multiple of 32: results do not depend on it
  // with the event trace on, the events between launches would stand between
  // the kernels, so the attribute is not asked for
  const bool pdl = !h->trace;
  bool first = true;
  for (int c = 0; c < h->ncol; ++c) {
    const int q0 = h->cstart[c], q1 = h->cstart[c + 1];
    const int s0 = h->sc_start[c], s1 = h->sc_start[c + 1];
    if (q1 <= q0) continue;
    TraceScope ts(h, TR_BILU_FWD);
    const long long rw = (q1 - q0 + RPW - 1) / RPW;
    launch_sweep(k_bilu_fwd_par<NB, MODE, V, C>, grid_for(rw * 32, T), T, h->stream,
                 pdl && !first, q0, q1, h->perm.p, h->frp.p, h->fslo.p, h->fpos.p, h->fcell.p,
                 F.fv, F.fcs, r, xT, vP, F.w, bjac ? 0 : 1, first ? 1 : 0);
    MSS_LAUNCH_CK("k_bilu_fwd_par");
    first = false;
    if (chains) {
      const long long sw = (s1 - s0 + RPW - 1) / RPW;
      launch_sweep(k_bilu_fwd_chain<NB, V, C>, grid_for(sw * 32, kChainThreads), kChainThreads,
                   h->stream, pdl, s0, s1, h->st_first.p, h->st_len.p, h->fslo.p, h->fdp.p,
                   h->fpos.p, F.fv, F.cL, h->cflag.p, F.w);
      MSS_LAUNCH_CK("k_bilu_fwd_chain");
    }
  }
  for (int c = h->ncol - 1; c >= 0; --c) {
    const int q0 = h->cstart[c], q1 = h->cstart[c + 1];
    const int s0 = h->sc_start[c], s1 = h->sc_start[c + 1];
    if (q1 <= q0) continue;
    TraceScope ts(h, TR_BILU_BWD);
    if (!bjac) {
      const long long rw = (q1 - q0 + RPW - 1) / RPW;
      launch_sweep(k_bilu_bwd_par<NB, V, C>, grid_for(rw * 32, T), T, h->stream, pdl, q0, q1,
                   h->frp.p, h->fshi.p, h->fpos.p, F.fv, F.fdinv, F.w);
      MSS_LAUNCH_CK("k_bilu_bwd_par");
    }
    const long long sw = (s1 - s0 + RPW - 1) / RPW;
    launch_sweep(k_bilu_bwd_chain<NB, V, C>, grid_for(sw * 32, kChainThreads), kChainThreads,
                 h->stream, pdl, s0, s1, h->st_first.p, h->st_len.p, h->fdp.p, h->fshi.p,
                 h->fpos.p, F.fv, F.fdinv, F.cG, h->cflag.p, F.w, bjac ? 0 : 1, h->perm.p,
                 (MODE & 1) ? xT : nullptr, (MODE & 2) ? vP : nullptr, h->p, h->t, y);
    MSS_LAUNCH_CK("k_bilu_bwd_chain");
  }
}

template <int NB, class C>
void last_stage_nb(Handle* h, const double* r, const C* xT, const C* vP, double* y) {
  const auto F = factors(h, (const C*)nullptr);
  const int mode = (xT ? 1 : 0) | (vP ? 2 : 0);
  switch (mode) {
    case 0: sweeps<NB, 0>(h, F, r, xT, vP, y); break;
    case 1: sweeps<NB, 1>(h, F, r, xT, vP, y); break;
    case 2: sweeps<NB, 2>(h, F, r, xT, vP, y); break;
    default: sweeps<NB, 3>(h, F, r, xT, vP, y); break;
  }
}

}  // namespace

int colour_points(Handle* h, int n, const int* rp, const int* ci, uint64_t seed, int* colour) {
  fill_int(h, colour, -1, n);
  DBuf<int> pick(h, n), left(h, 1), maxcol(h, 1);
  fill_int(h, maxcol.p, -1, 1);
  int remaining = n, rounds = 0;
  while (remaining > 0) {
    for (int r = 0; r < 3; ++r) {   // three rounds per read-back, as for the strips
      if (++rounds > n + 3) fail(MSS_ERR_CUDA, "colouring did not terminate");
      k_jp_pick<<<grid_for((long long)n * 32, 128), 128, 0, h->stream>>>(
          n, 1, n, rp, ci, seed, KEY_CELL, colour, pick.p, left.p);
      MSS_LAUNCH_CK("k_jp_pick");
      k_jp_commit<<<grid_for(n, 256), 256, 0, h->stream>>>(n, pick.p, colour, left.p, maxcol.p);
      MSS_LAUNCH_CK("k_jp_commit");
    }
    remaining = read_int(h, left.p);
  }
  return read_int(h, maxcol.p) + 1;
}

void bilu_setup(Handle* h) {
  TraceScope ts(h, TR_SETUP_BILU);
  MSS_NB_DISPATCH(h->nb, (bilu_setup_nb<NB>(h), bilu_numeric_nb<NB>(h)));
}

void bilu_refactor(Handle* h) {
  TraceScope ts(h, TR_SETUP_BILU);
  MSS_NB_DISPATCH(h->nb, bilu_numeric_nb<NB>(h));
}

void last_stage_apply(Handle* h, const double* r, const double* xT, const double* vP, double* y) {
  MSS_NB_DISPATCH(h->nb, (last_stage_nb<NB, double>(h, r, xT, vP, y)));
}

void last_stage_apply(Handle* h, const double* r, const float* xT, const float* vP, double* y) {
  MSS_NB_DISPATCH(h->nb, (last_stage_nb<NB, float>(h, r, xT, vP, y)));
}

// BF16 copies of the factor blocks, the in-strip chain blocks and D^-1 blocks,
// FP32 copies of the coupling column slices, and the FP32 work vector.
void pack_last_stage_mixed(Handle* h) {
  h->fvh.reset(h, h->fv.n);
  to_bf16(h, h->fv.p, h->fvh.p, (long long)h->fv.n);
  h->fdinvh.reset(h, h->fdinv.n);
  to_bf16(h, h->fdinv.p, h->fdinvh.p, (long long)h->fdinv.n);
  h->cLh.reset(h, h->cL.n);
  to_bf16(h, h->cL.p, h->cLh.p, (long long)h->cL.n);
  h->cGh.reset(h, h->cG.n);
  to_bf16(h, h->cG.p, h->cGh.p, (long long)h->cG.n);
  h->fcsf.reset(h, h->fcs.n);
  to_float(h, h->fcs.p, h->fcsf.p, (long long)h->fcs.n);
  h->wf.reset(h, (size_t)h->N * h->nb);
}

}  // namespace mss
