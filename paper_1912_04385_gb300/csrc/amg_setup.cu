// amg_setup.cu -- classical AMG set-up on the device (Sec. 5.1: classical
// AMG, coarse size <= max_coarse; coarsening read as PMIS).
//
// Per level: sign-aware strength of connection, PMIS C/F splitting with a
// SplitMix64 measure, direct classical interpolation with strong-F
// distribution and row truncation, R = P^T, and the Galerkin product
// A_c = R (A P) by a two-pass row-wise SpGEMM.
//
// Compiled with -fmad=false, and every floating-point reduction runs in the
// order the method defines it (ascending columns, ascending inner index), so
// the strength tests -- floating point deciding an index -- take the same
// decisions as the FP64 definition.
#include <cmath>
#include <cstring>

#include <memory>
#include <cstdlib>
#include <cstdio>
#include <chrono>

#include "common.cuh"

namespace mss {

void coarse_inverse(Handle* h, Hierarchy& H);   // amg_cycle.cu

namespace {

enum { ST_F = 0, ST_C = 1, ST_U = -1 };

__device__ __forceinline__ double unit53(uint64_t h) {
  return (double)(h >> 11) * (1.0 / 9007199254740992.0);
}

// j strong for i  <=>  -sgn(a_ii) a_ij >= theta * max_{k != i}(-sgn(a_ii) a_ik) > 0
__global__ void k_strength(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                           const double* __restrict__ v, double theta,
                           unsigned char* __restrict__ strong, int* __restrict__ scount) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int b = rp[i], e = rp[i + 1];
  double aii = 0.0;
  for (int k = b; k < e; ++k)
    if (ci[k] == i) aii = v[k];
  double sg = aii < 0.0 ? 1.0 : -1.0;
  double mx = -INFINITY;
  for (int k = b; k < e; ++k)
    if (ci[k] != i) {
      double val = sg * v[k];
      if (val > mx) mx = val;
    }
  double thr = theta * mx;
  int cnt = 0;
  for (int k = b; k < e; ++k) {
    unsigned char s = (ci[k] != i && mx > 0.0 && sg * v[k] >= thr) ? 1 : 0;
    strong[k] = s;
    cnt += s;
  }
  scount[i] = cnt;
}

__global__ void k_fill_strong(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                              const unsigned char* __restrict__ strong,
                              const int* __restrict__ srp, int* __restrict__ sci) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int q = srp[i];
  for (int k = rp[i]; k < rp[i + 1]; ++k)
    if (strong[k]) sci[q++] = ci[k];
}

// entries per column of an n-row CSR pattern (rows' ranges only: entries past
// rp[n] in an over-sized array are never read)
__global__ void k_count_cols(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                             int* __restrict__ cnt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int k = rp[i]; k < rp[i + 1]; ++k) atomicAdd(&cnt[ci[k]], 1);
}

// scatter of a CSR pattern (and optional values) into its transpose; the
// order inside a transposed row is fixed afterwards by k_sort_rows
__global__ void k_fill_transpose(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                 const double* __restrict__ v, int* __restrict__ fill,
                                 int* __restrict__ tci, double* __restrict__ tv) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int k = rp[i]; k < rp[i + 1]; ++k) {
    int pos = atomicAdd(&fill[ci[k]], 1);
    tci[pos] = i;
    if (v) tv[pos] = v[k];
  }
}

__global__ void k_sort_rows(int n, const int* __restrict__ rp, int* __restrict__ ci,
                            double* __restrict__ v) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int b = rp[i], e = rp[i + 1];
  for (int a = b + 1; a < e; ++a) {
    int c = ci[a];
    double x = v ? v[a] : 0.0;
    int q = a - 1;
    while (q >= b && ci[q] > c) {
      ci[q + 1] = ci[q];
      if (v) v[q + 1] = v[q];
      --q;
    }
    ci[q + 1] = c;
    if (v) v[q + 1] = x;
  }
}

__global__ void k_row_lengths(int n, const int* __restrict__ rp, int* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = rp[i + 1] - rp[i];
}

__global__ void k_pmis_init(int n, const int* __restrict__ tcount, uint64_t seed, int level,
                            double* __restrict__ lam, int* __restrict__ state,
                            int* __restrict__ undecided) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint64_t key = ((uint64_t)(unsigned)level << 32) | (uint64_t)(unsigned)i;
  lam[i] = (double)tcount[i] + unit53(splitmix64(seed, key));
  int st = tcount[i] == 0 ? ST_F : ST_U;
  state[i] = st;
  if (st == ST_U) atomicAdd(undecided, 1);
}

__device__ __forceinline__ bool beats(const double* lam, int a, int b) {
  double la = lam[a], lb = lam[b];
  return la > lb || (la == lb && a > b);
}

// an undecided point becomes C when its (measure, index) beats every
// undecided strong neighbour in either direction
// (also zeroes the round's undecided count, which the update kernel after it
// accumulates)
__global__ void k_pmis_select(int n, const int* __restrict__ srp, const int* __restrict__ sci,
                              const int* __restrict__ strp, const int* __restrict__ stci,
                              const double* __restrict__ lam, const int* __restrict__ state,
                              int* __restrict__ newc, int* __restrict__ undecided) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) *undecided = 0;
  if (i >= n) return;
  int pick = 0;
  if (state[i] == ST_U) {
    pick = 1;
    for (int k = srp[i]; k < srp[i + 1] && pick; ++k) {
      int j = sci[k];
      if (state[j] == ST_U && beats(lam, j, i)) pick = 0;
    }
    for (int k = strp[i]; k < strp[i + 1] && pick; ++k) {
      int j = stci[k];
      if (state[j] == ST_U && beats(lam, j, i)) pick = 0;
    }
  }
  newc[i] = pick;
}

// new C points are fixed; undecided points depending strongly on one become F
__global__ void k_pmis_update(int n, const int* __restrict__ srp, const int* __restrict__ sci,
                              int* __restrict__ state, const int* __restrict__ newc,
                              int* __restrict__ undecided) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (state[i] != ST_U) return;
  if (newc[i]) {
    state[i] = ST_C;
    return;
  }
  for (int k = srp[i]; k < srp[i + 1]; ++k)
    if (newc[sci[k]]) {
      state[i] = ST_F;
      return;
    }
  atomicAdd(undecided, 1);
}

// F points with strong dependencies but no strong C point become C
__global__ void k_pmis_finalize(int n, const int* __restrict__ srp, const int* __restrict__ sci,
                                const int* __restrict__ state, int* __restrict__ cf) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int st = state[i];
  int c = st == ST_C ? 1 : 0;
  if (st == ST_F && srp[i + 1] > srp[i]) {
    int hasc = 0;
    for (int k = srp[i]; k < srp[i + 1]; ++k) hasc |= state[sci[k]] == ST_C;
    c = !hasc;
  }
  cf[i] = c;
}

// The interpolation kernels are bound by the FP64 pipe, which executes a
// warp's instruction whatever the number of its active lanes (a thread per row
// leaves few lanes active in the inner loops). So their inner loops test
// signs on the bits (integer pipe) and share one reciprocal among the
// quotients of one divisor; both give the bits of the plain expressions.
//
// sign_of(x): -1 when x < 0.0, +1 when x > 0.0, 0 for zeros and NaN (the
// values both comparisons reject). opposite(sign_of(akk), akm) is the test
// "akm has the sign opposite to akk's", akk < 0.0 ? akm > 0.0 : akm < 0.0.
__device__ __forceinline__ int sign_of(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned long long mag = u & 0x7fffffffffffffffULL;
  if (mag == 0ULL || mag > 0x7ff0000000000000ULL) return 0;
  return (u >> 63) ? -1 : 1;
}
__device__ __forceinline__ bool opposite(int sk, double akm) {
  return sign_of(akm) == (sk < 0 ? 1 : -1);
}

// a / b, correctly rounded, from y = RN(1/b) computed once per divisor:
// q0 = RN(a y) is within 1.5 ulp of a/b; one correction with the remainder,
// q1 = RN(q0 + RN(a - b q0) y), is within one ulp; then r = a - b q1 is exact
// and RN(q1 + r y) = RN(a/b) (Markstein's theorem: P. W. Markstein,
// "Computation of elementary functions on the IBM RISC System/6000
// processor", IBM J. Res. Develop. 34(1), 1990; the FMA division sequences of
// Cornea, Harrison and Tang). The theorem needs every quantity normal: an
// operand with a binary exponent outside [-400, 400] (zeros, subnormals,
// infinities and NaN included) takes the division itself. The products are
// explicit FMAs, so -fmad=false leaves them as written.
struct Recip {
  double b, y;
  bool fast;
};
__device__ __forceinline__ bool mid_exponent(double x) {
  const unsigned e = (unsigned)((unsigned long long)__double_as_longlong(x) >> 52) & 0x7ffu;
  return e >= 1023u - 400u && e <= 1023u + 400u;
}
__device__ __forceinline__ Recip recip(double b) {
  Recip d;
  d.b = b;
  d.fast = mid_exponent(b);
  d.y = d.fast ? 1.0 / b : 0.0;
  return d;
}
__device__ __forceinline__ double quot(double a, const Recip& d) {
  if (!d.fast || !mid_exponent(a)) return a / d.b;
  double q = __dmul_rn(a, d.y);
  double r = __fma_rn(-q, d.b, a);
  q = __fma_rn(r, d.y, q);
  r = __fma_rn(-q, d.b, a);
  return __fma_rn(r, d.y, q);
}

// Direct classical interpolation with distribution of strong F couplings
// (same formula and operation order as the FP64 definition). Row i's work
// arrays live in the scratch segment [rp[i], rp[i+1]) of A's pattern.
__global__ void k_interp(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                         const double* __restrict__ v, const unsigned char* __restrict__ strong,
                         const int* __restrict__ cf, const int* __restrict__ cidx, int maxel,
                         int* __restrict__ scr_ci, double* __restrict__ scr_v,
                         int* __restrict__ scr_k, int* __restrict__ plen) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int b = rp[i], e = rp[i + 1];
  // the row's work lists in thread-local arrays when the row is short enough
  // (the common case), else in its scratch segment; the result goes to the
  // scratch segment either way
  constexpr int kLocal = 16;
  int lci[kLocal], lkeep[kLocal];
  double lnum[kLocal];
  const bool loc = e - b <= kLocal;
  int* cset = loc ? lci : scr_ci + b;
  double* num = loc ? lnum : scr_v + b;
  int* keep = loc ? lkeep : scr_k + b;
  if (cf[i]) {
    scr_ci[b] = cidx[i];
    scr_v[b] = 1.0;
    plen[i] = 1;
    return;
  }
  int nC = 0;
  double aii = 0.0;
  for (int k = b; k < e; ++k) {
    int j = ci[k];
    if (j == i) aii = v[k];
    else if (strong[k] && cf[j]) { cset[nC] = j; num[nC] = v[k]; ++nC; }
  }
  if (nC == 0) { plen[i] = 0; return; }
  double d = aii;
  for (int k = b; k < e; ++k) {
    int j = ci[k];
    if (j == i) continue;
    if (strong[k] && cf[j]) continue;
    if (strong[k] && !cf[j]) {
      double aik = v[k];
      double akk = 0.0;
      for (int f = rp[j]; f < rp[j + 1]; ++f)
        if (ci[f] == j) akk = v[f];
      const int sk = sign_of(akk);
      double sigma = 0.0;
      for (int f = rp[j]; f < rp[j + 1]; ++f) {
        int m = ci[f];
        if (m == j) continue;
        double akm = v[f];
        bool inC = false;
        for (int q = 0; q < nC; ++q) if (cset[q] == m) { inC = true; break; }
        if (inC && opposite(sk, akm)) sigma = sigma + akm;
      }
      if (sigma == 0.0) {
        d = d + aik;
      } else {
        const Recip rs = recip(sigma);
        for (int f = rp[j]; f < rp[j + 1]; ++f) {
          int m = ci[f];
          if (m == j) continue;
          double akm = v[f];
          if (!opposite(sk, akm)) continue;
          for (int q = 0; q < nC; ++q)
            if (cset[q] == m) {
              double tq = aik * akm;
              tq = quot(tq, rs);
              num[q] = num[q] + tq;
              break;
            }
        }
      }
    } else {
      d = d + v[k];
    }
  }
  if (d == 0.0 || !isfinite(d)) { plen[i] = 0; return; }
  {
    // -(num / d): RN(-x) = -RN(x)
    const Recip rd = recip(d);
    for (int q = 0; q < nC; ++q) num[q] = -quot(num[q], rd);
  }
  for (int q = 0; q < nC; ++q) keep[q] = 1;
  if (maxel > 0 && nC > maxel) {
    double total = 0.0;
    for (int q = 0; q < nC; ++q) total = total + num[q];
    for (int q = 0; q < nC; ++q) keep[q] = 0;
    for (int r = 0; r < maxel; ++r) {
      int best = -1;
      for (int q = 0; q < nC; ++q) {
        if (keep[q]) continue;
        if (best < 0 || fabs(num[q]) > fabs(num[best])) best = q;
      }
      keep[best] = 1;
    }
    double kept = 0.0;
    for (int q = 0; q < nC; ++q) if (keep[q]) kept = kept + num[q];
    if (kept != 0.0) {
      double sc = total / kept;
      for (int q = 0; q < nC; ++q) if (keep[q]) num[q] = num[q] * sc;
    }
  }
  int len = 0;
  for (int q = 0; q < nC; ++q)
    if (keep[q]) {
      cset[len] = cidx[cset[q]];
      num[len] = num[q];
      ++len;
    }
  if (loc)
    for (int q = 0; q < len; ++q) {
      scr_ci[b + q] = cset[q];
      scr_v[b + q] = num[q];
    }
  plen[i] = len;
}

// The same interpolation with one warp per row, for the coarse levels whose
// long rows serialise a thread: the strong C list is collected by ballots in
// column order, the strong F neighbours are taken in column order, and for
// each the scans of its row (its diagonal, the weight sum sigma, the
// distribution) run across the lanes. Every sum is still formed in the
// definition's order (sigma and d by the warp in lane order, each num[q]
// once per neighbour, neighbours in order); the scaling, truncation and
// compaction are the thread version's code on lane 0.
__device__ __forceinline__ int find_c(const int* cset, int nC, int m) {
  for (int q = 0; q < nC; ++q)
    if (cset[q] == m) return q;
  return -1;
}

__global__ void __launch_bounds__(256)
k_interp_warp(int n, const int* __restrict__ rp, const int* __restrict__ ci,
              const double* __restrict__ v, const unsigned char* __restrict__ strong,
              const int* __restrict__ cf, const int* __restrict__ cidx, int maxel,
              int* __restrict__ scr_ci, double* __restrict__ scr_v, int* __restrict__ scr_k,
              int* __restrict__ plen) {
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const long long iw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (iw >= n) return;                       // uniform per warp
  const int i = (int)iw;
  const int b = rp[i], e = rp[i + 1];
  int* cset = scr_ci + b;
  double* num = scr_v + b;
  int* keep = scr_k + b;
  if (cf[i]) {
    if (lane == 0) {
      cset[0] = cidx[i];
      num[0] = 1.0;
      plen[i] = 1;
    }
    return;
  }
  // strong C neighbours in column order, and the diagonal
  int nC = 0;
  double aii = 0.0;
  for (int k0 = b; k0 < e; k0 += 32) {
    const int k = k0 + lane;
    int j = -1;
    double vk = 0.0;
    bool isC = false;
    if (k < e) {
      j = ci[k];
      vk = v[k];
      isC = j != i && strong[k] && cf[j];
    }
    const unsigned dm = __ballot_sync(FULL, k < e && j == i);
    if (dm) aii = __shfl_sync(FULL, vk, 31 - __clz(dm));   // the last one, as a sequential scan
    const unsigned cm = __ballot_sync(FULL, isC);
    if (isC) {
      const int pos = nC + __popc(cm & ((1u << lane) - 1u));
      cset[pos] = j;
      num[pos] = vk;
    }
    nC += __popc(cm);
  }
  if (nC == 0) {
    if (lane == 0) plen[i] = 0;
    return;
  }
  __syncwarp();
  // weak terms into d, strong F neighbours distributed, in column order
  double d = aii;
  for (int k0 = b; k0 < e; k0 += 32) {
    const int k = k0 + lane;
    int j = -1, kind = 0;                    // 1 weak, 2 strong F
    double vk = 0.0;
    if (k < e) {
      j = ci[k];
      vk = v[k];
      if (j != i) {
        const bool sk = strong[k];
        const bool cj = cf[j];
        kind = sk ? (cj ? 0 : 2) : 1;
      }
    }
    unsigned live = __ballot_sync(FULL, kind != 0);
    while (live) {
      const int t = __ffs(live) - 1;
      live &= live - 1;
      const int kd = __shfl_sync(FULL, kind, t);
      const double aik = __shfl_sync(FULL, vk, t);
      if (kd == 1) {
        d = d + aik;
        continue;
      }
      const int jj = __shfl_sync(FULL, j, t);
      const int fb = rp[jj], fe = rp[jj + 1];
      double akk = 0.0;
      for (int f0 = fb; f0 < fe; f0 += 32) {
        const int f = f0 + lane;
        const bool isd = f < fe && ci[f] == jj;
        const unsigned m = __ballot_sync(FULL, isd);
        const double vf = isd ? v[f] : 0.0;
        if (m) akk = __shfl_sync(FULL, vf, 31 - __clz(m));
      }
      const int sk = sign_of(akk);
      double sigma = 0.0;
      for (int f0 = fb; f0 < fe; f0 += 32) {
        const int f = f0 + lane;
        double akm = 0.0;
        bool add = false;
        if (f < fe) {
          const int mm = ci[f];
          akm = v[f];
          add = mm != jj && find_c(cset, nC, mm) >= 0 && opposite(sk, akm);
        }
        unsigned am = __ballot_sync(FULL, add);
        while (am) {
          const int t2 = __ffs(am) - 1;
          am &= am - 1;
          sigma = sigma + __shfl_sync(FULL, akm, t2);
        }
      }
      if (sigma == 0.0) {
        d = d + aik;
      } else {
        const Recip rs = recip(sigma);
        for (int f0 = fb; f0 < fe; f0 += 32) {
          const int f = f0 + lane;
          if (f < fe) {
            const int mm = ci[f];
            const double akm = v[f];
            if (mm != jj && opposite(sk, akm)) {
              const int q = find_c(cset, nC, mm);
              if (q >= 0) {
                double tq = aik * akm;
                tq = quot(tq, rs);
                num[q] = num[q] + tq;
              }
            }
          }
        }
        __syncwarp();
      }
    }
  }
  __syncwarp();
  if (lane != 0) return;
  if (d == 0.0 || !isfinite(d)) {
    plen[i] = 0;
    return;
  }
  {
    const Recip rd = recip(d);
    for (int q = 0; q < nC; ++q) num[q] = -quot(num[q], rd);
  }
  for (int q = 0; q < nC; ++q) keep[q] = 1;
  if (maxel > 0 && nC > maxel) {
    double total = 0.0;
    for (int q = 0; q < nC; ++q) total = total + num[q];
    for (int q = 0; q < nC; ++q) keep[q] = 0;
    for (int r = 0; r < maxel; ++r) {
      int best = -1;
      for (int q = 0; q < nC; ++q) {
        if (keep[q]) continue;
        if (best < 0 || fabs(num[q]) > fabs(num[best])) best = q;
      }
      keep[best] = 1;
    }
    double kept = 0.0;
    for (int q = 0; q < nC; ++q) if (keep[q]) kept = kept + num[q];
    if (kept != 0.0) {
      const double sc = total / kept;
      for (int q = 0; q < nC; ++q) if (keep[q]) num[q] = num[q] * sc;
    }
  }
  int len = 0;
  for (int q = 0; q < nC; ++q)
    if (keep[q]) {
      cset[len] = cidx[cset[q]];
      num[len] = num[q];
      ++len;
    }
  plen[i] = len;
}

__global__ void k_seg_copy(int n, const int* __restrict__ src_off, const int* __restrict__ src_ci,
                           const double* __restrict__ src_v, const int* __restrict__ dst_rp,
                           int* __restrict__ dst_ci, double* __restrict__ dst_v) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int s = src_off[i], d = dst_rp[i], len = dst_rp[i + 1] - dst_rp[i];
  for (int k = 0; k < len; ++k) {
    dst_ci[d + k] = src_ci[s + k];
    dst_v[d + k] = src_v[s + k];
  }
}

// ---- SpGEMM C = X Y, row by row ---------------------------------------------
__global__ void k_spgemm_count(int n, const int* __restrict__ xrp, const int* __restrict__ xci,
                               const int* __restrict__ yrp, int* __restrict__ cnt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int c = 0;
  for (int k = xrp[i]; k < xrp[i + 1]; ++k) {
    int r = xci[k];
    c += yrp[r + 1] - yrp[r];
  }
  cnt[i] = c;
}

// contributions x_ik y_kj accumulate in ascending k, then ascending j in row
// k; the row is kept sorted by column in its scratch segment
// Row i of C = X Y: the products x_ik y_kj in order (k ascending, then the
// entries of row k), each added to its column's entry, the row's columns kept
// sorted by insertion. With SHARED the row's list lives in shared memory
// (kAccumS entries per thread, entry q of thread t at q * kAccumT + t) until
// it outgrows it, then moves to the row's scratch segment [off[i], off[i+1])
// and continues there; without it, the list is in the scratch segment from
// the start (rows of few products: the shared copy costs occupancy and saves
// little). Either way every entry is the same sum in the same order; the
// result ends in the scratch segment.
constexpr int kAccumT = 128;   // threads per block (the shared layout's stride)
constexpr int kAccumS = 24;    // entries per thread in shared memory

template <bool SHARED>
__global__ void __launch_bounds__(kAccumT)
k_spgemm_accum(int n, const int* __restrict__ xrp, const int* __restrict__ xci,
               const double* __restrict__ xv, const int* __restrict__ yrp,
               const int* __restrict__ yci, const double* __restrict__ yv,
               const int* __restrict__ off, int* __restrict__ sc_ci, double* __restrict__ sc_v,
               int* __restrict__ ulen) {
  __shared__ int s_ci[SHARED ? kAccumS * kAccumT : 1];
  __shared__ double s_v[SHARED ? kAccumS * kAccumT : 1];
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int* gc = sc_ci + off[i];
  double* gv = sc_v + off[i];
  int* lc = s_ci + threadIdx.x;
  double* lv = s_v + threadIdx.x;
  int cnt = 0;
  bool spilled = !SHARED;
  for (int k = xrp[i]; k < xrp[i + 1]; ++k) {
    int r = xci[k];
    double x = xv[k];
    for (int f = yrp[r]; f < yrp[r + 1]; ++f) {
      int j = yci[f];
      double prod = x * yv[f];
      if (!spilled) {
        int lo = 0, hi = cnt;
        while (lo < hi) {
          int mid = (lo + hi) >> 1;
          if (lc[mid * kAccumT] < j) lo = mid + 1; else hi = mid;
        }
        if (lo < cnt && lc[lo * kAccumT] == j) {
          lv[lo * kAccumT] = lv[lo * kAccumT] + prod;
          continue;
        }
        if (cnt < kAccumS) {
          for (int q = cnt; q > lo; --q) {
            lc[q * kAccumT] = lc[(q - 1) * kAccumT];
            lv[q * kAccumT] = lv[(q - 1) * kAccumT];
          }
          lc[lo * kAccumT] = j;
          lv[lo * kAccumT] = 0.0 + prod;
          ++cnt;
          continue;
        }
        // the list outgrows its shared slots: on in the scratch segment
        for (int q = 0; q < cnt; ++q) {
          gc[q] = lc[q * kAccumT];
          gv[q] = lv[q * kAccumT];
        }
        spilled = true;
      }
      int lo = 0, hi = cnt;
      while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (gc[mid] < j) lo = mid + 1; else hi = mid;
      }
      if (lo < cnt && gc[lo] == j) {
        gv[lo] = gv[lo] + prod;
      } else {
        for (int q = cnt; q > lo; --q) {
          gc[q] = gc[q - 1];
          gv[q] = gv[q - 1];
        }
        gc[lo] = j;
        gv[lo] = 0.0 + prod;
        ++cnt;
      }
    }
  }
  if (!spilled)
    for (int q = 0; q < cnt; ++q) {
      gc[q] = lc[q * kAccumT];
      gv[q] = lv[q * kAccumT];
    }
  ulen[i] = cnt;
}

// 1 / a_ii and the Gershgorin bound max_i sum_j |a_ij| / |a_ii|
__global__ void k_dinv_bound(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                             const double* __restrict__ v, double* __restrict__ dinv,
                             unsigned long long* __restrict__ bound, int* __restrict__ bad) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  double s = 0.0;   // non-negative, so its bit pattern orders like the value
  if (i < n) {
    double aii = 0.0;
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
      if (ci[k] == i) aii = v[k];
      s = s + fabs(v[k]);
    }
    if (aii == 0.0 || !isfinite(aii)) {
      atomicMin(bad, i);
      dinv[i] = 0.0;
      s = 0.0;
    } else {
      double di = 1.0 / aii;
      dinv[i] = di;
      s = s * fabs(di);
    }
  }
  unsigned long long bits = (unsigned long long)__double_as_longlong(s);
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long ob = __shfl_xor_sync(0xffffffffu, bits, o);
    bits = ob > bits ? ob : bits;
  }
  if ((threadIdx.x & 31) == 0 && bits != 0ULL) atomicMax(bound, bits);
}

void sparse_product(Handle* h, int n, const int* xrp, const int* xci, const double* xv,
                    const int* yrp, const int* yci, const double* yv, DBuf<int>& crp,
                    DBuf<int>& cci, DBuf<double>& cv, int& cnnz) {
  DBuf<int> cnt(h, n), off(h, n + 1), ulen(h, n);
  k_spgemm_count<<<grid_for(n, 128), 128, 0, h->stream>>>(n, xrp, xci, yrp, cnt.p);
  MSS_LAUNCH_CK("k_spgemm_count");
  exclusive_scan(h, cnt.p, off.p, n);
  int tot = read_int(h, off.p + n);
  DBuf<int> sc_ci(h, tot > 0 ? tot : 1);
  DBuf<double> sc_v(h, tot > 0 ? tot : 1);
  // the shared-memory lists for rows of many products on average (measured
  // at 1024^2: R (A P) 270 -> 157 us on level 0; A P with about 12 products
  // a row 142 -> 180 us, so such products keep the scratch lists)
  if (tot > 16LL * n)
    k_spgemm_accum<true><<<grid_for(n, kAccumT), kAccumT, 0, h->stream>>>(
        n, xrp, xci, xv, yrp, yci, yv, off.p, sc_ci.p, sc_v.p, ulen.p);
  else
    k_spgemm_accum<false><<<grid_for(n, kAccumT), kAccumT, 0, h->stream>>>(
        n, xrp, xci, xv, yrp, yci, yv, off.p, sc_ci.p, sc_v.p, ulen.p);
  MSS_LAUNCH_CK("k_spgemm_accum");
  crp.reset(h, n + 1);
  exclusive_scan(h, ulen.p, crp.p, n);
  cnnz = read_int(h, crp.p + n);
  cci.reset(h, cnnz > 0 ? cnnz : 1);
  cv.reset(h, cnnz > 0 ? cnnz : 1);
  k_seg_copy<<<grid_for(n, 128), 128, 0, h->stream>>>(n, off.p, sc_ci.p, sc_v.p, crp.p, cci.p,
                                                      cv.p);
  MSS_LAUNCH_CK("k_seg_copy");
}

// the transpose (m rows) of an n-row CSR pattern with at most nnz entries
// (nnz sizes the output; the entries are those of the rows' ranges)
void transpose(Handle* h, int n, int m, const int* rp, const int* ci, const double* v, int nnz,
               DBuf<int>& trp, DBuf<int>& tci, DBuf<double>* tv) {
  DBuf<int> cnt(h, m > 0 ? m : 1), fill(h, m > 0 ? m : 1);
  fill_int(h, cnt.p, 0, m);
  if (nnz > 0 && n > 0) {
    k_count_cols<<<grid_for(n, 256), 256, 0, h->stream>>>(n, rp, ci, cnt.p);
    MSS_LAUNCH_CK("k_count_cols");
  }
  trp.reset(h, m + 1);
  exclusive_scan(h, cnt.p, trp.p, m);
  copy_dev(h, fill.p, trp.p, sizeof(int) * (size_t)m);
  tci.reset(h, nnz > 0 ? nnz : 1);
  if (tv) tv->reset(h, nnz > 0 ? nnz : 1);
  k_fill_transpose<<<grid_for(n, 128), 128, 0, h->stream>>>(n, rp, ci, v, fill.p, tci.p,
                                                            tv ? tv->p : nullptr);
  MSS_LAUNCH_CK("k_fill_transpose");
  k_sort_rows<<<grid_for(m, 128), 128, 0, h->stream>>>(m, trp.p, tci.p, tv ? tv->p : nullptr);
  MSS_LAUNCH_CK("k_sort_rows");
}

// Strength of connection of a scalar CSR matrix: the flag per nonzero, the
// strength graph S (strong dependencies by row) and its transpose, as PMIS
// reads them.
struct Strength {
  DBuf<unsigned char> strong;
  DBuf<int> srp, sci, strp, stci;
};

void strength_graph(Handle* h, int n, int nnz, const int* rp, const int* ci, const double* v,
                    double theta, Strength& S) {
  S.strong.reset(h, nnz > 0 ? nnz : 1);
  DBuf<int> scount(h, n);
  S.srp.reset(h, n + 1);
  k_strength<<<grid_for(n, 128), 128, 0, h->stream>>>(n, rp, ci, v, theta, S.strong.p,
                                                      scount.p);
  MSS_LAUNCH_CK("k_strength");
  exclusive_scan(h, scount.p, S.srp.p, n);
  // S has at most nnz entries: sized by that bound, no read-back (every
  // kernel on S reads the rows' ranges only)
  S.sci.reset(h, nnz > 0 ? nnz : 1);
  k_fill_strong<<<grid_for(n, 128), 128, 0, h->stream>>>(n, rp, ci, S.strong.p, S.srp.p,
                                                         S.sci.p);
  MSS_LAUNCH_CK("k_fill_strong");
  transpose(h, n, n, S.srp.p, S.sci.p, nullptr, nnz, S.strp, S.stci, nullptr);
}

// PMIS C/F split (1 = C) of AMG level `level`; |S_i^T| are the row lengths
// of the transposed strength graph
void pmis_split(Handle* h, int n, const Strength& S, uint64_t seed, int level, DBuf<int>& cf) {
  DBuf<int> tcount(h, n);
  k_row_lengths<<<grid_for(n, 256), 256, 0, h->stream>>>(n, S.strp.p, tcount.p);
  MSS_LAUNCH_CK("k_row_lengths");
  DBuf<double> lam(h, n);
  DBuf<int> state(h, n), newc(h, n), und(h, 1);
  fill_int(h, und.p, 0, 1);
  k_pmis_init<<<grid_for(n, 256), 256, 0, h->stream>>>(n, tcount.p, seed, level, lam.p, state.p,
                                                       und.p);
  MSS_LAUNCH_CK("k_pmis_init");
  // the first three rounds run without a read-back (rounds with nothing
  // undecided change nothing)
  int undecided = 1;
  int rounds = 0;
  while (undecided > 0) {
    // three synchronous rounds per read-back: a round with nothing
    // undecided changes nothing, so the split is the one of round-by-round
    // checking with fewer host synchronisations
    for (int r = 0; r < 3; ++r) {
      if (++rounds > n + 3) fail(MSS_ERR_AMG, "PMIS did not terminate");
      k_pmis_select<<<grid_for(n, 256), 256, 0, h->stream>>>(n, S.srp.p, S.sci.p, S.strp.p,
                                                             S.stci.p, lam.p, state.p, newc.p,
                                                             und.p);
      MSS_LAUNCH_CK("k_pmis_select");
      k_pmis_update<<<grid_for(n, 256), 256, 0, h->stream>>>(n, S.srp.p, S.sci.p, state.p,
                                                             newc.p, und.p);
      MSS_LAUNCH_CK("k_pmis_update");
    }
    undecided = read_int(h, und.p);
  }
  cf.reset(h, n);
  k_pmis_finalize<<<grid_for(n, 256), 256, 0, h->stream>>>(n, S.srp.p, S.sci.p, state.p, cf.p);
  MSS_LAUNCH_CK("k_pmis_finalize");
}

// Classical interpolation P (n x nc, CSR) for the split cf with coarse
// indices cidx; returns nnz(P)
// (with nc_dev, *nc_out receives *nc_dev in the same read-back as nnz(P))
int classical_interp(Handle* h, int n, int nnz, const int* rp, const int* ci, const double* v,
                     const unsigned char* strong, const int* cf, const int* cidx, int maxel,
                     DBuf<int>& prp, DBuf<int>& pci, DBuf<double>& pv,
                     const int* nc_dev = nullptr, int* nc_out = nullptr) {
  DBuf<int> scr_ci(h, nnz), scr_k(h, nnz), plen(h, n);
  DBuf<double> scr_v(h, nnz);
  if (n <= 65536 && nnz > 8LL * n) {   // few, long rows: one warp per row
    k_interp_warp<<<grid_for((long long)n * 32, 256), 256, 0, h->stream>>>(
        n, rp, ci, v, strong, cf, cidx, maxel, scr_ci.p, scr_v.p, scr_k.p, plen.p);
    MSS_LAUNCH_CK("k_interp_warp");
  } else {
    k_interp<<<grid_for(n, 128), 128, 0, h->stream>>>(n, rp, ci, v, strong, cf, cidx, maxel,
                                                      scr_ci.p, scr_v.p, scr_k.p, plen.p);
    MSS_LAUNCH_CK("k_interp");
  }
  prp.reset(h, n + 1);
  exclusive_scan(h, plen.p, prp.p, n);
  int nnzP = 0;
  if (nc_dev) {
    const int* src[2] = {prp.p + n, nc_dev};
    int got[2];
    read_ints(h, src, got, 2);
    nnzP = got[0];
    *nc_out = got[1];
  } else {
    nnzP = read_int(h, prp.p + n);
  }
  pci.reset(h, nnzP > 0 ? nnzP : 1);
  pv.reset(h, nnzP > 0 ? nnzP : 1);
  k_seg_copy<<<grid_for(n, 128), 128, 0, h->stream>>>(n, rp, scr_ci.p, scr_v.p, prp.p, pci.p,
                                                      pv.p);
  MSS_LAUNCH_CK("k_seg_copy");
  return nnzP;
}

void level_prepare(Handle* h, Level& L) {
  int n = L.n;
  L.dinv.reset(h, n);
  // the bound's bits and the first row with a zero diagonal in one word pair,
  // read back together (one host synchronisation per level)
  DBuf<unsigned long long> res(h, 2);
  unsigned long long* bound = res.p;
  int* bad = reinterpret_cast<int*>(res.p + 1);
  MSS_CK(cudaMemsetAsync(res.p, 0, 2 * sizeof(unsigned long long), h->stream));
  fill_int(h, bad, 0x7fffffff, 1);
  k_dinv_bound<<<grid_for(n, 256), 256, 0, h->stream>>>(n, L.rp.p, L.ci.p, L.v.p, L.dinv.p,
                                                        bound, bad);
  MSS_LAUNCH_CK("k_dinv_bound");
  unsigned long long both[2] = {0, 0};
  read_back(h, both, res.p, sizeof(both));
  const unsigned long long bits = both[0];
  int badrow = 0;
  std::memcpy(&badrow, &both[1], sizeof(int));
  if (badrow != 0x7fffffff)
    fail(MSS_ERR_AMG, "AMG level of size " + std::to_string(n) + ": zero diagonal in row " +
                          std::to_string(badrow));
  double lam;
  std::memcpy(&lam, &bits, sizeof(lam));
  L.lam = lam;
  L.b.reset(h, n);
  L.x.reset(h, n);
  L.x2.reset(h, n);
  L.r.reset(h, n);
  L.d.reset(h, n);
}

__global__ void k_flag_eq(int n, const int* __restrict__ a, int c, int* __restrict__ f) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) f[i] = a[i] == c ? 1 : 0;
}

__global__ void k_place_eq(int n, const int* __restrict__ a, int c, int base,
                           const int* __restrict__ rank, int* __restrict__ order) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && a[i] == c) order[base + rank[i]] = i;
}

// Multicolour Gauss-Seidel order of a level: Jones-Plassmann colours of A's
// graph, then the points colour-major, ascending inside each colour.
void level_colours(Handle* h, Level& L) {
  const int n = L.n;
  DBuf<int> col(h, n), flag(h, n), rank(h, n + 1);
  L.ncolour = colour_points(h, n, L.rp.p, L.ci.p, h->opt.seed, col.p);
  L.cstart.assign(L.ncolour + 1, 0);
  L.mcorder.reset(h, n);
  int base = 0;
  for (int c = 0; c < L.ncolour; ++c) {
    k_flag_eq<<<grid_for(n, 256), 256, 0, h->stream>>>(n, col.p, c, flag.p);
    MSS_LAUNCH_CK("k_flag_eq");
    exclusive_scan(h, flag.p, rank.p, n);
    k_place_eq<<<grid_for(n, 256), 256, 0, h->stream>>>(n, col.p, c, base, rank.p, L.mcorder.p);
    MSS_LAUNCH_CK("k_place_eq");
    L.cstart[c] = base;
    base += read_int(h, rank.p + n);
  }
  L.cstart[L.ncolour] = base;
  if (base != n) fail(MSS_ERR_CUDA, "AMG level colours do not cover every point");
}

// ---- system AMG for CPTR: 2 x 2 blocks on a point graph ---------------------
// Scalar form of a 2 x 2 block CSR with the two unknowns of a point
// interleaved: row 2i+k holds, for each block of point row i in order, the
// entries (k, 0) and (k, 1) at columns 2j and 2j+1.
__global__ void k_b2s(int np, const int* __restrict__ brp, const int* __restrict__ bci,
                      const double* __restrict__ bv, int* __restrict__ srp,
                      int* __restrict__ sci, double* __restrict__ sv) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * np) return;
  const int i = t >> 1, k = t & 1;
  const int b = brp[i], e = brp[i + 1], len = e - b;
  const int base = 4 * b + 2 * k * len;
  srp[t] = base;
  if (t == 2 * np - 1) srp[2 * np] = 4 * e;
  for (int q = 0; q < len; ++q)
    for (int l = 0; l < 2; ++l) {
      sci[base + 2 * q + l] = 2 * bci[b + q] + l;
      sv[base + 2 * q + l] = bv[(size_t)4 * (b + q) + 2 * k + l];
    }
}

// Norm matrix of the blocks: -|B_ij|_F off the diagonal, |B_ii|_F on it
// (squares summed in the order b00, b01, b10, b11)
__global__ void k_block_norm(int np, const int* __restrict__ brp, const int* __restrict__ bci,
                             const double* __restrict__ bv, double* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  for (int e = brp[i]; e < brp[i + 1]; ++e) {
    const double* q = bv + (size_t)4 * e;
    const double f = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    out[e] = bci[e] == i ? f : -f;
  }
}

__global__ void k_block_entry(int nnzb, const double* __restrict__ bv, int idx,
                              double* __restrict__ out) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < nnzb) out[e] = bv[(size_t)4 * e + idx];
}

// inverse of each point's 2 x 2 diagonal block: Gauss-Jordan without
// pivoting, divisions as written (the smoother's D_i^-1)
__global__ void k_dinv2(int np, const int* __restrict__ brp, const int* __restrict__ bci,
                        const double* __restrict__ bv, double* __restrict__ dinv2,
                        int* __restrict__ bad) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  int d = -1;
  for (int e = brp[i]; e < brp[i + 1]; ++e)
    if (bci[e] == i) d = e;
  if (d < 0) {
    atomicMin(bad, i);
    return;
  }
  double a[4], inv[4] = {1.0, 0.0, 0.0, 1.0};
  for (int t = 0; t < 4; ++t) a[t] = bv[(size_t)4 * d + t];
  for (int k = 0; k < 2; ++k) {
    const double piv = a[2 * k + k];
    if (piv == 0.0 || !isfinite(piv)) {
      atomicMin(bad, i);
      return;
    }
    for (int j = 0; j < 2; ++j) {
      a[2 * k + j] = a[2 * k + j] / piv;
      inv[2 * k + j] = inv[2 * k + j] / piv;
    }
    const int r = 1 - k;
    const double f = a[2 * r + k];
    for (int j = 0; j < 2; ++j) {
      a[2 * r + j] = a[2 * r + j] - f * a[2 * k + j];
      inv[2 * r + j] = inv[2 * r + j] - f * inv[2 * k + j];
    }
  }
  for (int t = 0; t < 4; ++t) dinv2[(size_t)4 * i + t] = inv[t];
}

// the point split per unknown: cf2[2i+k] = cf[i]
__global__ void k_dup2(int np, const int* __restrict__ cf, int* __restrict__ cf2) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < 2 * np) cf2[t] = cf[t >> 1];
}

// interleaved P: row 2i+k is row i of P^k with columns 2c+k
__global__ void k_p2_len(int np, const int* __restrict__ prp0, const int* __restrict__ prp1,
                         int* __restrict__ len) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * np) return;
  const int i = t >> 1;
  const int* rp = (t & 1) ? prp1 : prp0;
  len[t] = rp[i + 1] - rp[i];
}

__global__ void k_p2_fill(int np, const int* __restrict__ prp0, const int* __restrict__ pci0,
                          const double* __restrict__ pv0, const int* __restrict__ prp1,
                          const int* __restrict__ pci1, const double* __restrict__ pv1,
                          const int* __restrict__ prp, int* __restrict__ pci,
                          double* __restrict__ pv) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * np) return;
  const int i = t >> 1, k = t & 1;
  const int* rp = k ? prp1 : prp0;
  const int* ci = k ? pci1 : pci0;
  const double* v = k ? pv1 : pv0;
  int q = prp[t];
  for (int e = rp[i]; e < rp[i + 1]; ++e, ++q) {
    pci[q] = 2 * ci[e] + k;
    pv[q] = v[e];
  }
}

// 2 x 2 blocks of a scalar interleaved matrix: block row I holds every point
// with an entry in row 2I or 2I+1 (the merged, ascending point columns);
// fill == false counts them, fill == true writes columns and values (the
// values must be zeroed first: absent entries stay zero)
__global__ void k_s2b(int np, const int* __restrict__ srp, const int* __restrict__ sci,
                      const double* __restrict__ sv, int* __restrict__ cnt,
                      const int* __restrict__ brp, int* __restrict__ bci,
                      double* __restrict__ bv, int fill) {
  int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= np) return;
  int a = srp[2 * I], ae = srp[2 * I + 1], b = srp[2 * I + 1], be = srp[2 * I + 2];
  int q = fill ? brp[I] : 0, last = -1;
  while (a < ae || b < be) {
    const int ja = a < ae ? sci[a] / 2 : 0x7fffffff;
    const int jb = b < be ? sci[b] / 2 : 0x7fffffff;
    const int j = ja < jb ? ja : jb;
    if (j != last) {
      if (fill) bci[q] = j;
      ++q;
      last = j;
    }
    if (ja == j) {
      if (fill) bv[(size_t)4 * (q - 1) + (sci[a] & 1)] = sv[a];
      ++a;
    } else {
      if (fill) bv[(size_t)4 * (q - 1) + 2 + (sci[b] & 1)] = sv[b];
      ++b;
    }
  }
  if (!fill) cnt[I] = q;
}

}  // namespace

// Host time per set-up phase, printed when MSS_SETUP_TIMES is set (each mark
// synchronises the stream, so only for diagnostics).
struct PhaseClock {
  Handle* h;
  bool on;
  std::chrono::steady_clock::time_point t;
  double acc[7] = {};
  explicit PhaseClock(Handle* hh)
      : h(hh), on(std::getenv("MSS_SETUP_TIMES") != nullptr), t(std::chrono::steady_clock::now()) {}
  void mark(int k) {
    if (!on) return;
    cudaStreamSynchronize(h->stream);
    const auto now = std::chrono::steady_clock::now();
    acc[k] += std::chrono::duration<double, std::milli>(now - t).count();
    t = now;
  }
  ~PhaseClock() {
    if (on)
      std::fprintf(stderr, "mss amg build (ms): prepare %.2f strength %.2f pmis %.2f interp %.2f "
                           "transpose %.2f rap %.2f coarse %.2f\n",
                   acc[0], acc[1], acc[2], acc[3], acc[4], acc[5], acc[6]);
  }
};

void amg_build(Handle* h, Hierarchy& H, int n0, int nnz0, const int* rp0, const int* ci0,
               const double* vals0, const float* learned, std::vector<DBuf<int>>* frozen_cf) {
  const mss_options& o = h->opt;
  PhaseClock pc(h);
  H.lev.clear();
  H.lev.reserve(32);
  {
    Level L0;
    L0.n = n0;
    L0.nnz = nnz0;
    L0.rp.reset(h, n0 + 1);
    L0.ci.reset(h, nnz0);
    L0.v.reset(h, nnz0);
    copy_dev(h, L0.rp.p, rp0, sizeof(int) * ((size_t)n0 + 1));
    copy_dev(h, L0.ci.p, ci0, sizeof(int) * (size_t)nnz0);
    copy_dev(h, L0.v.p, vals0, sizeof(double) * (size_t)nnz0);
    H.lev.push_back(std::move(L0));
  }
  const int max_levels = o.amg_max_levels < 1 ? 1 : (o.amg_max_levels > 25 ? 25 : o.amg_max_levels);
  for (int l = 0;; ++l) {
    level_prepare(h, H.lev[l]);
    pc.mark(0);
    int n = H.lev[l].n, nnz = H.lev[l].nnz;
    if (n <= o.amg_max_coarse || l + 1 >= max_levels) break;
    const int* rp = H.lev[l].rp.p;
    const int* ci = H.lev[l].ci.p;
    const double* v = H.lev[l].v.p;
    Strength S;
    strength_graph(h, n, nnz, rp, ci, v, o.amg_theta, S);
    Level& L = H.lev[l];
    // Newton-loop reuse: the level keeps the C/F split of the earlier set-up
    const bool frozen = frozen_cf && l < (int)frozen_cf->size() &&
                        (*frozen_cf)[l].p != nullptr && (*frozen_cf)[l].n == (size_t)n;
    if (frozen) {
      L.cf = std::move((*frozen_cf)[l]);
    } else {
      pc.mark(1);
      pmis_split(h, n, S, o.seed, l, L.cf);
      pc.mark(2);
    }
    DBuf<int> cidx(h, n + 1);
    exclusive_scan(h, L.cf.p, cidx.p, n);
    // the interpolation is formed before the coarse size is known (one
    // read-back for both); a split with no C point or no F point makes no
    // level, and its P is dropped
    int nc = 0;
    L.nnzP = classical_interp(h, n, nnz, rp, ci, v, S.strong.p, L.cf.p, cidx.p,
                              o.interp_max_elems, L.prp, L.pci, L.pv, cidx.p + n, &nc);
    if (nc == 0 || nc == n) {     // coarsening stalled: this level is the coarsest
      L.cf.release();
      L.prp.release();
      L.pci.release();
      L.pv.release();
      L.nnzP = 0;
      break;
    }
    L.nc = nc;
    if (learned && l == 0) {
      // learned weights on classical interpolation's pattern (level 0 only)
      std::unique_ptr<GnnGraph, void (*)(GnnGraph*)> g(
          gnn_create(h, n, rp, ci, v, L.cf.p, L.prp.p, L.pci.p, L.pv.p, nnz), gnn_destroy);
      gnn_apply_to_p(g.get(), learned, L.pv.p);
    }
    pc.mark(3);
    transpose(h, n, nc, L.prp.p, L.pci.p, L.pv.p, L.nnzP, L.rrp, L.rci, &L.rv);
    pc.mark(4);
    // Galerkin product A_c = R (A P)
    DBuf<int> aprp, apci;
    DBuf<double> apv;
    int apnnz = 0;
    sparse_product(h, n, rp, ci, v, L.prp.p, L.pci.p, L.pv.p, aprp, apci, apv, apnnz);
    Level next;
    next.n = nc;
    sparse_product(h, nc, L.rrp.p, L.rci.p, L.rv.p, aprp.p, apci.p, apv.p, next.rp, next.ci,
                   next.v, next.nnz);
    H.lev.push_back(std::move(next));
    pc.mark(5);
  }
  pc.mark(0);
  coarse_inverse(h, H);
  pc.mark(6);
  if (o.smoother == MSS_MCSGS)   // the coarsest level is solved directly, not smoothed
    for (size_t l = 0; l + 1 < H.lev.size(); ++l) level_colours(h, H.lev[l]);
}

// System AMG of the 2 x 2 block B_ee for CPTR (Sec. 4.2, Eq. CPTRM1): nodal
// coarsening (PMIS on the Frobenius norms of the blocks), classical
// interpolation per unknown on the common split, P interleaved without
// cross-unknown weights, A_c = R (A P) on the scalar interleaved form, read
// back as 2 x 2 blocks for the next level. Levels are stored in the scalar
// interleaved form (n = 2 points), with each point's inverse diagonal block
// for the block Jacobi smoother and the split duplicated per unknown.
void amg_build_system(Handle* h, Hierarchy& H, int np0, int nnzb0, const int* rp0,
                      const int* ci0, const double* bv0) {
  const mss_options& o = h->opt;
  H.lev.clear();
  H.lev.reserve(32);
  H.bs = 2;
  int np = np0, nnzb = nnzb0;
  DBuf<int> brp(h, np + 1), bci(h, nnzb);
  DBuf<double> bv(h, (size_t)4 * nnzb);
  copy_dev(h, brp.p, rp0, sizeof(int) * ((size_t)np + 1));
  copy_dev(h, bci.p, ci0, sizeof(int) * (size_t)nnzb);
  copy_dev(h, bv.p, bv0, sizeof(double) * 4 * (size_t)nnzb);
  const int max_levels = o.amg_max_levels < 1 ? 1 : (o.amg_max_levels > 25 ? 25 : o.amg_max_levels);
  for (int l = 0;; ++l) {
    {
      Level L;
      L.n = 2 * np;
      L.nnz = 4 * nnzb;
      L.rp.reset(h, 2 * np + 1);
      L.ci.reset(h, L.nnz);
      L.v.reset(h, L.nnz);
      k_b2s<<<grid_for(2 * np, 128), 128, 0, h->stream>>>(np, brp.p, bci.p, bv.p, L.rp.p, L.ci.p,
                                                          L.v.p);
      MSS_LAUNCH_CK("k_b2s");
      L.dinv2.reset(h, (size_t)4 * np);
      DBuf<int> bad(h, 1);
      fill_int(h, bad.p, 0x7fffffff, 1);
      k_dinv2<<<grid_for(np, 256), 256, 0, h->stream>>>(np, brp.p, bci.p, bv.p, L.dinv2.p, bad.p);
      MSS_LAUNCH_CK("k_dinv2");
      const int b = read_int(h, bad.p);
      if (b != 0x7fffffff)
        fail(MSS_ERR_AMG, "system AMG level of " + std::to_string(np) +
                              " points: singular 2 x 2 diagonal block at point " +
                              std::to_string(b));
      H.lev.push_back(std::move(L));
    }
    level_prepare(h, H.lev[l]);
    if (np <= o.amg_max_coarse || l + 1 >= max_levels) break;
    // nodal coarsening
    DBuf<double> nv(h, nnzb);
    k_block_norm<<<grid_for(np, 128), 128, 0, h->stream>>>(np, brp.p, bci.p, bv.p, nv.p);
    MSS_LAUNCH_CK("k_block_norm");
    DBuf<int> cfp;
    {
      Strength Sn;
      strength_graph(h, np, nnzb, brp.p, bci.p, nv.p, o.amg_theta, Sn);
      pmis_split(h, np, Sn, o.seed, l, cfp);
    }
    DBuf<int> cidx(h, np + 1);
    exclusive_scan(h, cfp.p, cidx.p, np);
    const int ncp = read_int(h, cidx.p + np);
    if (ncp == 0 || ncp == np) break;   // coarsening stalled: this level is the coarsest
    // classical interpolation per unknown on the common split
    DBuf<int> prpk[2], pcik[2];
    DBuf<double> pvk[2];
    for (int k = 0; k < 2; ++k) {
      DBuf<double> vk(h, nnzb);
      k_block_entry<<<grid_for(nnzb, 256), 256, 0, h->stream>>>(nnzb, bv.p, 3 * k, vk.p);
      MSS_LAUNCH_CK("k_block_entry");
      DBuf<unsigned char> sk(h, nnzb);
      DBuf<int> scount(h, np);
      k_strength<<<grid_for(np, 128), 128, 0, h->stream>>>(np, brp.p, bci.p, vk.p, o.amg_theta,
                                                           sk.p, scount.p);
      MSS_LAUNCH_CK("k_strength");
      classical_interp(h, np, nnzb, brp.p, bci.p, vk.p, sk.p, cfp.p, cidx.p, o.interp_max_elems,
                       prpk[k], pcik[k], pvk[k]);
    }
    Level& L = H.lev[l];
    L.nc = 2 * ncp;
    L.cf.reset(h, 2 * np);
    k_dup2<<<grid_for(2 * np, 256), 256, 0, h->stream>>>(np, cfp.p, L.cf.p);
    MSS_LAUNCH_CK("k_dup2");
    {
      DBuf<int> plen(h, 2 * np);
      k_p2_len<<<grid_for(2 * np, 256), 256, 0, h->stream>>>(np, prpk[0].p, prpk[1].p, plen.p);
      MSS_LAUNCH_CK("k_p2_len");
      L.prp.reset(h, 2 * np + 1);
      exclusive_scan(h, plen.p, L.prp.p, 2 * np);
      L.nnzP = read_int(h, L.prp.p + 2 * np);
      L.pci.reset(h, L.nnzP > 0 ? L.nnzP : 1);
      L.pv.reset(h, L.nnzP > 0 ? L.nnzP : 1);
      k_p2_fill<<<grid_for(2 * np, 128), 128, 0, h->stream>>>(
          np, prpk[0].p, pcik[0].p, pvk[0].p, prpk[1].p, pcik[1].p, pvk[1].p, L.prp.p, L.pci.p,
          L.pv.p);
      MSS_LAUNCH_CK("k_p2_fill");
    }
    transpose(h, 2 * np, 2 * ncp, L.prp.p, L.pci.p, L.pv.p, L.nnzP, L.rrp, L.rci, &L.rv);
    // Galerkin product on the scalar interleaved form, then its blocks
    DBuf<int> aprp, apci, acrp, acci;
    DBuf<double> apv, acv;
    int apnnz = 0, acnnz = 0;
    sparse_product(h, 2 * np, L.rp.p, L.ci.p, L.v.p, L.prp.p, L.pci.p, L.pv.p, aprp, apci, apv,
                   apnnz);
    sparse_product(h, 2 * ncp, L.rrp.p, L.rci.p, L.rv.p, aprp.p, apci.p, apv.p, acrp, acci, acv,
                   acnnz);
    DBuf<int> cnt(h, ncp), nrp(h, ncp + 1);
    k_s2b<<<grid_for(ncp, 128), 128, 0, h->stream>>>(ncp, acrp.p, acci.p, acv.p, cnt.p, nullptr,
                                                     nullptr, nullptr, 0);
    MSS_LAUNCH_CK("k_s2b");
    exclusive_scan(h, cnt.p, nrp.p, ncp);
    const int nnzb_c = read_int(h, nrp.p + ncp);
    DBuf<int> nci(h, nnzb_c > 0 ? nnzb_c : 1);
    DBuf<double> nbv(h, (size_t)4 * (nnzb_c > 0 ? nnzb_c : 1));
    fill_double(h, nbv.p, 0.0, (long long)4 * nnzb_c);
    k_s2b<<<grid_for(ncp, 128), 128, 0, h->stream>>>(ncp, acrp.p, acci.p, acv.p, nullptr, nrp.p,
                                                     nci.p, nbv.p, 1);
    MSS_LAUNCH_CK("k_s2b");
    brp = std::move(nrp);
    bci = std::move(nci);
    bv = std::move(nbv);
    np = ncp;
    nnzb = nnzb_c;
  }
  coarse_inverse(h, H);
}

}  // namespace mss
