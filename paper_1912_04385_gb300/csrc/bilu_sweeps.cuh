// bilu_sweeps.cuh -- the forward and backward sweeps of the strip-coloured
// block ILU(0) last stage (Algorithm 2, last stage), as device bodies that take
// the warp index of their launch: the one-system kernels of bilu.cu pass
// (blockIdx.x * blockDim.x + threadIdx.x) / 32, the multi-system tile walker
// of the batched solve (fused.cu) the same index within the system's own
// launch shape, so both compute the same values.
#pragma once

#include "common.cuh"

namespace mss {
namespace dev {

// Programmatic dependent launch: a sweep kernel launched with the
// programmatic-serialization attribute may start while the previous kernel of
// its stream still runs. pdl_wait() blocks until that kernel has completed and
// its writes are visible (it returns at once in a kernel launched without
// the attribute); pdl_trigger(), issued only after the wait, lets the next
// such kernel start, so that what a kernel reads before its own wait is never
// newer than its predecessor's predecessor.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ int warp_max(int v) {
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// ---- sweeps ----------------------------------------------------------------
// Each sweep of one colour is split in two launches: a fully parallel pass
// (NB lanes per row) that does all the work coupling the row to other strips
// (earlier colours in the forward sweep, later colours in the backward
// sweep), and a chain pass (NB lanes per strip, rows in order) that adds the
// couplings inside the strip; the value of the neighbouring row in the strip
// is forwarded in registers.
//
// forward, parallel: w_q = u_q - sum_{other-strip lower} L_qk w_k, with
// u = r - Abar[:,t] x_T - Abar[:,p] v_P (MODE bit 1: x_T term, bit 2: v_P)
template <int NB, int MODE, class V, class C>
__device__ __forceinline__ void fwd_par(long long warp, int q0, int q1,
                                        const int* __restrict__ perm, const int* __restrict__ frp,
                                        const int* __restrict__ fslo, const int* __restrict__ fpos,
                                        const int* __restrict__ fcell, const V* __restrict__ fv,
                                        const C* __restrict__ fcs, const double* __restrict__ r,
                                        const C* __restrict__ xT, const C* __restrict__ vP,
                                        C* __restrict__ w, int lower, int wait_first) {
  constexpr int RPW = 32 / NB;
  constexpr int B2 = NB * NB;
  const int lane = threadIdx.x & 31;
  const int sub = lane / NB, comp = lane - sub * NB;
  const long long qq = q0 + warp * RPW + sub;
  if (sub >= RPW || qq >= q1) return;
  const int q = (int)qq;
  const int cell = perm[q];
  // the u terms read r and the earlier stages' results, which only the
  // first colour's predecessor may still be writing (wait_first)
  if (wait_first) pdl_wait();
  C acc = (C)r[(size_t)cell * NB + comp];
  const int b = frp[q], e = frp[q + 1];
  if (MODE) {
    for (int f = b; f < e; ++f) {
      const int j = fcell[f];
      const C* cs = fcs + (size_t)f * 2 * NB;
      if (MODE & 1) acc -= cs[comp] * xT[j];
      if (MODE & 2) acc -= cs[NB + comp] * vP[j];
    }
  }
  if (!wait_first) pdl_wait();
  pdl_trigger();
  if (lower) {
    const int d = fslo[q];
    for (int f = b; f < d; ++f) {
      const V* Lr = fv + (size_t)f * B2 + comp * NB;
      const C* wk = w + (size_t)fpos[f] * NB;
#pragma unroll
      for (int c = 0; c < NB; ++c) acc -= cvt<C>(Lr[c]) * wk[c];
    }
  }
  w[(size_t)q * NB + comp] = acc;
}

// forward, chain: w_q -= sum_{in-strip lower} L_qk w_k, rows in order. The
// coupling to the previous row comes from the dense per-position copy cL and
// the previous row's values held in the lanes' registers. Two rows are held
// in registers; at each step the row's values are taken and its register row
// is refilled two rows ahead before the step's dependent work, with
// addresses as offsets from the strip's first row (fewer instructions than
// per-row 64-bit addressing; the chains are 18-20 % shorter than with a ring
// of rows addressed by position; 4 and 8 rows ahead measured no faster). The
// previous row's values pass through shuffles, so a step has no warp barrier;
// only a row with other in-strip couplings, read from memory, first
// synchronises the strip's lanes. The backward chain does the same in reverse.
// Chain passes have few warps (32 / NB strips each) and are bound by the FP64
// pipe of the SMs they run on: two-warp CTAs spread them over all SMs.
constexpr int kChainThreads = 64;
constexpr int kChainRows = 2;     // rows of a chain held in registers (the refill distance)

template <int NB, class V, class C>
__device__ __forceinline__ void fwd_chain(long long warp, int s0, int s1,
                                          const int* __restrict__ st_first,
                                          const int* __restrict__ st_len,
                                          const int* __restrict__ fslo, const int* __restrict__ fdp,
                                          const int* __restrict__ fpos, const V* __restrict__ fv,
                                          const V* __restrict__ cL, const int* __restrict__ cflag,
                                          C* __restrict__ w) {
  constexpr int RPW = 32 / NB;
  constexpr int B2 = NB * NB;
  const int lane = threadIdx.x & 31;
  const int sub = lane / NB, comp = lane - sub * NB;
  const long long kk = s0 + warp * RPW + sub;
  const bool active = sub < RPW && kk < s1;
  const int first = active ? st_first[kk] : 0;
  const int len = active ? st_len[kk] : 0;
  const int maxlen = warp_max(len);
  const int base = sub * NB;
  const unsigned gmask = ((1u << NB) - 1u) << base;   // the strip's lanes
  // the strip's rows for this lane: t at wl[i * NB], the chain row at
  // ml[i * B2 + c], the flag at fl[i]; two rows held in registers (even and
  // odd steps), each refilled two rows ahead right after its use
  C* wl = w + (size_t)first * NB + comp;
  const V* ml = cL + (size_t)first * B2 + comp * NB;
  const int* fl = cflag + first;
  constexpr int D = kChainRows;
  C tq[D], mq[D][NB];
  int fq[D];
#pragma unroll
  for (int u = 0; u < D; ++u) {
    tq[u] = 0;
    fq[u] = 0;
#pragma unroll
    for (int c = 0; c < NB; ++c) mq[u][c] = 0;
    if (u < len) {
      fq[u] = fl[u];
#pragma unroll
      for (int c = 0; c < NB; ++c) mq[u][c] = cvt<C>(ml[u * B2 + c]);
    }
  }
  // the factor data above; w only after the previous sweep kernel
  pdl_wait();
#pragma unroll
  for (int u = 0; u < D; ++u)
    if (u < len) tq[u] = wl[u * NB];
  pdl_trigger();
  C prev = 0;                               // component comp of w_{q-1}
  auto step = [&](int it, C& t, C (&m)[NB], int& f) {
    // this row's values, then the refill two rows ahead is issued before the
    // step's dependent work
    const C tc = t;
    C mc[NB];
#pragma unroll
    for (int c = 0; c < NB; ++c) mc[c] = m[c];
    const int fc = f;
    if (it + D < len) {
      t = wl[(it + D) * NB];
      f = fl[it + D];
#pragma unroll
      for (int c = 0; c < NB; ++c) m[c] = cvt<C>(ml[(it + D) * B2 + c]);
    }
    C pc[NB];
#pragma unroll
    for (int c = 0; c < NB; ++c) pc[c] = __shfl_sync(0xffffffffu, prev, (base + c) & 31);
    if (it < len) {
      C acc = tc;
#pragma unroll
      for (int c = 0; c < NB; ++c) acc -= mc[c] * pc[c];
      if (fc & 1) {                          // other in-strip couplings, from memory
        __syncwarp(gmask);                   // rows written by the strip's other lanes
        const int q = first + it;
        for (int g = fslo[q]; g < fdp[q]; ++g) {
          const V* Lr = fv + (size_t)g * B2 + comp * NB;
          const C* wk = w + (size_t)fpos[g] * NB;
#pragma unroll
          for (int c = 0; c < NB; ++c) acc -= cvt<C>(Lr[c]) * wk[c];
        }
      }
      wl[it * NB] = acc;
      prev = acc;
    }
  };
  for (int it = 0; it < maxlen; it += D) {
#pragma unroll
    for (int u = 0; u < D; ++u)
      if (it + u < maxlen) step(it + u, tq[u], mq[u], fq[u]);
  }
}

// backward, parallel: s_q = U_qq^{-1} (w_q - sum_{other-strip upper} U_qj x_j)
// (later colours, final); stored back into w
template <int NB, class V, class C>
__device__ __forceinline__ void bwd_par(long long warp, int q0, int q1,
                                        const int* __restrict__ frp, const int* __restrict__ fshi,
                                        const int* __restrict__ fpos,
                                        const V* __restrict__ fv, const V* __restrict__ fdinv,
                                        C* __restrict__ w) {
  constexpr int RPW = 32 / NB;
  constexpr int B2 = NB * NB;
  const int lane = threadIdx.x & 31;
  const int sub = lane / NB, comp = lane - sub * NB;
  const long long qq = q0 + warp * RPW + sub;
  const bool on = sub < RPW && qq < q1;
  const int q = on ? (int)qq : q0;
  pdl_wait();
  pdl_trigger();
  C acc = 0;
  if (on) {
    acc = w[(size_t)q * NB + comp];
    for (int g = fshi[q]; g < frp[q + 1]; ++g) {
      const V* Ur = fv + (size_t)g * B2 + comp * NB;
      const C* xj = w + (size_t)fpos[g] * NB;
#pragma unroll
      for (int c = 0; c < NB; ++c) acc -= cvt<C>(Ur[c]) * xj[c];
    }
  }
  const int base = sub * NB;
  const V* Ui = fdinv + (size_t)q * B2 + comp * NB;
  C s = 0;
#pragma unroll
  for (int c = 0; c < NB; ++c) {
    C tc = __shfl_sync(0xffffffffu, acc, (base + c) & 31);
    if (on) s += cvt<C>(Ui[c]) * tc;
  }
  if (on) w[(size_t)q * NB + comp] = s;
}

// backward, chain: x_q = s_q - sum_{in-strip upper} G_qj x_j, rows of a
// strip in reverse order (cG and the next row's values in registers, rows
// fetched two steps ahead as in the forward chain); x_q goes back into w.
// Block Jacobi (upper = 0): x_q = D_qq^{-1} u_q. Each final row also goes to
// the output y = x + v + M3 u in cell order.
template <int NB, class V, class C>
__device__ __forceinline__ void bwd_chain(long long warp, int s0, int s1,
                                          const int* __restrict__ st_first,
                                          const int* __restrict__ st_len,
                                          const int* __restrict__ fdp, const int* __restrict__ fshi,
                                          const int* __restrict__ fpos, const V* __restrict__ fv,
                                          const V* __restrict__ fdinv, const V* __restrict__ cG,
                                          const int* __restrict__ cflag, C* __restrict__ w,
                                          int upper, const int* __restrict__ perm,
                                          const C* __restrict__ xT, const C* __restrict__ vP, int p,
                                          int t, double* __restrict__ y) {
  constexpr int RPW = 32 / NB;
  constexpr int B2 = NB * NB;
  const int lane = threadIdx.x & 31;
  const int sub = lane / NB, comp = lane - sub * NB;
  // a row's values are final once its step is done: y = x + v + M3 u in cell
  // order, y_cell = w_q (+ x_T at t, + v_P at p)
  auto emit = [&](int q, C val) {
    const int cell = perm[q];
    C out = val;
    if (xT && comp == t) out += xT[cell];
    if (vP && comp == p) out += vP[cell];
    y[(size_t)cell * NB + comp] = (double)out;
  };
  const long long kk = s0 + warp * RPW + sub;
  const bool active = sub < RPW && kk < s1;
  const int first = active ? st_first[kk] : 0;
  const int len = active ? st_len[kk] : 0;
  const int maxlen = warp_max(len);
  const int base = sub * NB;
  const unsigned gmask = ((1u << NB) - 1u) << base;   // the strip's lanes
  if (!upper) {
    pdl_wait();
    pdl_trigger();
    for (int it = 0; it < maxlen; ++it) {
      const bool on = it < len;
      const int q = on ? first + it : 0;
      const C tv = on ? w[(size_t)q * NB + comp] : (C)0;
      const V* Ui = fdinv + (size_t)q * B2 + comp * NB;
      C x = 0;
#pragma unroll
      for (int c = 0; c < NB; ++c) {
        C tc = __shfl_sync(0xffffffffu, tv, (base + c) & 31);
        if (on) x += cvt<C>(Ui[c]) * tc;
      }
      if (on) {
        w[(size_t)q * NB + comp] = x;
        emit(q, x);
      }
    }
    return;
  }
  // the strip's rows for this lane in reverse: row r = len - 1 - it, its s
  // at wl[r * NB], the chain block row at gl[r * B2 + c], the flag at fl[r];
  // two rows held in registers, each refilled two rows ahead after its use
  C* wl = w + (size_t)first * NB + comp;
  const V* gl = cG + (size_t)first * B2 + comp * NB;
  const int* fl = cflag + first;
  constexpr int D = kChainRows;
  C tq[D], mq[D][NB];
  int fq[D];
#pragma unroll
  for (int u = 0; u < D; ++u) {
    tq[u] = 0;
    fq[u] = 0;
#pragma unroll
    for (int c = 0; c < NB; ++c) mq[u][c] = 0;
    if (u < len) {
      const int r = len - 1 - u;
      fq[u] = fl[r];
#pragma unroll
      for (int c = 0; c < NB; ++c) mq[u][c] = cvt<C>(gl[r * B2 + c]);
    }
  }
  pdl_wait();
#pragma unroll
  for (int u = 0; u < D; ++u)
    if (u < len) tq[u] = wl[(len - 1 - u) * NB];
  pdl_trigger();
  C nxt = 0;                                // component comp of x_{q+1}
  auto step = [&](int it, C& t, C (&m)[NB], int& f) {
    const int r = len - 1 - it;
    // this row's values, then the refill two rows ahead is issued before the
    // step's dependent work
    const C tc = t;
    C mc[NB];
#pragma unroll
    for (int c = 0; c < NB; ++c) mc[c] = m[c];
    const int fc = f;
    if (it + D < len) {
      t = wl[(r - D) * NB];
      f = fl[r - D];
#pragma unroll
      for (int c = 0; c < NB; ++c) m[c] = cvt<C>(gl[(r - D) * B2 + c]);
    }
    C nc[NB];
#pragma unroll
    for (int c = 0; c < NB; ++c) nc[c] = __shfl_sync(0xffffffffu, nxt, (base + c) & 31);
    if (it < len) {
      C x = tc;                              // s_q from the parallel pass
#pragma unroll
      for (int c = 0; c < NB; ++c) x -= mc[c] * nc[c];
      if (fc & 2) {                          // other in-strip couplings, from memory
        __syncwarp(gmask);                   // rows written by the strip's other lanes
        const int q = first + r;
        for (int g = fdp[q] + 1; g < fshi[q]; ++g) {
          const V* Gr = fv + (size_t)g * B2 + comp * NB;
          const C* xj = w + (size_t)fpos[g] * NB;
#pragma unroll
          for (int c = 0; c < NB; ++c) x -= cvt<C>(Gr[c]) * xj[c];
        }
      }
      wl[r * NB] = x;
      emit(first + r, x);
      nxt = x;
    }
  };
  for (int it = 0; it < maxlen; it += D) {
#pragma unroll
    for (int u = 0; u < D; ++u)
      if (it + u < maxlen) step(it + u, tq[u], mq[u], fq[u]);
  }
}

}  // namespace dev
}  // namespace mss
