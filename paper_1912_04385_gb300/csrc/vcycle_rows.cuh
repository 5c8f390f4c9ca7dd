// vcycle_rows.cuh -- row operations of the AMG V-cycle (Sec. 5.1), shared by
// the per-level kernels and the fused coarse-level kernel of amg_cycle.cu and
// by the multi-system tile walker of the batched solve (fused.cu), so that all
// of them give the same values.
#pragma once

#include "common.cuh"

namespace mss {
namespace dev {

// LD reads the vectors: plain loads in the per-level kernels; in the fused
// kernel, whose blocks read what other blocks wrote before a grid barrier,
// loads that bypass the non-coherent L1.
struct LdPlain {
  template <class T>
  __device__ __forceinline__ static T ld(const T* p) { return *p; }
};
struct LdL2 {
  template <class T>
  __device__ __forceinline__ static T ld(const T* p) { return __ldcg(p); }
};

// Each operation takes the row's index m into the matrix arrays (rp, and
// dinv) and its index i into the vectors: the same row in the per-level
// kernels (m = i), a row of the block's copy of its rows in shared memory in
// the fused coarse-level kernel (m = i - first row of the block).

// x_out = x_in + omega D^-1 (b - A x_in)
template <class V, class C, class LD>
__device__ __forceinline__ void jacobi_row(int m, int i, const int* __restrict__ rp,
                                           const int* __restrict__ ci, const V* __restrict__ v,
                                           const C* __restrict__ dinv, const C* b, C omega,
                                           const C* xin, C* xout) {
  C s = 0;
  for (int k = rp[m]; k < rp[m + 1]; ++k) s += cvt<C>(v[k]) * LD::ld(xin + ci[k]);
  xout[i] = LD::ld(xin + i) + omega * (dinv[m] * (LD::ld(b + i) - s));
}

// r = b - A x
template <class V, class C, class LD>
__device__ __forceinline__ void residual_row(int m, int i, const int* __restrict__ rp,
                                             const int* __restrict__ ci,
                                             const V* __restrict__ v, const C* b, const C* x,
                                             C* r) {
  C s = 0;
  for (int k = rp[m]; k < rp[m + 1]; ++k) s += cvt<C>(v[k]) * LD::ld(x + ci[k]);
  r[i] = LD::ld(b + i) - s;
}

// b = R r on the next level and, with x1, that level's first Jacobi sweep
// from zero x1 = omega D^-1 b (the expression the sweep kernels use; dinv is
// the next level's, indexed like rp)
template <class V, class C, class LD>
__device__ __forceinline__ void restrict_row(int m, int i, const int* __restrict__ rp,
                                             const int* __restrict__ ci,
                                             const V* __restrict__ v, const C* r, C* b,
                                             const C* __restrict__ dinv, C omega, C* x1) {
  C s = 0;
  for (int k = rp[m]; k < rp[m + 1]; ++k) s += cvt<C>(v[k]) * LD::ld(r + ci[k]);
  b[i] = s;
  if (x1) x1[i] = omega * dinv[m] * s;
}

// xout = x + P xc (x and xout may be the same vector: each entry is read
// and written by its own thread only)
template <class V, class C, class LD>
__device__ __forceinline__ void prolong_row(int m, int i, const int* __restrict__ rp,
                                            const int* __restrict__ ci,
                                            const V* __restrict__ v, const C* xc, const C* x,
                                            C* xout) {
  C s = 0;
  for (int k = rp[m]; k < rp[m + 1]; ++k) s += cvt<C>(v[k]) * LD::ld(xc + ci[k]);
  xout[i] = LD::ld(x + i) + s;
}

// (Ainv b) for the row a of the dense inverse by one warp: lanes over the
// row, then a tree
template <class C, class LD>
__device__ __forceinline__ C gemv_row(const C* __restrict__ a, int lane, int n, const C* b) {
  C s = 0;
  for (int j = lane; j < n; j += 32) s += a[j] * LD::ld(b + j);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  return s;
}

// b = v[:, var] (the stage's right-hand side) and, with x1, the first
// Jacobi sweep from zero x1 = omega D^-1 b
template <class C>
__device__ __forceinline__ void gather_var_row(int i, int N, int nb, const double* __restrict__ v,
                                               int var, C* __restrict__ out,
                                               const C* __restrict__ dinv, C omega,
                                               C* __restrict__ x1) {
  if (i >= N) return;
  const C bi = (C)v[(size_t)i * nb + var];
  out[i] = bi;
  if (x1) x1[i] = omega * dinv[i] * bi;
}

// out_i = r[i*nb + var] - sum_j vals_ij x_j over the block pattern (and the
// next stage's first sweep from zero, as above)
template <class C>
__device__ __forceinline__ void pattern_sub_row(int i, int N, int nb, const int* __restrict__ rp,
                                                const int* __restrict__ ci,
                                                const C* __restrict__ vals,
                                                const C* __restrict__ x,
                                                const double* __restrict__ r, int var,
                                                C* __restrict__ out, const C* __restrict__ dinv,
                                                C omega, C* __restrict__ x1) {
  if (i >= N) return;
  C s = 0;
  for (int k = rp[i]; k < rp[i + 1]; ++k) s += vals[k] * x[ci[k]];
  const C bi = (C)r[(size_t)i * nb + var] - s;
  out[i] = bi;
  if (x1) x1[i] = omega * dinv[i] * bi;
}

}  // namespace dev
}  // namespace mss
