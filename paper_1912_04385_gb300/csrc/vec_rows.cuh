// vec_rows.cuh -- device bodies of the block matrix-vector product y = Abar x
// (Sec. 4, Eq. splitPrec1) and of the right-hand-side scaling bbar = N^{-1} b
// (Eqs. CPR, CPTR31/32), shared by the one-system kernels (spmv.cu,
// setup_scale.cu) and the multi-system tile walker of the batched solve
// (fused.cu).
#pragma once

#include "common.cuh"

namespace mss {
namespace dev {

// y = Abar x for the rows of one warp: NB lanes per block row (lane c
// produces component c), 32 / NB rows per warp
template <int NB>
__device__ __forceinline__ void bsr_spmv_rows(long long warp, int N, const int* __restrict__ rp,
                                              const int* __restrict__ ci,
                                              const double* __restrict__ vals,
                                              const double* __restrict__ x,
                                              double* __restrict__ y) {
  constexpr int RPW = 32 / NB;
  constexpr int B2 = NB * NB;
  const int lane = threadIdx.x & 31;
  const int sub = lane / NB, comp = lane - sub * NB;
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

// entry tid = i * NB + r of bbar: row r of W_i b_i on the scaled rows (p, and
// t for CPTR3 / CPTR), a copy elsewhere; explicit fused multiply-adds
template <int NB>
__device__ __forceinline__ void scale_vec_entry(long long tid, const double* __restrict__ b, int N,
                                                int p, int t, int scheme,
                                                const double* __restrict__ wrows,
                                                double* __restrict__ out) {
  if (tid >= (long long)N * NB) return;
  int i = (int)(tid / NB), r = (int)(tid % NB);
  bool scaled_row = scheme != 2 && (r == p || ((scheme == 0 || scheme == 3) && r == t));
  if (!scaled_row) {
    out[tid] = b[tid];
    return;
  }
  const double* w = wrows + (size_t)i * 2 * NB + (r == p ? 0 : NB);
  double acc = 0.0;
  for (int k = 0; k < NB; ++k) acc = fma(w[k], b[(size_t)i * NB + k], acc);
  out[tid] = acc;
}

}  // namespace dev
}  // namespace mss
