// spmv.cu -- y = Abar x on the scaled cell-blocked matrix, the operator
// FGMRES iterates with (Sec. 4, Eq. splitPrec1; Sec. 5.1). Kept in a file of
// its own: the kernel's ncu counters are tied to this source.
#include "common.cuh"
#include "vec_rows.cuh"

namespace mss {
namespace {

// y = Abar x, NB lanes per block row (lane c produces component c)
template <int NB>
__global__ void k_bsr_spmv(int N, const int* __restrict__ rp, const int* __restrict__ ci,
                           const double* __restrict__ vals, const double* __restrict__ x,
                           double* __restrict__ y) {
  dev::bsr_spmv_rows<NB>(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5, N, rp, ci, vals,
                         x, y);
}

template <int NB>
void spmv_nb(Handle* h, const double* x, double* y) {
  constexpr int RPW = 32 / NB;
  long long warps = (h->N + RPW - 1) / RPW;
  k_bsr_spmv<NB><<<grid_for(warps * 32, h->tb), h->tb, 0, h->stream>>>(h->N, h->rp.p, h->ci.p,
                                                                   h->abar.p, x, y);
  MSS_LAUNCH_CK("k_bsr_spmv");
}

}  // namespace

void bsr_spmv(Handle* h, const double* x, double* y) {
  TraceScope ts(h, TR_SPMV);
  MSS_NB_DISPATCH(h->nb, spmv_nb<NB>(h, x, y));
}

}  // namespace mss
