// residual.cu -- residual check of a BSR system for a given x:
// ||b - J x||_2 and ||b||_2 (the unscaled true residual a caller checks
// after a solve; the solver itself stops on the scaled system, Sec. 5.1).
//
// Two kernels: per-cell partial sums of squares into a scratch array of 2N
// doubles, then one block reduces them in a fixed order, so the result does
// not depend on the launch shape.
#include "common.cuh"

namespace mss {

namespace {

constexpr int RT = 256;

// scratch[i] = sum_k (b - J x)_{i,k}^2, scratch[N + i] = sum_k b_{i,k}^2;
// NB lanes per block row, lane c owns component c
template <int NB>
__global__ void k_cell_residual_sq(int N, const int* __restrict__ rp,
                                   const int* __restrict__ ci, const double* __restrict__ vals,
                                   const double* __restrict__ b, const double* __restrict__ x,
                                   double* __restrict__ scratch) {
  constexpr int RPW = 32 / NB;
  constexpr int B2 = NB * NB;
  const int lane = threadIdx.x & 31;
  const int sub = lane / NB, comp = lane - sub * NB;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long ii = warp * RPW + sub;
  const bool on = sub < RPW && ii < N;
  const int i = on ? (int)ii : 0;
  double r2 = 0.0, b2 = 0.0;
  if (on) {
    double acc = 0.0;
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
      const double* a = vals + (size_t)e * B2 + comp * NB;
      const double* xj = x + (size_t)ci[e] * NB;
#pragma unroll
      for (int c = 0; c < NB; ++c) acc += a[c] * xj[c];
    }
    const double bi = b[(size_t)i * NB + comp];
    const double ri = bi - acc;
    r2 = ri * ri;
    b2 = bi * bi;
  }
  // sum over the NB lanes of the row, in component order
  const int base = sub * NB;
  double sr = 0.0, sb = 0.0;
#pragma unroll
  for (int c = 0; c < NB; ++c) {
    sr += __shfl_sync(0xffffffffu, r2, (base + c) & 31);
    sb += __shfl_sync(0xffffffffu, b2, (base + c) & 31);
  }
  if (on && comp == 0) {
    scratch[i] = sr;
    scratch[(size_t)N + i] = sb;
  }
}

// norms[0] = sqrt(sum scratch[0..N)), norms[1] = sqrt(sum scratch[N..2N));
// one block: thread t sums a contiguous chunk, then a fixed tree
__global__ void k_reduce_cells(int N, const double* __restrict__ scratch,
                               double* __restrict__ norms) {
  __shared__ double sr[RT], sb[RT];
  const int t = threadIdx.x;
  const long long chunk = ((long long)N + RT - 1) / RT;
  const long long lo = t * chunk, hi = lo + chunk < N ? lo + chunk : N;
  double a = 0.0, c = 0.0;
  for (long long k = lo; k < hi; ++k) {
    a += scratch[k];
    c += scratch[(size_t)N + k];
  }
  sr[t] = a;
  sb[t] = c;
  __syncthreads();
  for (int s = RT / 2; s > 0; s >>= 1) {
    if (t < s) {
      sr[t] += sr[t + s];
      sb[t] += sb[t + s];
    }
    __syncthreads();
  }
  if (t == 0) {
    norms[0] = sqrt(sr[0]);
    norms[1] = sqrt(sb[0]);
  }
}

template <int NB>
void launch_residual(cudaStream_t s, const mss_bsr* J, const double* b, const double* x,
                     double* scratch, double* norms) {
  constexpr int RPW = 32 / NB;
  const long long warps = ((long long)J->n_rows + RPW - 1) / RPW;
  k_cell_residual_sq<NB><<<grid_for(warps * 32, RT), RT, 0, s>>>(J->n_rows, J->row_ptr,
                                                                 J->col_idx, J->vals, b, x,
                                                                 scratch);
  MSS_LAUNCH_CK("k_cell_residual_sq");
  k_reduce_cells<<<1, RT, 0, s>>>(J->n_rows, scratch, norms);
  MSS_LAUNCH_CK("k_reduce_cells");
}

}  // namespace

void check_residual_args(const mss_bsr* J, int nb, const double* b, const double* x,
                         const double* norms) {
  if (!J || !J->row_ptr || !J->col_idx || !J->vals || !b || !x || !norms)
    fail(MSS_ERR_INVALID_ARG, "null pointer");
  if (J->n_rows < 1 || J->nnzb < J->n_rows) fail(MSS_ERR_INVALID_ARG, "bad matrix sizes");
  if (nb < 2 || nb > MSS_MAX_NB) fail(MSS_ERR_INVALID_ARG, "nb must be in [2, 16]");
}

void residual_norms(cudaStream_t s, const mss_bsr* J, int nb, const double* b, const double* x,
                    double* scratch, double* norms) {
  MSS_NB_DISPATCH(nb, launch_residual<NB>(s, J, b, x, scratch, norms));
}

void residual_norm(Handle* h, const mss_bsr* J, int nb, const double* b, const double* x,
                   double* norms) {
  check_residual_args(J, nb, b, x, norms);
  DBuf<double> scratch(h, 2 * (size_t)J->n_rows);
  residual_norms(h->stream, J, nb, b, x, scratch.p, norms);
}

}  // namespace mss
