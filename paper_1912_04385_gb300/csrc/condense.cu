// condense.cu -- static condensation of the secondary unknowns (Sec. 3, Eqs.
// global and reduced) and their recovery after the solve.
//
// The global system [J11 J12; J21 J22] [d1; d2] = -[r1; r2] has secondary
// unknowns coupled only inside their cell, so J12 and J22 are one block per
// cell and the Schur complement keeps the cell graph's pattern:
//   A_ij = J11_ij - T_i J21_ij,  b_i = -r1_i + T_i r2_i,  T_i = J12_i J22_i^{-1};
// afterwards d2_i = J22_i^{-1} (-r2_i - sum_j J21_ij d1_j).
//
// One warp per cell: the warp inverts J22_i by Gauss-Jordan without pivoting
// in its shared memory (Sec. 3 aligns the secondary equations so that the
// pivots are nonzero), forms T_i there, and streams the row's J11 and J21
// blocks once, lanes over the entries of each A block. Every block row is
// independent, so the kernel is a single pass over the inputs, bound by HBM.
#include "common.cuh"

namespace mss {
namespace {

constexpr int kCondWarps = 4;   // warps (cells) per CTA
constexpr int kRecoverRow = 64; // blocks per row the recovery accepts (a cell's neighbours)

__device__ __forceinline__ bool row_ok(const int* rp, int i, int nnzb) {
  const int b = rp[i], e = rp[i + 1];
  return b >= 0 && e >= b && e <= nnzb;
}

// Gauss-Jordan on the warp's n x (n + m) augmented matrix M (row-major, in
// shared memory), no pivoting: afterwards the right part holds the left
// part's inverse times the original right part. Returns false on a zero or
// non-finite pivot (the same decision in every lane).
__device__ bool warp_gauss_jordan(double* M, int n, int m) {
  const int lane = threadIdx.x & 31;
  const int w = n + m;
  for (int k = 0; k < n; ++k) {
    const double piv = M[k * w + k];
    if (piv == 0.0 || !isfinite(piv)) return false;
    const double rpiv = 1.0 / piv;
    __syncwarp();
    for (int j = lane; j < w; j += 32) M[k * w + j] *= rpiv;
    __syncwarp();
    // column k is only read here (it is zeroed below), so the factors
    // M[i][k] stay the ones of this step while the lanes update the rows
    for (int idx = lane; idx < n * w; idx += 32) {
      const int i = idx / w, j = idx - i * w;
      if (i == k || j == k) continue;
      M[idx] -= M[i * w + k] * M[k * w + j];
    }
    __syncwarp();
    for (int i = lane; i < n; i += 32)
      if (i != k) M[i * w + k] = 0.0;
    __syncwarp();
  }
  return true;
}

__global__ void __launch_bounds__(32 * kCondWarps)
k_condense(int N, int nnzb, int n1, int n2, const int* __restrict__ rp,
           const double* __restrict__ j11, const double* __restrict__ j21,
           const double* __restrict__ j12, const double* __restrict__ j22,
           const double* __restrict__ r1, const double* __restrict__ r2, double* __restrict__ a,
           double* __restrict__ b, int* __restrict__ bad_row, int* __restrict__ bad_pivot) {
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int i = blockIdx.x * kCondWarps + wib;
  if (i >= N) return;                           // uniform per warp
  const int per = n2 * 2 * n2 + n1 * n2;        // doubles per warp
  double* M = smem + (size_t)wib * per;         // [J22 | I] -> [I | J22^-1]
  double* T = M + n2 * 2 * n2;                  // n1 x n2
  if (!row_ok(rp, i, nnzb)) {
    if (lane == 0) atomicMin(bad_row, i);
    return;
  }
  if (n2 > 0) {
    const double* D = j22 + (size_t)i * n2 * n2;
    for (int idx = lane; idx < n2 * 2 * n2; idx += 32) {
      const int r = idx / (2 * n2), c = idx - r * 2 * n2;
      M[idx] = c < n2 ? D[r * n2 + c] : (c - n2 == r ? 1.0 : 0.0);
    }
    __syncwarp();
    if (!warp_gauss_jordan(M, n2, n2)) {
      if (lane == 0) atomicMin(bad_pivot, i);
      return;
    }
    // T = J12_i J22_i^{-1}
    const double* B = j12 + (size_t)i * n1 * n2;
    for (int idx = lane; idx < n1 * n2; idx += 32) {
      const int r = idx / n2, c = idx - r * n2;
      double s = 0.0;
      for (int k = 0; k < n2; ++k) s += B[r * n2 + k] * M[k * 2 * n2 + n2 + c];
      T[idx] = s;
    }
    __syncwarp();
  }
  // b_i = -r1_i + T r2_i
  for (int r = lane; r < n1; r += 32) {
    double s = 0.0;
    for (int k = 0; k < n2; ++k) s += T[r * n2 + k] * r2[(size_t)i * n2 + k];
    b[(size_t)i * n1 + r] = -r1[(size_t)i * n1 + r] + s;
  }
  // A_ij = J11_ij - T J21_ij for every block of the row: the row's blocks
  // are contiguous, so the lanes run over all its entries at once (no lane
  // idles at the end of each block), each lane stepping its (block, row,
  // column) position without divisions
  const int e0 = rp[i], e1 = rp[i + 1];
  const int B2 = n1 * n1;
  const int len = (e1 - e0) * B2;
  const double* X = j11 + (size_t)e0 * B2;
  double* Z = a + (size_t)e0 * B2;
  int eb = 0, r = 0, c = lane;
  while (c >= n1) { c -= n1; ++r; }
  while (r >= n1) { r -= n1; ++eb; }
  const int dr = 32 / n1, dc = 32 - dr * n1;   // lane step 32 = dr rows + dc columns
  for (int t = lane; t < len; t += 32) {
    const double* Y = j21 + (size_t)(e0 + eb) * n2 * n1 + c;
    double s = 0.0;
    for (int k = 0; k < n2; ++k) s += T[r * n2 + k] * Y[k * n1];
    Z[t] = X[t] - s;
    c += dc;
    r += dr;
    if (c >= n1) { c -= n1; ++r; }
    while (r >= n1) { r -= n1; ++eb; }
  }
}

// d2_i = J22_i^{-1} (-r2_i - sum_j J21_ij d1_j): the right-hand side by warp
// sums over the row's (block, column) entries, then Gauss-Jordan on
// [J22_i | w] in shared memory.
__global__ void __launch_bounds__(32 * kCondWarps)
k_recover(int N, int nnzb, int n1, int n2, int maxrow, const int* __restrict__ rp,
          const int* __restrict__ ci, const double* __restrict__ j21,
          const double* __restrict__ j22, const double* __restrict__ r2,
          const double* __restrict__ d1, double* __restrict__ d2, int* __restrict__ bad_row,
          int* __restrict__ bad_pivot) {
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int i = blockIdx.x * kCondWarps + wib;
  if (i >= N) return;
  double* M = smem + (size_t)wib * (n2 * (n2 + 1) + maxrow * n2);
  if (!row_ok(rp, i, nnzb) || rp[i + 1] - rp[i] > maxrow) {
    if (lane == 0) atomicMin(bad_row, i);
    return;
  }
  const int e0 = rp[i], e1 = rp[i + 1];
  bool cols_ok = true;
  for (int e = e0 + lane; e < e1; e += 32) {
    const int j = ci[e];
    cols_ok = cols_ok && j >= 0 && j < N;
  }
  if (!__all_sync(0xffffffffu, cols_ok)) {
    if (lane == 0) atomicMin(bad_row, i);
    return;
  }
  // one lane per (block, secondary row): a dot product over the block row's
  // n1 entries (contiguous across lanes), the partial sums of each row then
  // added in block order by one lane
  double* part = M + n2 * (n2 + 1);             // nblocks x n2
  const int pairs = (e1 - e0) * n2;
  for (int t = lane; t < pairs; t += 32) {
    const int eb = t / n2, k = t - eb * n2;
    const int e = e0 + eb;
    const double* Y = j21 + (size_t)e * n2 * n1 + (size_t)k * n1;
    const double* x = d1 + (size_t)ci[e] * n1;
    double s = 0.0;
    for (int c = 0; c < n1; ++c) s += Y[c] * x[c];
    part[t] = s;
  }
  __syncwarp();
  for (int k = lane; k < n2; k += 32) {
    double s = 0.0;
    for (int eb = 0; eb < e1 - e0; ++eb) s += part[eb * n2 + k];
    M[k * (n2 + 1) + n2] = -r2[(size_t)i * n2 + k] - s;
  }
  const double* D = j22 + (size_t)i * n2 * n2;
  for (int idx = lane; idx < n2 * n2; idx += 32) {
    const int r = idx / n2, c = idx - r * n2;
    M[r * (n2 + 1) + c] = D[idx];
  }
  __syncwarp();
  if (!warp_gauss_jordan(M, n2, 1)) {
    if (lane == 0) atomicMin(bad_pivot, i);
    return;
  }
  for (int r = lane; r < n2; r += 32) d2[(size_t)i * n2 + r] = M[r * (n2 + 1) + n2];
}

void check_full(const mss_full* J) {
  if (!J || !J->row_ptr || !J->col_idx || !J->j11) fail(MSS_ERR_INVALID_ARG, "null matrix");
  if (J->n_rows < 1 || J->nnzb < J->n_rows) fail(MSS_ERR_INVALID_ARG, "bad matrix sizes");
  if (J->n1 < 1 || J->n1 > MSS_CONDENSE_MAX_UNKNOWNS || J->n2 < 0 ||
      J->n2 > MSS_CONDENSE_MAX_UNKNOWNS)
    fail(MSS_ERR_INVALID_ARG, "n1 must be in [1, 16] and n2 in [0, 16]");
  if (J->n2 > 0 && (!J->j21 || !J->j12 || !J->j22))
    fail(MSS_ERR_INVALID_ARG, "null secondary blocks");
}

void report(Handle* h, const int* flags) {
  int f[2];
  read_back(h, f, flags, sizeof(f));
  if (f[0] != 0x7fffffff)
    fail(MSS_ERR_INVALID_ARG, "row_ptr or col_idx out of range (or, in the recovery, a row "
                              "of more than 64 blocks) at cell " + std::to_string(f[0]));
  if (f[1] != 0x7fffffff)
    fail(MSS_ERR_SINGULAR_BLOCK,
         "cell " + std::to_string(f[1]) + ": J22 block needs pivoting (zero pivot)");
}

}  // namespace

void condense(Handle* h, const mss_full* J, const double* r1, const double* r2, double* a,
              double* b) {
  check_full(J);
  if (!r1 || !a || !b || (J->n2 > 0 && !r2)) fail(MSS_ERR_INVALID_ARG, "null vector");
  DBuf<int> flags(h, 2);
  fill_int(h, flags.p, 0x7fffffff, 2);
  const int N = J->n_rows, n1 = J->n1, n2 = J->n2;
  const size_t smem = sizeof(double) * (size_t)kCondWarps * (n2 * 2 * n2 + n1 * n2);
  const unsigned grid = (unsigned)((N + kCondWarps - 1) / kCondWarps);
  {
    TraceScope ts(h, TR_CONDENSE);
    k_condense<<<grid, 32 * kCondWarps, smem, h->stream>>>(N, J->nnzb, n1, n2, J->row_ptr,
                                                           J->j11, J->j21, J->j12, J->j22, r1, r2,
                                                           a, b, flags.p, flags.p + 1);
    MSS_LAUNCH_CK("k_condense");
  }
  report(h, flags.p);
}

void recover(Handle* h, const mss_full* J, const double* r2, const double* d1, double* d2) {
  check_full(J);
  if (J->n2 == 0) return;
  if (!r2 || !d1 || !d2) fail(MSS_ERR_INVALID_ARG, "null vector");
  DBuf<int> flags(h, 2);
  fill_int(h, flags.p, 0x7fffffff, 2);
  const int N = J->n_rows, n1 = J->n1, n2 = J->n2;
  const size_t smem = sizeof(double) * (size_t)kCondWarps * (n2 * (n2 + 1) + kRecoverRow * n2);
  const unsigned grid = (unsigned)((N + kCondWarps - 1) / kCondWarps);
  {
    TraceScope ts(h, TR_RECOVER);
    k_recover<<<grid, 32 * kCondWarps, smem, h->stream>>>(N, J->nnzb, n1, n2, kRecoverRow,
                                                          J->row_ptr,
                                                          J->col_idx, J->j21, J->j22, r2, d1, d2,
                                                          flags.p, flags.p + 1);
    MSS_LAUNCH_CK("k_recover");
  }
  report(h, flags.p);
}

}  // namespace mss
