// gnn.cu -- learned interpolation for the temperature AMG stage (not in the
// paper; the paper's T stage uses classical AMG, Sec. 5.1).
//
// A message-passing network of width 32 on the graph of the level-0
// temperature operator A = C_TT predicts, for every F point i and every C
// point j that classical interpolation uses, a relative correction s_ij; the
// learned weight is w_ij = p_ij (1 + s_ij), so a zero read-out is classical
// interpolation. Network:
//   x_i  = [a_ii / mean a_kk, sum_j a_ij / a_ii]
//   e_ij = [a_ij / a_ii, a_ji / a_jj, |a_ij| / max_k |a_ik|, cf_i, cf_j]
//   H0 = relu(X Wn + bn), G = relu(E We + be)
//   l = 1..3: M_i = sum_j G_ij * H_j (elementwise), H^l = relu([H | M] W_l + b_l)
//   z = relu([H3_i | H3_j | G_ij] Wo + bo), s_ij = z . wr + br
// Loss over smooth test vectors e_k (damped Jacobi on A e = 0), with the
// defect d_k = e_k - P e_k|C:
//   residual norm:    L = sum_k ||A d_k||^2 / sum_k ||A e_k||^2, or
//   diagonal norm:    L = sum_k sum_i |a_ii| d_ki^2 / sum_k sum_i |a_ii| e_ki^2
//   (the least-squares interpolation criterion of bootstrap AMG).
//
// Dense layers run on the tensor cores (mma.sync m16n8k16, BF16 operands,
// FP32 accumulation) with every FP32 operand split into two BF16 parts
// (x = hi + lo) and three products per tile, hi*hi + lo*hi + hi*lo (the
// "bf16x3" scheme of Henry, Tang and Heinecke, ARITH 2019), which keeps the
// products near FP32 accuracy; activations are stored in FP32; the loss and
// its derivative with respect to the weights are FP64. The products are thin
// ([rows x 64] x [64 x 32]): a layer reads and writes about 400 B per row
// for 4 kFLOP, so they are bound by memory traffic, not by the tensor pipe.
#include <cmath>
#include <memory>
#include <utility>

#include "common.cuh"

namespace mss {

// ---- parameter layout (float vector) --------------------------------------
namespace gp {
constexpr int W = 32;
constexpr int Wn = 0, bn = Wn + 2 * W, We = bn + W, be = We + 5 * W;
constexpr int W1 = be + W, b1 = W1 + 64 * W, W2 = b1 + W, b2 = W2 + 64 * W;
constexpr int W3 = b2 + W, b3 = W3 + 64 * W, Wo = b3 + W, bo = Wo + 96 * W;
constexpr int wr = bo + W, br = wr + W, total = br + 1;
}  // namespace gp

int gnn_num_params() { return gp::total; }

namespace {

constexpr int WID = 32;

// ---- tensor-core dense products ----------------------------------------------
// two consecutive-k values split into BF16 high parts and BF16 remainders
__device__ __forceinline__ void split2(float x0, float x1, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat16 h0 = __float2bfloat16_rn(x0), h1 = __float2bfloat16_rn(x1);
  __nv_bfloat162 H, L;
  H.x = h0;
  H.y = h1;
  L.x = __float2bfloat16_rn(x0 - __bfloat162float(h0));
  L.y = __float2bfloat16_rn(x1 - __bfloat162float(h1));
  hi = *reinterpret_cast<uint32_t*>(&H);
  lo = *reinterpret_cast<uint32_t*>(&L);
}

__device__ __forceinline__ void mma16816(float c[4], const uint32_t a[4], const uint32_t b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Y[r, 0:NO] = act(X[r, 0:KI] Bt^T + bias), one warp per 16 rows. Bt is the
// weight stored [NO x KI] row-major (the mma's column-major B) as BF16 high
// parts Bh and remainders Bl. X and Y are FP32 with leading dimensions ldx,
// ldy. act: 0 none, 1 relu.
template <int KI, int NO>
__global__ void k_dense(int rows, const float* __restrict__ X, int ldx,
                        const __nv_bfloat16* __restrict__ Bh, const __nv_bfloat16* __restrict__ Bl,
                        const float* __restrict__ bias, float* __restrict__ Y, int ldy, int act) {
  __shared__ uint32_t Bs[2][NO * KI / 2];
  for (int i = threadIdx.x; i < NO * KI / 2; i += blockDim.x) {
    Bs[0][i] = reinterpret_cast<const uint32_t*>(Bh)[i];
    Bs[1][i] = reinterpret_cast<const uint32_t*>(Bl)[i];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const long long r0 = ((long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 16;
  if (r0 >= rows) return;
  float c[NO / 8][4];
#pragma unroll
  for (int j = 0; j < NO / 8; ++j) c[j][0] = c[j][1] = c[j][2] = c[j][3] = 0.f;
  const long long ra = r0 + g, rb = r0 + g + 8;
  const bool va = ra < rows, vb = rb < rows;
#pragma unroll
  for (int k0 = 0; k0 < KI; k0 += 16) {
    uint32_t ah[4], al[4];
    float2 x00 = va ? *reinterpret_cast<const float2*>(X + ra * ldx + k0 + 2 * t) : float2{0, 0};
    float2 x10 = vb ? *reinterpret_cast<const float2*>(X + rb * ldx + k0 + 2 * t) : float2{0, 0};
    float2 x01 = va ? *reinterpret_cast<const float2*>(X + ra * ldx + k0 + 8 + 2 * t) : float2{0, 0};
    float2 x11 = vb ? *reinterpret_cast<const float2*>(X + rb * ldx + k0 + 8 + 2 * t) : float2{0, 0};
    split2(x00.x, x00.y, ah[0], al[0]);
    split2(x10.x, x10.y, ah[1], al[1]);
    split2(x01.x, x01.y, ah[2], al[2]);
    split2(x11.x, x11.y, ah[3], al[3]);
#pragma unroll
    for (int j = 0; j < NO / 8; ++j) {
      const int n = j * 8 + g;
      const int w0 = (n * KI + k0 + 2 * t) / 2, w1 = (n * KI + k0 + 8 + 2 * t) / 2;
      const uint32_t bh[2] = {Bs[0][w0], Bs[0][w1]}, bl[2] = {Bs[1][w0], Bs[1][w1]};
      mma16816(c[j], al, bh);
      mma16816(c[j], ah, bl);
      mma16816(c[j], ah, bh);
    }
  }
#pragma unroll
  for (int j = 0; j < NO / 8; ++j) {
    const int n = j * 8 + 2 * t;
    float b0 = bias ? bias[n] : 0.f, b1 = bias ? bias[n + 1] : 0.f;
    float y00 = c[j][0] + b0, y01 = c[j][1] + b1, y10 = c[j][2] + b0, y11 = c[j][3] + b1;
    if (act) {
      y00 = fmaxf(y00, 0.f); y01 = fmaxf(y01, 0.f);
      y10 = fmaxf(y10, 0.f); y11 = fmaxf(y11, 0.f);
    }
    if (va) *reinterpret_cast<float2*>(Y + ra * ldy + n) = float2{y00, y01};
    if (vb) *reinterpret_cast<float2*>(Y + rb * ldy + n) = float2{y10, y11};
  }
}

// dW[k, n] += sum_r X[r, k] dY[r, n] for the features k in [koff, koff + KI)
// that are below kreal, and (when db is given) db[n] += sum_r dY[r, n]; warps
// stride over 16-row chunks and add their partial products into the FP32
// gradient with atomics. Operands split as in k_dense.
template <int KI, int NO>
__global__ void k_wgrad(int rows, const float* __restrict__ X, int ldx, int koff,
                        const float* __restrict__ dY, int ldd, int kreal,
                        float* __restrict__ dW, float* __restrict__ db) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const long long warp = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
  float c[KI / 16][NO / 8][4];
#pragma unroll
  for (int i = 0; i < KI / 16; ++i)
#pragma unroll
    for (int j = 0; j < NO / 8; ++j) c[i][j][0] = c[i][j][1] = c[i][j][2] = c[i][j][3] = 0.f;
  float bsum[NO / 8][2];
#pragma unroll
  for (int j = 0; j < NO / 8; ++j) bsum[j][0] = bsum[j][1] = 0.f;
  for (long long r0 = warp * 16; r0 < rows; r0 += nw * 16) {
    // B = dY chunk: (k = row, n = column)
    uint32_t bh[NO / 8][2], bl[NO / 8][2];
    const long long q0 = r0 + 2 * t, q1 = q0 + 1, q2 = q0 + 8, q3 = q0 + 9;
#pragma unroll
    for (int j = 0; j < NO / 8; ++j) {
      const int n = j * 8 + g;
      float y0 = q0 < rows ? dY[q0 * ldd + n] : 0.f, y1 = q1 < rows ? dY[q1 * ldd + n] : 0.f;
      float y2 = q2 < rows ? dY[q2 * ldd + n] : 0.f, y3 = q3 < rows ? dY[q3 * ldd + n] : 0.f;
      split2(y0, y1, bh[j][0], bl[j][0]);
      split2(y2, y3, bh[j][1], bl[j][1]);
    }
    if (db) {
      // bias sums in FP32: lane (g, t) holds columns j*8+2t and j*8+2t+1
#pragma unroll
      for (int j = 0; j < NO / 8; ++j) {
        const int n = j * 8 + 2 * t;
        const long long r = r0 + g, r8 = r0 + g + 8;
        if (r < rows) { bsum[j][0] += dY[r * ldd + n]; bsum[j][1] += dY[r * ldd + n + 1]; }
        if (r8 < rows) { bsum[j][0] += dY[r8 * ldd + n]; bsum[j][1] += dY[r8 * ldd + n + 1]; }
      }
    }
#pragma unroll
    for (int i = 0; i < KI / 16; ++i) {
      // A = X^T chunk: (m = feature, k = row)
      const int f0 = koff + i * 16 + g, f1 = f0 + 8;
      float x00 = q0 < rows ? X[q0 * ldx + f0] : 0.f, x01 = q1 < rows ? X[q1 * ldx + f0] : 0.f;
      float x10 = q0 < rows ? X[q0 * ldx + f1] : 0.f, x11 = q1 < rows ? X[q1 * ldx + f1] : 0.f;
      float x02 = q2 < rows ? X[q2 * ldx + f0] : 0.f, x03 = q3 < rows ? X[q3 * ldx + f0] : 0.f;
      float x12 = q2 < rows ? X[q2 * ldx + f1] : 0.f, x13 = q3 < rows ? X[q3 * ldx + f1] : 0.f;
      uint32_t ah[4], al[4];
      split2(x00, x01, ah[0], al[0]);
      split2(x10, x11, ah[1], al[1]);
      split2(x02, x03, ah[2], al[2]);
      split2(x12, x13, ah[3], al[3]);
#pragma unroll
      for (int j = 0; j < NO / 8; ++j) {
        mma16816(c[i][j], al, bh[j]);
        mma16816(c[i][j], ah, bl[j]);
        mma16816(c[i][j], ah, bh[j]);
      }
    }
  }
#pragma unroll
  for (int i = 0; i < KI / 16; ++i)
#pragma unroll
    for (int j = 0; j < NO / 8; ++j) {
      const int k0 = koff + i * 16 + g, k1 = k0 + 8, n = j * 8 + 2 * t;
      if (k0 < kreal) {
        atomicAdd(dW + k0 * NO + n, c[i][j][0]);
        atomicAdd(dW + k0 * NO + n + 1, c[i][j][1]);
      }
      if (k1 < kreal) {
        atomicAdd(dW + k1 * NO + n, c[i][j][2]);
        atomicAdd(dW + k1 * NO + n + 1, c[i][j][3]);
      }
    }
  if (db) {
#pragma unroll
    for (int j = 0; j < NO / 8; ++j) {
      float s0 = bsum[j][0], s1 = bsum[j][1];
      // lanes with the same t hold the same columns: sum over g
      for (int o = 4; o < 32; o <<= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
      }
      if (g == 0) {
        atomicAdd(db + j * 8 + 2 * t, s0);
        atomicAdd(db + j * 8 + 2 * t + 1, s1);
      }
    }
  }
}

// ---- graph preparation ------------------------------------------------------
// off-diagonal edges of every row in CSR order (the diagonal is in every row)
__global__ void k_gnn_edges(int n, int m, const int* __restrict__ rp, const int* __restrict__ ci,
                            const double* __restrict__ a, int* __restrict__ ecol,
                            double* __restrict__ eval, double* __restrict__ diag,
                            int* __restrict__ bad) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int nd = 0;
  for (int q = rp[i]; q < rp[i + 1]; ++q) nd += ci[q] == i;
  if (nd != 1) {            // the edge offsets below assume one diagonal per row
    atomicExch(bad, 1);
    return;
  }
  int e = rp[i] - i;
  for (int q = rp[i]; q < rp[i + 1]; ++q) {
    if (ci[q] == i) {
      diag[i] = a[q];
      continue;
    }
    if (e < m) {
      ecol[e] = ci[q];
      eval[e] = a[q];
    }
    ++e;
  }
}

// reverse edge (j, i) of every edge (i, j), -1 if not stored
__global__ void k_gnn_rev(int n, const int* __restrict__ rp, const int* __restrict__ ecol,
                          int* __restrict__ rev, int* __restrict__ bad) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int e = rp[i] - i; e < rp[i + 1] - i - 1; ++e) {
    const int j = ecol[e];
    int lo = rp[j] - j, hi = rp[j + 1] - j - 2, f = -1;
    while (lo <= hi) {
      const int mid = (lo + hi) >> 1;
      const int c = ecol[mid];
      if (c == i) { f = mid; break; }
      if (c < i) lo = mid + 1; else hi = mid - 1;
    }
    rev[e] = f;
    if (f < 0) atomicExch(bad, 1);
  }
}

// node features (2 of 16 columns) and edge features (5 of 16 columns)
__global__ void k_gnn_features(int n, const int* __restrict__ rp, const int* __restrict__ ecol,
                               const double* __restrict__ eval, const int* __restrict__ rev,
                               const double* __restrict__ diag, const int* __restrict__ cf,
                               const double* __restrict__ dmean, float* __restrict__ X0,
                               float* __restrict__ E) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int e0 = rp[i] - i, e1 = rp[i + 1] - i - 1;
  double rs = diag[i], amax = 0.0;
  for (int e = e0; e < e1; ++e) {
    rs += eval[e];
    amax = fmax(amax, fabs(eval[e]));
  }
  float* x = X0 + (size_t)i * 16;
  x[0] = (float)(diag[i] / dmean[0]);
  x[1] = (float)(rs / diag[i]);
  for (int k = 2; k < 16; ++k) x[k] = 0.f;
  for (int e = e0; e < e1; ++e) {
    const int j = ecol[e];
    float* f = E + (size_t)e * 16;
    f[0] = (float)(eval[e] / diag[i]);
    f[1] = (float)((rev[e] >= 0 ? eval[rev[e]] : 0.0) / diag[j]);
    f[2] = amax > 0.0 ? (float)(fabs(eval[e]) / amax) : 0.f;
    f[3] = (float)cf[i];
    f[4] = (float)cf[j];
    for (int k = 5; k < 16; ++k) f[k] = 0.f;
  }
}

__global__ void k_mean(int n, const double* __restrict__ v, double* __restrict__ out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += v[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = red[0] / n;
}

// interpolation entries of F rows: count, then fill (ti, tj fine, te edge, tp, tpos)
__global__ void k_gnn_tcount(int n, const int* __restrict__ cf, const int* __restrict__ prp,
                             int* __restrict__ cnt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) cnt[i] = cf[i] ? 0 : prp[i + 1] - prp[i];
}

__global__ void k_gnn_cmap(int n, const int* __restrict__ cf, const int* __restrict__ cidx,
                           int* __restrict__ cmap) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && cf[i]) cmap[cidx[i]] = i;
}

__global__ void k_gnn_tfill(int n, const int* __restrict__ rp, const int* __restrict__ ecol,
                            const int* __restrict__ cf, const int* __restrict__ prp,
                            const int* __restrict__ pci, const double* __restrict__ pv,
                            const int* __restrict__ cmap, const int* __restrict__ trp,
                            int* __restrict__ ti, int* __restrict__ tj, int* __restrict__ te,
                            double* __restrict__ tp, int* __restrict__ tpos,
                            int* __restrict__ bad) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || cf[i]) return;
  int t = trp[i];
  for (int q = prp[i]; q < prp[i + 1]; ++q, ++t) {
    const int j = cmap[pci[q]];
    int lo = rp[i] - i, hi = rp[i + 1] - i - 2, f = -1;
    while (lo <= hi) {
      const int mid = (lo + hi) >> 1;
      const int c = ecol[mid];
      if (c == j) { f = mid; break; }
      if (c < j) lo = mid + 1; else hi = mid - 1;
    }
    if (f < 0) atomicExch(bad, 1);
    ti[t] = i;
    tj[t] = j;
    te[t] = f < 0 ? 0 : f;
    tp[t] = pv[q];
    tpos[t] = q;
  }
}

// ---- forward pieces ----------------------------------------------------------
// IN[i, 32:64] = sum_{e in row i} G[e] * IN[ecol(e), 0:32] (warp per row, lane = feature)
__global__ void k_gnn_message(int n, const int* __restrict__ rp, const int* __restrict__ ecol,
                              const float* __restrict__ G, float* __restrict__ IN) {
  const long long i = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int f = threadIdx.x & 31;
  if (i >= n) return;
  float s = 0.f;
  for (int e = rp[i] - (int)i; e < rp[i + 1] - (int)i - 1; ++e)
    s += G[(size_t)e * WID + f] * IN[(size_t)ecol[e] * 64 + f];
  IN[(size_t)i * 64 + 32 + f] = s;
}

// R[t] = [H3_i | H3_j | G_e]
__global__ void k_gnn_gather(int T, const int* __restrict__ ti, const int* __restrict__ tj,
                             const int* __restrict__ te, const float* __restrict__ H3,
                             const float* __restrict__ G, float* __restrict__ R) {
  const long long t = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int f = threadIdx.x & 31;
  if (t >= T) return;
  float* r = R + (size_t)t * 96;
  r[f] = H3[(size_t)ti[t] * WID + f];
  r[32 + f] = H3[(size_t)tj[t] * WID + f];
  r[64 + f] = G[(size_t)te[t] * WID + f];
}

// s_t = Z_t . wr + br; w_t = p_t (1 + s_t)
__global__ void k_gnn_readout(int T, const float* __restrict__ Z, const float* __restrict__ prm,
                              const double* __restrict__ tp, float* __restrict__ s,
                              double* __restrict__ w) {
  const long long t = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int f = threadIdx.x & 31;
  if (t >= T) return;
  float v = Z[(size_t)t * WID + f] * prm[gp::wr + f];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (f == 0) {
    const float st = v + prm[gp::br];
    s[t] = st;
    if (w) w[t] = tp[t] * (1.0 + (double)st);
  }
}

// ---- loss (FP64) ---------------------------------------------------------------
// d[i, k] = 0 at C points, e[i, k] - sum_t w_t e[tj_t, k] at F points (K columns, row-major n x K)
__global__ void k_gnn_defect(int n, int K, const int* __restrict__ cf, const int* __restrict__ trp,
                             const int* __restrict__ tj, const double* __restrict__ w,
                             const double* __restrict__ ev, double* __restrict__ d) {
  long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (long long)n * K) return;
  const int i = (int)(id / K), k = (int)(id % K);
  if (cf[i]) {
    d[id] = 0.0;
    return;
  }
  double v = ev[id];
  for (int t = trp[i]; t < trp[i + 1]; ++t) v -= w[t] * ev[(size_t)tj[t] * K + k];
  d[id] = v;
}

// y = A x (mode 0), A^T x (mode 1) or |D|^(1/2) x (mode 2) for K columns
__global__ void k_gnn_spmm(int n, int K, const int* __restrict__ rp, const int* __restrict__ ecol,
                           const double* __restrict__ eval, const int* __restrict__ rev,
                           const double* __restrict__ diag, const double* __restrict__ x,
                           double* __restrict__ y, int trans) {
  long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (long long)n * K) return;
  const int i = (int)(id / K), k = (int)(id % K);
  if (trans == 2) {
    y[id] = sqrt(fabs(diag[i])) * x[id];
    return;
  }
  double v = diag[i] * x[id];
  for (int e = rp[i] - i; e < rp[i + 1] - i - 1; ++e) {
    const double a = trans ? eval[rev[e]] : eval[e];
    v += a * x[(size_t)ecol[e] * K + k];
  }
  y[id] = v;
}

__global__ void k_gnn_sumsq(long long len, const double* __restrict__ v, double scale,
                            double* __restrict__ out) {
  __shared__ double red[256];
  double s = 0.0;
  for (long long i = threadIdx.x; i < len; i += blockDim.x) s += v[i] * v[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = red[0] * scale;
}

// v <- v * c (K columns); used for dL/dr = 2 r / den
__global__ void k_gnn_scale(long long len, double* __restrict__ v, const double* __restrict__ den,
                            double c) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < len) v[i] = v[i] * (c / den[0]);
}

// ds_t = -p_t sum_k dd[ti, k] e[tj, k]  (dd = dL/dd; C rows of dd are unused)
__global__ void k_gnn_ds(int T, int K, const int* __restrict__ ti, const int* __restrict__ tj,
                         const double* __restrict__ tp, const double* __restrict__ dd,
                         const double* __restrict__ ev, float* __restrict__ ds) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= T) return;
  double v = 0.0;
  for (int k = 0; k < K; ++k) v += dd[(size_t)ti[t] * K + k] * ev[(size_t)tj[t] * K + k];
  ds[t] = (float)(-v * tp[t]);
}

// damped Jacobi e <- e - omega D^-1 A e on K columns (two buffers)
__global__ void k_gnn_jacobi(int n, int K, const int* __restrict__ rp, const int* __restrict__ ecol,
                             const double* __restrict__ eval, const double* __restrict__ diag,
                             double omega, const double* __restrict__ x, double* __restrict__ y) {
  long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (long long)n * K) return;
  const int i = (int)(id / K), k = (int)(id % K);
  double v = diag[i] * x[id];
  for (int e = rp[i] - i; e < rp[i + 1] - i - 1; ++e) v += eval[e] * x[(size_t)ecol[e] * K + k];
  y[id] = x[id] - omega * v / diag[i];
}

// ---- backward pieces -------------------------------------------------------------
// dZ = ds * wr * [Z > 0]; dwr = sum_t ds_t Z_t; dbr = sum_t ds_t
__global__ void k_gnn_readout_bwd(int T, const float* __restrict__ Z, const float* __restrict__ ds,
                                  const float* __restrict__ prm, float* __restrict__ dZ,
                                  float* __restrict__ grad) {
  const long long t = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int f = threadIdx.x & 31;
  float gw = 0.f, gb = 0.f;
  if (t < T) {
    const float z = Z[(size_t)t * WID + f], d = ds[t];
    dZ[(size_t)t * WID + f] = z > 0.f ? d * prm[gp::wr + f] : 0.f;
    gw = d * z;
    gb = f == 0 ? d : 0.f;
  }
  // one atomic per block and feature
  __shared__ float sw[32][33];
  __shared__ float sb[32];
  const int wi = threadIdx.x >> 5;
  sw[wi][f] = gw;
  if (f == 0) sb[wi] = gb;
  __syncthreads();
  if (wi == 0) {
    float a = 0.f, b = 0.f;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      a += sw[k][f];
      if (f == 0) b += sb[k];
    }
    atomicAdd(grad + gp::wr + f, a);
    if (f == 0) atomicAdd(grad + gp::br, b);
  }
}

// dH3[i] = sum over row i's entries of dR[t, 0:32]; dH3[j] += dR[t, 32:64]
// (atomics); dG[e] = dR[t, 64:96] (one entry per edge at most)
__global__ void k_gnn_scatter_rows(int n, const int* __restrict__ trp, const float* __restrict__ dR,
                                   float* __restrict__ dH) {
  const long long i = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int f = threadIdx.x & 31;
  if (i >= n) return;
  float s = 0.f;
  for (int t = trp[i]; t < trp[i + 1]; ++t) s += dR[(size_t)t * 96 + f];
  dH[(size_t)i * WID + f] = s;
}

__global__ void k_gnn_scatter_cols(int T, const int* __restrict__ tj, const int* __restrict__ te,
                                   const float* __restrict__ dR, float* __restrict__ dH,
                                   float* __restrict__ dG) {
  const long long t = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int f = threadIdx.x & 31;
  if (t >= T) return;
  atomicAdd(dH + (size_t)tj[t] * WID + f, dR[(size_t)t * 96 + 32 + f]);
  dG[(size_t)te[t] * WID + f] += dR[(size_t)t * 96 + 64 + f];
}

// dY = dH * [Y > 0] (Y with leading dimension ldy)
__global__ void k_gnn_relu_bwd(long long rows, const float* __restrict__ dH, int ldh,
                               const float* __restrict__ Y, int ldy, float* __restrict__ dY) {
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= rows * WID) return;
  const long long r = id / WID;
  const int f = (int)(id % WID);
  dY[id] = Y[r * ldy + f] > 0.f ? dH[r * ldh + f] : 0.f;
}

// message backward for one layer: dM = dIN[:, 32:64], H = IN[:, 0:32]
//   dG[e] += dM_i * H_j        (edge e = (i, j) in row i)
//   dHn[j] = dIN[j, 0:32] + sum_{e' = (j, i) in row j} dM_i * G[rev(e')]
__global__ void k_gnn_message_bwd(int n, const int* __restrict__ rp, const int* __restrict__ ecol,
                                  const int* __restrict__ rev, const float* __restrict__ G,
                                  const float* __restrict__ IN, const float* __restrict__ dIN,
                                  float* __restrict__ dG, float* __restrict__ dHn) {
  const long long i = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int f = threadIdx.x & 31;
  if (i >= n) return;
  const float dmi = dIN[(size_t)i * 64 + 32 + f];
  float acc = dIN[(size_t)i * 64 + f];
  for (int e = rp[i] - (int)i; e < rp[i + 1] - (int)i - 1; ++e) {
    const int j = ecol[e];
    dG[(size_t)e * WID + f] += dmi * IN[(size_t)j * 64 + f];
    acc += dIN[(size_t)j * 64 + 32 + f] * G[(size_t)rev[e] * WID + f];
  }
  dHn[(size_t)i * WID + f] = acc;
}

// Adam (Kingma and Ba, 2015)
__global__ void k_adam(int np, float* __restrict__ p, float* __restrict__ m1, float* __restrict__ m2,
                       const float* __restrict__ g, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  const float gi = g[i];
  const float a = b1 * m1[i] + (1.f - b1) * gi;
  const float b = b2 * m2[i] + (1.f - b2) * gi * gi;
  m1[i] = a;
  m2[i] = b;
  p[i] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
}

// BF16 weights (high parts at [0, hoff), remainders at [hoff, 2 hoff)):
// forward Bt [out x in] and backward B [in x out], inner dimension padded
__global__ void k_gnn_pack(const float* __restrict__ prm, int off, int kin, int kpad, int nout,
                           int hoff, __nv_bfloat16* __restrict__ Bt,
                           __nv_bfloat16* __restrict__ B) {
  int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= kpad * nout) return;
  const int k = id / nout, n = id % nout;
  const float v = k < kin ? prm[off + k * nout + n] : 0.f;
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
  Bt[(size_t)n * kpad + k] = h;
  Bt[hoff + (size_t)n * kpad + k] = l;
  B[(size_t)k * nout + n] = h;
  B[hoff + (size_t)k * nout + n] = l;
}

unsigned blocks_for_warps(long long warps, int threads = 256) {
  return grid_for(warps * 32, threads);
}

}  // namespace

// ---- the graph object -------------------------------------------------------------
struct GnnGraph {
  Handle* h;
  int n = 0, m = 0, T = 0, K = 0;
  DBuf<int> rp, ecol, rev, cf, trp, ti, tj, te, tpos, flag;
  DBuf<double> eval, diag, dmean, tp, ev, d, r, dd, scal;
  int norm = 0;   // loss norm: 0 ||A d||^2 (residual), 1 sum |a_ii| d_i^2 (interpolation error)
  DBuf<float> X0, E, IN1, IN2, IN3, H3, G, R, Z, s, ds, dZ, dR, dH, dY, dIN, dG, dYe;
  DBuf<__nv_bfloat16> wt, wb;   // packed BF16 weights (forward / backward copies)
  explicit GnnGraph(Handle* hh) : h(hh) {}
};

namespace {

// offsets of the packed BF16 layers inside wt / wb
constexpr int PK_N = 0;                     // Wn: 16 x 32
constexpr int PK_E = PK_N + 16 * 32;        // We: 16 x 32
constexpr int PK_1 = PK_E + 16 * 32;        // W1..W3: 64 x 32
constexpr int PK_2 = PK_1 + 64 * 32;
constexpr int PK_3 = PK_2 + 64 * 32;
constexpr int PK_O = PK_3 + 64 * 32;        // Wo: 96 x 32
constexpr int PK_TOTAL = PK_O + 96 * 32;

void pack_weights(GnnGraph& g, const float* prm) {
  Handle* h = g.h;
  struct L { int off, kin, kpad, pk; } ls[] = {{gp::Wn, 2, 16, PK_N}, {gp::We, 5, 16, PK_E},
                                               {gp::W1, 64, 64, PK_1}, {gp::W2, 64, 64, PK_2},
                                               {gp::W3, 64, 64, PK_3}, {gp::Wo, 96, 96, PK_O}};
  for (auto& l : ls) {
    k_gnn_pack<<<grid_for(l.kpad * 32, 256), 256, 0, h->stream>>>(
        prm, l.off, l.kin, l.kpad, 32, PK_TOTAL, g.wt.p + l.pk, g.wb.p + l.pk);
    MSS_LAUNCH_CK("k_gnn_pack");
  }
}

// Bt points at the high parts; the remainders follow PK_TOTAL elements later
template <int KI, int NO>
void dense(Handle* h, int rows, const float* X, int ldx, const __nv_bfloat16* Bt,
           const float* bias, float* Y, int ldy, int act) {
  if (rows <= 0) return;
  const long long warps = (rows + 15) / 16;
  k_dense<KI, NO><<<blocks_for_warps(warps, 128), 128, 0, h->stream>>>(
      rows, X, ldx, Bt, Bt + PK_TOTAL, bias, Y, ldy, act);
  MSS_LAUNCH_CK("k_dense");
}

// weight gradient over KI features, in windows of at most 64 (registers)
template <int KI, int NO>
void wgrad(Handle* h, int rows, const float* X, int ldx, const float* dY, int ldd, int kreal,
           float* dW, float* db) {
  if (rows <= 0) return;
  long long warps = (rows + 15) / 16;
  const long long cap = 8LL * h->num_sms * 4;   // a few chunks per warp at scale
  if (warps > cap) warps = cap;
  constexpr int KW = KI > 64 ? KI / 2 : KI;
  for (int koff = 0; koff < KI; koff += KW) {
    k_wgrad<KW, NO><<<blocks_for_warps(warps, 128), 128, 0, h->stream>>>(
        rows, X, ldx, koff, dY, ldd, kreal, dW, koff == 0 ? db : nullptr);
    MSS_LAUNCH_CK("k_wgrad");
  }
}

void forward(GnnGraph& g, const float* prm, double* w) {
  Handle* h = g.h;
  pack_weights(g, prm);
  // embeddings
  dense<16, 32>(h, g.n, g.X0.p, 16, g.wt.p + PK_N, prm + gp::bn, g.IN1.p, 64, 1);
  dense<16, 32>(h, g.m, g.E.p, 16, g.wt.p + PK_E, prm + gp::be, g.G.p, 32, 1);
  float* IN[3] = {g.IN1.p, g.IN2.p, g.IN3.p};
  const int wk[3] = {PK_1, PK_2, PK_3};
  const int bk[3] = {gp::b1, gp::b2, gp::b3};
  for (int l = 0; l < 3; ++l) {
    k_gnn_message<<<blocks_for_warps(g.n), 256, 0, h->stream>>>(g.n, g.rp.p, g.ecol.p, g.G.p,
                                                                IN[l]);
    MSS_LAUNCH_CK("k_gnn_message");
    float* out = l < 2 ? IN[l + 1] : g.H3.p;
    dense<64, 32>(h, g.n, IN[l], 64, g.wt.p + wk[l], prm + bk[l], out, l < 2 ? 64 : 32, 1);
  }
  if (g.T > 0) {
    k_gnn_gather<<<blocks_for_warps(g.T), 256, 0, h->stream>>>(g.T, g.ti.p, g.tj.p, g.te.p,
                                                               g.H3.p, g.G.p, g.R.p);
    MSS_LAUNCH_CK("k_gnn_gather");
    dense<96, 32>(h, g.T, g.R.p, 96, g.wt.p + PK_O, prm + gp::bo, g.Z.p, 32, 1);
    k_gnn_readout<<<blocks_for_warps(g.T), 256, 0, h->stream>>>(g.T, g.Z.p, prm, g.tp.p, g.s.p,
                                                                w);
    MSS_LAUNCH_CK("k_gnn_readout");
  }
}

}  // namespace

GnnGraph* gnn_create(Handle* h, int n, const int* rp, const int* ci, const double* a,
                     const int* cf, const int* prp, const int* pci, const double* pv, int nnz) {
  std::unique_ptr<GnnGraph> G(new GnnGraph(h));
  GnnGraph& g = *G;
  g.n = n;
  g.m = nnz - n;
  if (g.m < 0) fail(MSS_ERR_INVALID_ARG, "operator without a stored diagonal");
  g.rp.reset(h, n + 1);
  copy_dev(h, g.rp.p, rp, sizeof(int) * ((size_t)n + 1));
  g.cf.reset(h, n);
  copy_dev(h, g.cf.p, cf, sizeof(int) * (size_t)n);
  g.ecol.reset(h, g.m > 0 ? g.m : 1);
  g.eval.reset(h, g.m > 0 ? g.m : 1);
  g.rev.reset(h, g.m > 0 ? g.m : 1);
  g.diag.reset(h, n);
  g.dmean.reset(h, 1);
  g.flag.reset(h, 1);
  fill_int(h, g.flag.p, 0, 1);
  k_gnn_edges<<<grid_for(n, 128), 128, 0, h->stream>>>(n, g.m, rp, ci, a, g.ecol.p, g.eval.p,
                                                       g.diag.p, g.flag.p);
  MSS_LAUNCH_CK("k_gnn_edges");
  if (read_int(h, g.flag.p))
    fail(MSS_ERR_INVALID_ARG, "the temperature operator needs one diagonal entry per row");
  k_gnn_rev<<<grid_for(n, 128), 128, 0, h->stream>>>(n, g.rp.p, g.ecol.p, g.rev.p, g.flag.p);
  MSS_LAUNCH_CK("k_gnn_rev");
  if (read_int(h, g.flag.p))
    fail(MSS_ERR_INVALID_ARG, "the temperature operator's pattern is not structurally symmetric");
  k_mean<<<1, 256, 0, h->stream>>>(n, g.diag.p, g.dmean.p);
  MSS_LAUNCH_CK("k_mean");
  g.X0.reset(h, (size_t)n * 16);
  g.E.reset(h, (size_t)(g.m > 0 ? g.m : 1) * 16);
  k_gnn_features<<<grid_for(n, 128), 128, 0, h->stream>>>(n, g.rp.p, g.ecol.p, g.eval.p, g.rev.p,
                                                          g.diag.p, g.cf.p, g.dmean.p, g.X0.p,
                                                          g.E.p);
  MSS_LAUNCH_CK("k_gnn_features");
  // interpolation entries of the F rows
  DBuf<int> cnt(h, n), cidx(h, n + 1), cmap(h, n);
  exclusive_scan(h, cf, cidx.p, n);
  k_gnn_cmap<<<grid_for(n, 256), 256, 0, h->stream>>>(n, cf, cidx.p, cmap.p);
  MSS_LAUNCH_CK("k_gnn_cmap");
  k_gnn_tcount<<<grid_for(n, 256), 256, 0, h->stream>>>(n, cf, prp, cnt.p);
  MSS_LAUNCH_CK("k_gnn_tcount");
  g.trp.reset(h, n + 1);
  exclusive_scan(h, cnt.p, g.trp.p, n);
  g.T = read_int(h, g.trp.p + n);
  const size_t T1 = g.T > 0 ? g.T : 1;
  g.ti.reset(h, T1);
  g.tj.reset(h, T1);
  g.te.reset(h, T1);
  g.tp.reset(h, T1);
  g.tpos.reset(h, T1);
  fill_int(h, g.flag.p, 0, 1);
  k_gnn_tfill<<<grid_for(n, 128), 128, 0, h->stream>>>(n, g.rp.p, g.ecol.p, cf, prp, pci, pv,
                                                       cmap.p, g.trp.p, g.ti.p, g.tj.p, g.te.p,
                                                       g.tp.p, g.tpos.p, g.flag.p);
  MSS_LAUNCH_CK("k_gnn_tfill");
  if (read_int(h, g.flag.p))
    fail(MSS_ERR_INVALID_ARG, "an interpolation entry is not an edge of the operator");
  // activations
  const size_t m1 = g.m > 0 ? g.m : 1;
  g.IN1.reset(h, (size_t)n * 64);
  g.IN2.reset(h, (size_t)n * 64);
  g.IN3.reset(h, (size_t)n * 64);
  g.H3.reset(h, (size_t)n * WID);
  g.G.reset(h, m1 * WID);
  g.R.reset(h, T1 * 96);
  g.Z.reset(h, T1 * WID);
  g.s.reset(h, T1);
  g.wt.reset(h, 2 * PK_TOTAL);
  g.wb.reset(h, 2 * PK_TOTAL);
  return G.release();
}

void gnn_destroy(GnnGraph* g) { delete g; }

int gnn_entries(const GnnGraph* g) { return g->T; }
int gnn_nodes(const GnnGraph* g) { return g->n; }
int gnn_edges(const GnnGraph* g) { return g->m; }

void gnn_weights(GnnGraph* g, const float* prm, double* w) { forward(*g, prm, w); }

// writes the learned weights into P's values (CSR positions tpos)
__global__ void k_gnn_write_p(int T, const int* __restrict__ tpos, const double* __restrict__ w,
                              double* __restrict__ pv) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < T) pv[tpos[t]] = w[t];
}

void gnn_apply_to_p(GnnGraph* g, const float* prm, double* pv) {
  if (g->T == 0) return;
  DBuf<double> w(g->h, g->T);
  forward(*g, prm, w.p);
  k_gnn_write_p<<<grid_for(g->T, 256), 256, 0, g->h->stream>>>(g->T, g->tpos.p, w.p, pv);
  MSS_LAUNCH_CK("k_gnn_write_p");
}

void gnn_set_vectors(GnnGraph* gg, int K, const double* starts, int nu, double omega, int norm) {
  GnnGraph& g = *gg;
  Handle* h = g.h;
  if (K < 1 || K > 64 || nu < 0) fail(MSS_ERR_INVALID_ARG, "K in [1, 64] and nu >= 0");
  if (norm != 0 && norm != 1) fail(MSS_ERR_INVALID_ARG, "loss norm 0 (residual) or 1 (diagonal)");
  g.norm = norm;
  const long long len = (long long)g.n * K;
  g.K = K;
  g.ev.reset(h, len);
  DBuf<double> tmp(h, len);
  copy_dev(h, g.ev.p, starts, sizeof(double) * (size_t)len);
  for (int s = 0; s < nu; ++s) {
    k_gnn_jacobi<<<grid_for(len, 256), 256, 0, h->stream>>>(g.n, K, g.rp.p, g.ecol.p, g.eval.p,
                                                           g.diag.p, omega, g.ev.p, tmp.p);
    MSS_LAUNCH_CK("k_gnn_jacobi");
    std::swap(g.ev.p, tmp.p);
  }
  g.d.reset(h, len);
  g.r.reset(h, len);
  g.dd.reset(h, len);
  g.scal.reset(h, 2);
  // denominator sum_k ||op e_k||^2, op = A or |D|^(1/2)
  k_gnn_spmm<<<grid_for(len, 256), 256, 0, h->stream>>>(g.n, K, g.rp.p, g.ecol.p, g.eval.p,
                                                        g.rev.p, g.diag.p, g.ev.p, g.r.p,
                                                        norm ? 2 : 0);
  MSS_LAUNCH_CK("k_gnn_spmm");
  k_gnn_sumsq<<<1, 256, 0, h->stream>>>(len, g.r.p, 1.0, g.scal.p + 1);
  MSS_LAUNCH_CK("k_gnn_sumsq");
}

double gnn_loss_grad(GnnGraph* gg, const float* prm, float* grad) {
  GnnGraph& g = *gg;
  Handle* h = g.h;
  if (g.K == 0) fail(MSS_ERR_NOT_SETUP, "test vectors not set");
  const long long len = (long long)g.n * g.K;
  DBuf<double> w(h, g.T > 0 ? g.T : 1);
  forward(g, prm, w.p);
  k_gnn_defect<<<grid_for(len, 256), 256, 0, h->stream>>>(g.n, g.K, g.cf.p, g.trp.p, g.tj.p, w.p,
                                                         g.ev.p, g.d.p);
  MSS_LAUNCH_CK("k_gnn_defect");
  k_gnn_spmm<<<grid_for(len, 256), 256, 0, h->stream>>>(g.n, g.K, g.rp.p, g.ecol.p, g.eval.p,
                                                       g.rev.p, g.diag.p, g.d.p, g.r.p,
                                                       g.norm ? 2 : 0);
  MSS_LAUNCH_CK("k_gnn_spmm");
  k_gnn_sumsq<<<1, 256, 0, h->stream>>>(len, g.r.p, 1.0, g.scal.p);
  MSS_LAUNCH_CK("k_gnn_sumsq");
  double sc[2];
  read_back(h, sc, g.scal.p, sizeof(sc));
  const double L = sc[0] / sc[1];
  if (!grad) return L;
  // dL/dd = op^T (2 r / den)
  k_gnn_scale<<<grid_for(len, 256), 256, 0, h->stream>>>(len, g.r.p, g.scal.p + 1, 2.0);
  MSS_LAUNCH_CK("k_gnn_scale");
  k_gnn_spmm<<<grid_for(len, 256), 256, 0, h->stream>>>(g.n, g.K, g.rp.p, g.ecol.p, g.eval.p,
                                                       g.rev.p, g.diag.p, g.r.p, g.dd.p,
                                                       g.norm ? 2 : 1);
  MSS_LAUNCH_CK("k_gnn_spmm");
  MSS_CK(cudaMemsetAsync(grad, 0, sizeof(float) * gp::total, h->stream));
  const size_t T1 = g.T > 0 ? g.T : 1, m1 = g.m > 0 ? g.m : 1;
  g.ds.reset(h, T1);
  g.dZ.reset(h, T1 * WID);
  g.dR.reset(h, T1 * 96);
  g.dH.reset(h, (size_t)g.n * WID);
  g.dY.reset(h, (size_t)(g.n > (int)T1 ? g.n : T1) * WID + (size_t)m1 * WID);
  g.dIN.reset(h, (size_t)g.n * 64);
  g.dG.reset(h, m1 * WID);
  MSS_CK(cudaMemsetAsync(g.dG.p, 0, sizeof(float) * m1 * WID, h->stream));
  MSS_CK(cudaMemsetAsync(g.dH.p, 0, sizeof(float) * (size_t)g.n * WID, h->stream));
  if (g.T > 0) {
    k_gnn_ds<<<grid_for(g.T, 256), 256, 0, h->stream>>>(g.T, g.K, g.ti.p, g.tj.p, g.tp.p, g.dd.p,
                                                       g.ev.p, g.ds.p);
    MSS_LAUNCH_CK("k_gnn_ds");
    k_gnn_readout_bwd<<<blocks_for_warps(g.T), 256, 0, h->stream>>>(g.T, g.Z.p, g.ds.p, prm,
                                                                    g.dZ.p, grad);
    MSS_LAUNCH_CK("k_gnn_readout_bwd");
    wgrad<96, 32>(h, g.T, g.R.p, 96, g.dZ.p, 32, 96, grad + gp::Wo, grad + gp::bo);
    dense<32, 96>(h, g.T, g.dZ.p, 32, g.wb.p + PK_O, nullptr, g.dR.p, 96, 0);
    k_gnn_scatter_rows<<<blocks_for_warps(g.n), 256, 0, h->stream>>>(g.n, g.trp.p, g.dR.p,
                                                                     g.dH.p);
    MSS_LAUNCH_CK("k_gnn_scatter_rows");
    k_gnn_scatter_cols<<<blocks_for_warps(g.T), 256, 0, h->stream>>>(g.T, g.tj.p, g.te.p, g.dR.p,
                                                                     g.dH.p, g.dG.p);
    MSS_LAUNCH_CK("k_gnn_scatter_cols");
  }
  // message-passing layers, last to first; dH holds dL/dH^l
  float* IN[3] = {g.IN1.p, g.IN2.p, g.IN3.p};
  const int wk[3] = {PK_1, PK_2, PK_3};
  const int wo[3] = {gp::W1, gp::W2, gp::W3};
  const int bo[3] = {gp::b1, gp::b2, gp::b3};
  for (int l = 2; l >= 0; --l) {
    const float* Y = l < 2 ? IN[l + 1] : g.H3.p;
    const int ldy = l < 2 ? 64 : 32;
    k_gnn_relu_bwd<<<grid_for((long long)g.n * WID, 256), 256, 0, h->stream>>>(
        g.n, g.dH.p, WID, Y, ldy, g.dY.p);
    MSS_LAUNCH_CK("k_gnn_relu_bwd");
    wgrad<64, 32>(h, g.n, IN[l], 64, g.dY.p, 32, 64, grad + wo[l], grad + bo[l]);
    dense<32, 64>(h, g.n, g.dY.p, 32, g.wb.p + wk[l], nullptr, g.dIN.p, 64, 0);
    k_gnn_message_bwd<<<blocks_for_warps(g.n), 256, 0, h->stream>>>(
        g.n, g.rp.p, g.ecol.p, g.rev.p, g.G.p, IN[l], g.dIN.p, g.dG.p, g.dH.p);
    MSS_LAUNCH_CK("k_gnn_message_bwd");
  }
  // embeddings: dH now holds dL/dH0 (H0 = IN1[:, 0:32])
  k_gnn_relu_bwd<<<grid_for((long long)g.n * WID, 256), 256, 0, h->stream>>>(
      g.n, g.dH.p, WID, g.IN1.p, 64, g.dY.p);
  MSS_LAUNCH_CK("k_gnn_relu_bwd");
  wgrad<16, 32>(h, g.n, g.X0.p, 16, g.dY.p, 32, 2, grad + gp::Wn, grad + gp::bn);
  if (g.m > 0) {
    float* dYe = g.dY.p + (size_t)(g.n > (int)T1 ? g.n : T1) * WID;
    k_gnn_relu_bwd<<<grid_for((long long)g.m * WID, 256), 256, 0, h->stream>>>(
        g.m, g.dG.p, WID, g.G.p, WID, dYe);
    MSS_LAUNCH_CK("k_gnn_relu_bwd");
    wgrad<16, 32>(h, g.m, g.E.p, 16, dYe, 32, 5, grad + gp::We, grad + gp::be);
  }
  return L;
}

void gnn_adam(Handle* h, float* prm, float* m1, float* m2, const float* grad, int step, float lr,
              float b1, float b2, float eps) {
  if (step < 1) fail(MSS_ERR_INVALID_ARG, "Adam step counts from 1");
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  k_adam<<<grid_for(gp::total, 256), 256, 0, h->stream>>>(gp::total, prm, m1, m2, grad, lr, b1,
                                                          b2, eps, c1, c2);
  MSS_LAUNCH_CK("k_adam");
}

}  // namespace mss
