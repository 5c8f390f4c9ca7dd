// krylov.cu -- preconditioner orchestration (Algorithms 1 and 2) and
// right-preconditioned restarted FGMRES (Sec. 5.1).
//
// Arnoldi uses classical Gram-Schmidt, once (CGS1, default) or twice (CGS2):
// every pass is one streaming sweep over the basis that computes all
// projections at once; CGS2 fuses its second projections into the first
// update, and the last update carries the norm. The FP64 work per element is
// 2(j+1) FMAs for CGS1 and 4(j+1) for CGS2. All
// reductions are two-stage with a fixed block count and a fixed summation
// order, so results are identical from run to run.
//
// The solve state (step j, counts, norms, status) lives in device memory and
// every kernel reads j from it, so one fixed sequence of launches performs any
// Arnoldi step. Two drivers run that sequence: a host loop that reads the
// state back after each step, or one CUDA graph holding the whole restarted
// solve, whose two nested while-loop conditional nodes (restart cycles,
// Arnoldi steps) are continued or ended by the control kernels. Both run the
// same kernels in the same order and give the same bits.
#include <cmath>
#include <vector>

#include "common.cuh"
#include "krylov_kernels.cuh"

namespace mss {
namespace {

// ---- kernels: the bodies of krylov_kernels.cuh with vb = blockIdx.x and
// G = gridDim.x (single-thread kernels run one block)
__global__ void k_mdot(long long n, long long chunk, const double* __restrict__ V, long long ld,
                       const GState* __restrict__ st, const double* __restrict__ w, int wnorm,
                       double* __restrict__ partial) {
  dev::mdot(n, chunk, V, ld, st, w, wnorm, partial, blockIdx.x, gridDim.x);
}

__global__ void k_update(long long n, long long chunk, const double* __restrict__ V, long long ld,
                         const GState* __restrict__ st, const double* __restrict__ hcoef,
                         double* __restrict__ w, int mode, double* __restrict__ partial) {
  dev::update(n, chunk, V, ld, st, hcoef, w, mode, partial, blockIdx.x, gridDim.x);
}

__global__ void k_reduce(int G, const double* __restrict__ partial, double* __restrict__ out,
                         const GState* __restrict__ st, int mode) {
  dev::reduce(G, partial, out, st, mode, blockIdx.x);
}

__global__ void k_arnoldi_finish(int m, const double* __restrict__ h1,
                                 const double* __restrict__ h2, const double* __restrict__ sq,
                                 double* __restrict__ H, double* __restrict__ cs,
                                 double* __restrict__ sn, double* __restrict__ g,
                                 double* __restrict__ ks, const GState* __restrict__ st) {
  if (blockIdx.x != 0) return;
  dev::arnoldi_finish(m, h1, h2, sq, H, cs, sn, g, ks, st);
}

__global__ void k_normalize_store(long long n, const double* __restrict__ w,
                                  const double* __restrict__ ks, double* __restrict__ V,
                                  long long ld, const GState* __restrict__ st,
                                  double* __restrict__ vnext) {
  dev::normalize_store(n, w, ks, V, ld, st, vnext, blockIdx.x, gridDim.x);
}

__global__ void k_store_z(long long n, const double* __restrict__ z, double* __restrict__ Z,
                          long long ld, const GState* __restrict__ st) {
  dev::store_z(n, z, Z, ld, st, blockIdx.x, gridDim.x);
}

__global__ void k_cycle_head(long long n, const double* __restrict__ r, double* __restrict__ V,
                             double* __restrict__ vnext, GState* __restrict__ st) {
  dev::cycle_head(n, r, V, vnext, st, blockIdx.x, gridDim.x);
}

__global__ void k_init_g(int m, double* __restrict__ g, GState* __restrict__ st,
                         cudaGraphConditionalHandle inner, int use) {
  dev::init_g(m, g, st, inner, use, blockIdx.x);
}

__global__ void k_step_control(int m, const double* __restrict__ ks, GState* __restrict__ st,
                               cudaGraphConditionalHandle inner, int use) {
  if (blockIdx.x != 0) return;
  dev::step_control(m, ks, st, inner, use);
}

__global__ void k_backsolve(int m, const double* __restrict__ H, const double* __restrict__ g,
                            double* __restrict__ y, const GState* __restrict__ st) {
  if (blockIdx.x != 0) return;
  dev::backsolve(m, H, g, y, st);
}

__global__ void k_xupdate(long long n, const double* __restrict__ Z, long long ld,
                          const double* __restrict__ y, double* __restrict__ x,
                          const GState* __restrict__ st) {
  dev::xupdate(n, Z, ld, y, x, st, blockIdx.x, gridDim.x);
}

__global__ void k_resid_norm(long long n, long long chunk, const double* __restrict__ b,
                             double* __restrict__ r, double* __restrict__ partial) {
  dev::resid_norm(n, chunk, b, r, partial, blockIdx.x);
}

__global__ void k_sqnorm(long long n, long long chunk, const double* __restrict__ a,
                         double* __restrict__ partial) {
  dev::sqnorm(n, chunk, a, partial, blockIdx.x);
}

__global__ void k_cycle_control(const double* __restrict__ ks, GState* __restrict__ st,
                                cudaGraphConditionalHandle outer, int use) {
  if (blockIdx.x != 0) return;
  dev::cycle_control(ks, st, outer, use);
}

__global__ void k_solve_init(const double* __restrict__ ks, GState* __restrict__ st,
                             cudaGraphConditionalHandle outer, int use) {
  if (blockIdx.x != 0) return;
  dev::solve_init(ks, st, outer, use);
}

}  // namespace

static Red reduction_shape(Handle* h, long long n) {
  Red r;
  long long g = (n + 4095) / 4096;
  long long cap = 4LL * h->num_sms;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  r.G = (int)g;
  r.chunk = (n + g - 1) / g;
  r.chunk = (r.chunk + 31) / 32 * 32;
  return r;
}

Krylov workspace(Handle* h) {
  Krylov K;
  K.n = (long long)h->N * h->nb;
  K.m = h->opt.restart;
  K.ld = (K.n + 31) / 32 * 32;
  const int m = K.m;
  auto drop_graph = [&] {   // the solve graph holds pointers into the workspace
    if (h->sgraph) cudaGraphExecDestroy(h->sgraph);
    h->sgraph = nullptr;
  };
  if (h->m != m || h->V.n < (size_t)(m + 1) * K.ld) {
    drop_graph();
    h->m = m;
    h->V.reset(h, (size_t)(m + 1) * K.ld);
    h->Z.reset(h, (size_t)m * K.ld);
    h->bbar.reset(h, K.ld);
    h->res.reset(h, K.ld);
    // hbuf: H (m+1)m | cs m | sn m | g m+1 | y m | h1 m+1 | h2 m+1 | sq 2
    h->hbuf.reset(h, (size_t)(m + 1) * m + 7 * (size_t)(m + 2));
    h->kscal.reset(h, 8);
    h->gst.reset(h, 16);
    h->rfix.reset(h, K.ld);
    h->zfix.reset(h, K.ld);
    h->wfix.reset(h, K.ld);
  }
  K.rs = reduction_shape(h, K.n);
  if (h->part.n < (size_t)(m + 2) * K.rs.G) {
    drop_graph();
    h->part.reset(h, (size_t)(m + 2) * K.rs.G);
  }
  K.sgrid = grid_for(K.n, 256) > 4096 ? 4096 : grid_for(K.n, 256);
  K.H = h->hbuf.p;
  K.cs = K.H + (size_t)(m + 1) * m;
  K.sn = K.cs + (m + 2);
  K.g = K.sn + (m + 2);
  K.yv = K.g + (m + 2);
  K.h1 = K.yv + (m + 2);
  K.h2 = K.h1 + (m + 2);
  K.sq = K.h2 + (m + 2);
  K.ks = h->kscal.p;
  K.part = h->part.p;
  K.V = h->V.p;
  K.Z = h->Z.p;
  K.rfix = h->rfix.p;
  K.zfix = h->zfix.p;
  K.wfix = h->wfix.p;
  K.st = reinterpret_cast<GState*>(h->gst.p);
  return K;
}

namespace {

// ---- the four launch sequences of a solve ----------------------------------
// bbar = N^{-1} b, x = 0, ||bbar||, r = bbar
void seq_init(Handle* h, const Krylov& K, const double* b, double* x,
              cudaGraphConditionalHandle outer, int use) {
  scale_vector(h, b, h->bbar.p);
  fill_double(h, x, 0.0, K.n);
  k_sqnorm<<<K.rs.G, KT, 0, h->stream>>>(K.n, K.rs.chunk, h->bbar.p, K.part);
  MSS_LAUNCH_CK("k_sqnorm");
  k_reduce<<<1, KT, 0, h->stream>>>(K.rs.G, K.part, K.ks + 7, K.st, 2);
  MSS_LAUNCH_CK("k_reduce");
  k_solve_init<<<1, 32, 0, h->stream>>>(K.ks, K.st, outer, use);
  MSS_LAUNCH_CK("k_solve_init");
  copy_dev(h, h->res.p, h->bbar.p, sizeof(double) * (size_t)K.n);
}

void seq_head(Handle* h, const Krylov& K, cudaGraphConditionalHandle inner, int use) {
  k_cycle_head<<<K.sgrid, 256, 0, h->stream>>>(K.n, h->res.p, K.V, K.rfix, K.st);
  MSS_LAUNCH_CK("k_cycle_head");
  k_init_g<<<1, 128, 0, h->stream>>>(K.m, K.g, K.st, inner, use);   // restart <= 120
  MSS_LAUNCH_CK("k_init_g");
}

// one Arnoldi step j: z_j = M^{-1} v_j, w = Abar z_j, orthogonalise, normalise
void seq_step(Handle* h, const Krylov& K, cudaGraphConditionalHandle inner, int use) {
  const long long n = K.n;
  const Red rs = K.rs;
  precond_apply(h, K.rfix, K.zfix);
  k_store_z<<<K.sgrid, 256, 0, h->stream>>>(n, K.zfix, K.Z, K.ld, K.st);
  MSS_LAUNCH_CK("k_store_z");
  bsr_spmv(h, K.zfix, K.wfix);
  TraceScope ts(h, TR_ORTHO);
  const bool cgs2 = h->opt.orthog == MSS_CGS2;
  // CGS pass 1: h1 = V^T w and ||w0||^2
  k_mdot<<<rs.G, KT, 0, h->stream>>>(n, rs.chunk, K.V, K.ld, K.st, K.wfix, 1, K.part);
  MSS_LAUNCH_CK("k_mdot");
  k_reduce<<<K.m + 1, KT, 0, h->stream>>>(rs.G, K.part, K.h1, K.st, 0);
  MSS_LAUNCH_CK("k_reduce");
  k_reduce<<<1, KT, 0, h->stream>>>(rs.G, K.part, K.sq, K.st, 1);
  MSS_LAUNCH_CK("k_reduce");
  if (cgs2) {
    // update with h1, fused pass-2 projections h2
    k_update<<<rs.G, KT, 0, h->stream>>>(n, rs.chunk, K.V, K.ld, K.st, K.h1, K.wfix, 0, K.part);
    MSS_LAUNCH_CK("k_update");
    k_reduce<<<K.m + 1, KT, 0, h->stream>>>(rs.G, K.part, K.h2, K.st, 0);
    MSS_LAUNCH_CK("k_reduce");
  }
  // update (with h2 after CGS2, with h1 after CGS1) and the norm
  k_update<<<rs.G, KT, 0, h->stream>>>(n, rs.chunk, K.V, K.ld, K.st, cgs2 ? K.h2 : K.h1, K.wfix,
                                       1, K.part);
  MSS_LAUNCH_CK("k_update");
  k_reduce<<<1, KT, 0, h->stream>>>(rs.G, K.part, K.sq + 1, K.st, 2);
  MSS_LAUNCH_CK("k_reduce");
  k_arnoldi_finish<<<1, 32, 0, h->stream>>>(K.m, K.h1, cgs2 ? K.h2 : nullptr, K.sq, K.H, K.cs,
                                            K.sn, K.g, K.ks, K.st);
  MSS_LAUNCH_CK("k_arnoldi_finish");
  k_normalize_store<<<K.sgrid, 256, 0, h->stream>>>(n, K.wfix, K.ks, K.V, K.ld, K.st, K.rfix);
  MSS_LAUNCH_CK("k_normalize_store");
  k_step_control<<<1, 32, 0, h->stream>>>(K.m, K.ks, K.st, inner, use);
  MSS_LAUNCH_CK("k_step_control");
}

// end of a cycle: x += Z_k y_k, true residual, stop or restart
void seq_tail(Handle* h, const Krylov& K, double* x, cudaGraphConditionalHandle outer, int use) {
  k_backsolve<<<1, 32, 0, h->stream>>>(K.m, K.H, K.g, K.yv, K.st);
  MSS_LAUNCH_CK("k_backsolve");
  k_xupdate<<<K.sgrid, 256, 0, h->stream>>>(K.n, K.Z, K.ld, K.yv, x, K.st);
  MSS_LAUNCH_CK("k_xupdate");
  bsr_spmv(h, x, h->res.p);
  k_resid_norm<<<K.rs.G, KT, 0, h->stream>>>(K.n, K.rs.chunk, h->bbar.p, h->res.p, K.part);
  MSS_LAUNCH_CK("k_resid_norm");
  k_reduce<<<1, KT, 0, h->stream>>>(K.rs.G, K.part, K.ks + 6, K.st, 2);
  MSS_LAUNCH_CK("k_reduce");
  k_cycle_control<<<1, 32, 0, h->stream>>>(K.ks, K.st, outer, use);
  MSS_LAUNCH_CK("k_cycle_control");
}

GState read_state(Handle* h, const Krylov& K) {
  GState s;
  read_back(h, &s, K.st, sizeof(GState));
  return s;
}

void write_params(Handle* h, const Krylov& K, double tol, int maxit) {
  GState s{};
  s.tol = tol;
  s.maxit = maxit;
  write_to_device(h, K.st, &s, sizeof(GState));
}

int finish(const GState& s, mss_result* out) {
  mss_result res{};
  res.iters = s.total;
  res.restarts = s.restarts;
  res.status = s.status;
  res.rel_res_implicit = s.rel_impl;
  res.rel_res_true = s.rel_true;
  if (out) *out = res;
  if (s.rhs_bad) fail(MSS_ERR_BREAKDOWN, "right-hand side is not finite");
  if (s.status == MSS_ERR_BREAKDOWN)
    fail(MSS_ERR_BREAKDOWN, "non-finite value or zero Givens denominator in the Arnoldi process");
  return s.status;
}

// Host-driven: the state is read back after every step and every cycle.
int fgmres_host(Handle* h, const Krylov& K, const double* b, double* x, double tol, int maxit,
                mss_result* out) {
  const cudaGraphConditionalHandle none = 0;
  write_params(h, K, tol, maxit);
  seq_init(h, K, b, x, none, 0);
  GState s = read_state(h, K);
  while (s.go_outer) {
    seq_head(h, K, none, 0);
    bool go = s.total < maxit;
    while (go) {
      seq_step(h, K, none, 0);
      s = read_state(h, K);
      if (s.status == MSS_ERR_BREAKDOWN) return finish(s, out);
      go = s.go_inner;
    }
    seq_tail(h, K, x, none, 0);
    s = read_state(h, K);
  }
  return finish(s, out);
}

// init -> while (cycle) { head -> while (step) { step } -> tail }
void build_solve_graph(Handle* h, const Krylov& K) {
  if (h->sgraph) {
    cudaGraphExecDestroy(h->sgraph);
    h->sgraph = nullptr;
  }
  h->gb.reset(h, K.ld);
  h->gx.reset(h, K.ld);
  // capture on a private non-blocking stream (the handle's stream may be the
  // legacy default stream, which cannot be captured); launched on h->stream
  MSS_CK(cudaStreamSynchronize(h->stream));
  cudaStream_t cap = nullptr;
  MSS_CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  const cudaStream_t saved = h->stream;
  h->stream = cap;
  cudaGraph_t top = nullptr;
  auto restore = [&] {
    h->stream = saved;
    cudaStreamDestroy(cap);
    if (top) cudaGraphDestroy(top);
  };
  MSS_CK(cudaGraphCreate(&top, 0));
  try {
    cudaGraphConditionalHandle outer, inner;
    MSS_CK(cudaGraphConditionalHandleCreate(&outer, top, 0, cudaGraphCondAssignDefault));
    cudaGraphNode_t n0 = capture_into(h, top, nullptr, 0, &h->sg_launch[0],
                                      [&] { seq_init(h, K, h->gb.p, h->gx.p, outer, 1); });
    cudaGraphNode_t wo;
    cudaGraph_t ob = add_while(top, n0, outer, &wo);
    MSS_CK(cudaGraphConditionalHandleCreate(&inner, ob, 0, cudaGraphCondAssignDefault));
    cudaGraphNode_t n1 = capture_into(h, ob, nullptr, 0, &h->sg_launch[1],
                                      [&] { seq_head(h, K, inner, 1); });
    cudaGraphNode_t wi;
    cudaGraph_t ib = add_while(ob, n1, inner, &wi);
    capture_into(h, ib, nullptr, 0, &h->sg_launch[2], [&] { seq_step(h, K, inner, 1); });
    capture_into(h, ob, &wi, 1, &h->sg_launch[3], [&] { seq_tail(h, K, h->gx.p, outer, 1); });
    MSS_CK(cudaGraphInstantiate(&h->sgraph, top, 0));
  } catch (...) {
    restore();
    throw;
  }
  restore();
  h->sg_m = K.m;
  h->sg_n = K.n;
}

// Device-driven: one graph launch per solve, one read-back at the end.
int fgmres_graph(Handle* h, const Krylov& K, const double* b, double* x, double tol, int maxit,
                 mss_result* out) {
  if (!h->sgraph || h->sg_m != K.m || h->sg_n != K.n) build_solve_graph(h, K);
  write_params(h, K, tol, maxit);
  copy_dev(h, h->gb.p, b, sizeof(double) * (size_t)K.n);
  MSS_CK(cudaGraphLaunch(h->sgraph, h->stream));
  copy_dev(h, x, h->gx.p, sizeof(double) * (size_t)K.n);
  GState s = read_state(h, K);
  const long long cycles = (s.rhs_bad || s.bnorm == 0.0) ? 0 : s.restarts + 1;
  add_launches(h->sg_launch[0] + cycles * (h->sg_launch[1] + h->sg_launch[3]) +
               (long long)s.total * h->sg_launch[2]);
  return finish(s, out);
}

}  // namespace

// Mixed form of the same stages: BF16 operator blocks and factors, FP32
// vectors and arithmetic; r and y stay FP64 (the Krylov vectors).
static void precond_apply_mixed(Handle* h, const double* r, double* y) {
  const int scheme = h->opt.scheme;
  if (scheme == MSS_ILU0) {
    last_stage_apply(h, r, (const float*)nullptr, (const float*)nullptr, y);
    return;
  }
  // each kernel that forms a V-cycle's right-hand side also writes its first
  // Jacobi sweep from zero into the V-cycle's output vector
  if (scheme == MSS_CPR) {
    gather_var(h, r, h->p, h->rTf.p, sweep0_mixed(h, h->amgP, h->vPf.p));
    vcycle_mixed(h, h->amgP, h->rTf.p, h->vPf.p, true);
    last_stage_apply(h, r, (const float*)nullptr, h->vPf.p, y);
    return;
  }
  if (scheme == MSS_CPTR) {
    gather_pair(h, r, h->rEf.p);
    vcycle_mixed(h, h->amgP, h->rEf.p, h->xEf.p);
    split_pair(h, (const float*)h->xEf.p, h->vPf.p, h->xTf.p);
    last_stage_apply(h, r, h->xTf.p, h->vPf.p, y);
    return;
  }
  if (h->opt.stage_order == MSS_STAGE_T_FIRST) {
    gather_var(h, r, h->t, h->rTf.p, sweep0_mixed(h, h->amgT, h->xTf.p));
    vcycle_mixed(h, h->amgT, h->rTf.p, h->xTf.p, true);
    csr_block_pattern_spmv_sub(h, h->aptf.p, h->xTf.p, r, h->p, h->zPf.p,
                               sweep0_mixed(h, h->amgP, h->vPf.p));
    vcycle_mixed(h, h->amgP, h->zPf.p, h->vPf.p, true);
  } else {
    gather_var(h, r, h->p, h->rTf.p, sweep0_mixed(h, h->amgP, h->vPf.p));
    vcycle_mixed(h, h->amgP, h->rTf.p, h->vPf.p, true);
    csr_block_pattern_spmv_sub(h, h->atpf.p, h->vPf.p, r, h->t, h->zPf.p,
                               sweep0_mixed(h, h->amgT, h->xTf.p));
    vcycle_mixed(h, h->amgT, h->zPf.p, h->xTf.p, true);
  }
  last_stage_apply(h, r, h->xTf.p, h->vPf.p, y);
}

// y = M^{-1} r: Algorithm 2 (CPTR3), Algorithm 1 (CPR), its CPTR form, or the
// last stage only
void precond_apply(Handle* h, const double* r, double* y) {
  TraceScope ts(h, TR_APPLY);
  if (h->opt.precision == MSS_MIXED) {
    precond_apply_mixed(h, r, y);
    return;
  }
  const int scheme = h->opt.scheme;
  if (scheme == MSS_ILU0) {
    last_stage_apply(h, r, (const double*)nullptr, (const double*)nullptr, y);
    return;
  }
  // each kernel that forms a V-cycle's right-hand side also writes its first
  // Jacobi sweep from zero into the V-cycle's output vector
  if (scheme == MSS_CPR) {
    gather_var(h, r, h->p, h->rT.p, sweep0(h, h->amgP, h->vP.p));
    vcycle(h, h->amgP, h->rT.p, h->vP.p, true);            // x = M1 r (pressure)
    last_stage_apply(h, r, (const double*)nullptr, h->vP.p, y);          // y = x + M2 (r - Abar x)
    return;
  }
  if (scheme == MSS_CPTR) {
    // Sec. 4.2: x_e = M_ee^{-1} r_e by the system AMG on (P, T) (Eq. CPTRM1),
    // then y = x + ilu(Abar)^{-1} (r - Abar x) with x = x_e at (p, t)
    gather_pair(h, r, h->rE.p);
    vcycle(h, h->amgP, h->rE.p, h->xE.p);
    split_pair(h, (const double*)h->xE.p, h->vP.p, h->xT.p);
    last_stage_apply(h, r, h->xT.p, h->vP.p, y);
    return;
  }
  if (h->opt.stage_order == MSS_STAGE_T_FIRST) {
    gather_var(h, r, h->t, h->rT.p, sweep0(h, h->amgT, h->xT.p));
    vcycle(h, h->amgT, h->rT.p, h->xT.p, true);            // x = M1 r (temperature)
    csr_block_pattern_spmv_sub(h, h->apt.p, h->xT.p, r, h->p, h->zP.p,    // z_P
                               sweep0(h, h->amgP, h->vP.p));
    vcycle(h, h->amgP, h->zP.p, h->vP.p, true);            // v = M2 z (pressure)
  } else {
    gather_var(h, r, h->p, h->rT.p, sweep0(h, h->amgP, h->vP.p));
    vcycle(h, h->amgP, h->rT.p, h->vP.p, true);            // x = M1 r (pressure)
    csr_block_pattern_spmv_sub(h, h->atp.p, h->vP.p, r, h->t, h->zP.p,    // z_T
                               sweep0(h, h->amgT, h->xT.p));
    vcycle(h, h->amgT, h->zP.p, h->xT.p, true);            // v = M2 z (temperature)
  }
  last_stage_apply(h, r, h->xT.p, h->vP.p, y);             // y = x + v + M3 u
}


int fgmres(Handle* h, const double* b, double* x, double tol, int maxit, mss_result* out) {
  Krylov K = workspace(h);
  const int st = h->opt.driver == MSS_DRIVER_GRAPH ? fgmres_graph(h, K, b, x, tol, maxit, out)
                                                   : fgmres_host(h, K, b, x, tol, maxit, out);
  check_tail(h, h->amgT);
  check_tail(h, h->amgP);
  return st;
}

}  // namespace mss
