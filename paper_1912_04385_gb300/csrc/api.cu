// api.cu -- the C-ABI of libmss (include/mss.h): argument checks, set-up
// orchestration (Sec. 4 scaling, subsystem extraction, AMG, last stage) and
// the solve entry points. Internal errors become status codes here.
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <new>

#include <thread>
#include <exception>
#include <memory>
#include <string>
#include "common.cuh"

struct mss_handle {
  mss::Handle h;
};

using namespace mss;

namespace {

template <class F>
int guarded(mss_handle* hh, F&& f) {
  try {
    f();
    if (hh) hh->h.last_error.clear();
    return MSS_OK;
  } catch (const Error& e) {
    if (hh) hh->h.last_error = e.msg;
    return e.code;
  } catch (const std::bad_alloc&) {
    if (hh) hh->h.last_error = "host allocation failed";
    return MSS_ERR_OOM;
  } catch (...) {
    if (hh) hh->h.last_error = "unexpected internal error";
    return MSS_ERR_CUDA;
  }
}

void check_options(const mss_options& o) {
  auto bad = [](const char* what) { fail(MSS_ERR_INVALID_ARG, std::string("option ") + what); };
  if (o.scheme < MSS_CPTR3 || o.scheme > MSS_CPTR) bad("scheme");
  if (o.stage_order != MSS_STAGE_T_FIRST && o.stage_order != MSS_STAGE_P_FIRST)
    bad("stage_order");
  if (o.stage3 != MSS_BILU0 && o.stage3 != MSS_BLOCK_JACOBI) bad("stage3");
  if (o.ilu_order != MSS_MULTICOLOR && o.ilu_order != MSS_STRIPS && o.ilu_order != MSS_STRIPS_JP)
    bad("ilu_order");
  if (o.ilu_strip < 1 || o.ilu_strip > 1024) bad("ilu_strip (1..1024)");
  if (o.orthog != MSS_CGS1 && o.orthog != MSS_CGS2) bad("orthog");
  if (o.smoother != MSS_JACOBI && o.smoother != MSS_CHEBYSHEV && o.smoother != MSS_MCSGS)
    bad("smoother");
  if (o.nu_pre < 0 || o.nu_pre > 16 || o.nu_post < 0 || o.nu_post > 16) bad("nu_pre/nu_post");
  if (o.smoother == MSS_JACOBI && o.nu_pre < 1) bad("nu_pre (Jacobi needs >= 1)");
  if (o.cheb_degree < 1 || o.cheb_degree > 16) bad("cheb_degree");
  if (o.amg_max_coarse < 1 || o.amg_max_coarse > 8192) bad("amg_max_coarse");
  if (o.amg_max_levels < 1 || o.amg_max_levels > 25) bad("amg_max_levels");
  if (o.interp_max_elems < 0) bad("interp_max_elems");
  if (o.restart < 1 || o.restart > 120) bad("restart (1..120)");
  if (o.precision != MSS_FP64 && o.precision != MSS_MIXED) bad("precision");
  if (o.driver != MSS_DRIVER_HOST && o.driver != MSS_DRIVER_GRAPH) bad("driver");
  if (o.factor_form < MSS_FACTOR_AUTO || o.factor_form > MSS_FACTOR_LANES) bad("factor_form");
  if (!(o.amg_theta > 0.0 && o.amg_theta <= 1.0)) bad("amg_theta");
  if (!(o.jacobi_omega > 0.0 && o.jacobi_omega < 2.0)) bad("jacobi_omega");
  if (!(o.cheb_lo_ratio > 1.0) || !(o.cheb_hi_factor > 0.0)) bad("Chebyshev interval");
  if (o.learned_interp != nullptr && o.scheme != MSS_CPTR3) bad("learned_interp (CPTR3 only)");
}

// Worker handle i: its own non-blocking stream, allocations from the device
// pool, the main handle's sizes and options. The workers build the AMG
// hierarchies, the longer branches of the set-up; their streams take the
// device's highest priority, so their blocks are dispatched ahead of the
// factorisation's whenever both wait for an SM.
Handle* worker(Handle& H, int i) {
  if (!H.aux[i]) {
    std::unique_ptr<Handle> a(new Handle());
    a->device = H.device;
    a->num_sms = H.num_sms;
    int least = 0, greatest = 0;
    MSS_CK(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    MSS_CK(cudaStreamCreateWithPriority(&a->owned.s, cudaStreamNonBlocking, greatest));
    a->stream = a->owned.s;
    H.aux[i] = std::move(a);
  }
  Handle* a = H.aux[i].get();
  a->opt = H.opt;
  a->N = H.N;
  a->nnzb = H.nnzb;
  a->nb = H.nb;
  a->p = H.p;
  a->t = H.t;
  return a;
}

// Makes stream `later` wait for the work queued so far on stream `first`.
void order_streams(cudaStream_t first, cudaStream_t later) {
  cudaEvent_t e;
  MSS_CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  MSS_CK(cudaEventRecord(e, first));
  MSS_CK(cudaStreamWaitEvent(later, e, 0));
  MSS_CK(cudaEventDestroy(e));
}

// Runs set-up tasks on worker handles in threads; join() waits for them,
// orders the main stream after their streams and rethrows the first error.
struct Fork {
  Handle& H;
  std::thread th[2];
  std::exception_ptr err[2];
  bool used[2] = {false, false};
  explicit Fork(Handle& h) : H(h) {}
  template <class F>
  void run(int i, F fn) {
    Handle* a = worker(H, i);
    order_streams(H.stream, a->stream);   // the worker reads what H's stream wrote
    used[i] = true;
    MSS_CK(cudaGetDevice(&a->device));
    const int dev = a->device;
    th[i] = std::thread([this, i, a, dev, fn] {
      try {
        MSS_CK(cudaSetDevice(dev));
        fn(a);
      } catch (...) {
        err[i] = std::current_exception();
      }
    });
  }
  void join() {
    for (int i = 0; i < 2; ++i)
      if (th[i].joinable()) th[i].join();
    for (int i = 0; i < 2; ++i)
      if (used[i]) order_streams(H.aux[i]->stream, H.stream);
    for (int i = 0; i < 2; ++i)
      if (err[i]) std::rethrow_exception(err[i]);
  }
  ~Fork() {
    for (int i = 0; i < 2; ++i)
      if (th[i].joinable()) th[i].join();
  }
};

void release_setup(Handle& H) {
  H.ready = false;
  // hierarchy memory came from the workers' streams: free it there only
  // after everything queued on the handle's stream
  for (auto& a : H.aux)
    if (a) order_streams(H.stream, a->stream);
  if (H.sgraph) {   // the solve graph holds pointers into the set-up
    cudaGraphExecDestroy(H.sgraph);
    H.sgraph = nullptr;
  }
  H.amgT = Hierarchy();
  H.amgP = Hierarchy();
  H.rp.release(); H.ci.release(); H.diag.release();
  H.abar.release(); H.wrows.release(); H.apt.release(); H.atp.release();
  H.colour.release(); H.perm.release(); H.iperm.release();
  H.frp.release(); H.fpos.release(); H.fcell.release(); H.fdp.release(); H.fsrc.release();
  H.st_first.release(); H.st_len.release(); H.sc_start.clear();
  H.fslo.release(); H.fshi.release(); H.cL.release(); H.cG.release(); H.cflag.release();
  H.fv.release(); H.fdinv.release(); H.fcs.release();
  H.rT.release(); H.xT.release(); H.zP.release(); H.vP.release(); H.w.release();
  H.rE.release(); H.xE.release(); H.rEf.release(); H.xEf.release();
  H.fvh.release(); H.fdinvh.release(); H.cLh.release(); H.cGh.release();
  H.fcsf.release(); H.aptf.release(); H.atpf.release();
  H.rTf.release(); H.xTf.release(); H.zPf.release(); H.vPf.release(); H.wf.release();
  H.cstart.clear();
  H.ncol = 0;
}

void need_ready(const Handle& H) {
  if (!H.ready) fail(MSS_ERR_NOT_SETUP, "mss_setup has not completed on this handle");
}

// The value-dependent set-up on a validated pattern (H.rp, H.ci, H.diag):
// the scaling and extraction (Eqs. CPR, CPTR31, CPTR32), the two AMG
// hierarchies on worker threads beside the last stage on this thread (with
// its ordering and factor pattern when `ordering`, else on the existing
// ones), the reduced-precision copies and the fused coarse levels. cfT / cfP:
// C/F splits kept from an earlier set-up (Newton-loop reuse), or null.
void numeric_setup(Handle& H, const double* vals, bool ordering, std::vector<DBuf<int>>* cfT,
                   std::vector<DBuf<int>>* cfP) {
  const mss_options& o = H.opt;
  const int N = H.N, nnzb = H.nnzb;
  Handle* h = &H;
  // B_PP and C_TT (the hierarchies' level 0) and the P-T couplings of CPTR3
  // are written by the scaling kernel beside Abar
  DBuf<double> bpp, ctt, bee;
  {
    TraceScope ts(h, TR_SETUP_SCALE);
    Extract ex;
    if (o.scheme == MSS_CPR || o.scheme == MSS_CPTR3) {
      bpp.reset(h, nnzb);
      ex.pp = bpp.p;
    }
    if (o.scheme == MSS_CPTR3) {
      if (H.apt.n != (size_t)nnzb) H.apt.reset(h, nnzb);
      if (H.atp.n != (size_t)nnzb) H.atp.reset(h, nnzb);
      ctt.reset(h, nnzb);
      ex.tt = ctt.p;
      ex.pt = H.apt.p;
      ex.tp = H.atp.p;
    }
    // left scaling (Eq. splitPrec1 with Eq. CPR or Eqs. CPTR31/CPTR32)
    build_scaling(h, vals, H.col_major, ex);
  }
  // The scalar subsystems' AMG hierarchies and the last-stage factorisation
  // depend only on Abar: the hierarchies are built by worker threads on
  // their own streams while this thread factorises on the handle's stream.
  {
    TraceScope ts(h, TR_SETUP_AMG);
    if (o.scheme == MSS_CPTR) {
      bee.reset(h, (size_t)4 * nnzb);
      extract_pair(h, bee.p);                     // B_ee (Eq. CPTR1)
    }
    // MSS_SETUP_TIMES=1 prints the phases' host times (diagnostics)
    static const bool times = std::getenv("MSS_SETUP_TIMES") != nullptr;
    const auto tf = std::chrono::steady_clock::now();
    auto since = [&] {
      return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tf)
          .count();
    };
    double tp = 0, tt = 0, tb = 0;
    Fork fork(H);
    if (o.scheme == MSS_CPTR)
      fork.run(0, [&](Handle* a) {
        amg_build_system(a, H.amgP, N, nnzb, H.rp.p, H.ci.p, bee.p);
        if (times) {
          cudaStreamSynchronize(a->stream);
          tp = since();
        }
      });
    if (o.scheme == MSS_CPR || o.scheme == MSS_CPTR3)
      fork.run(0, [&](Handle* a) {
        amg_build(a, H.amgP, N, nnzb, H.rp.p, H.ci.p, bpp.p, nullptr, cfP);
        if (times) {
          cudaStreamSynchronize(a->stream);
          tp = since();
        }
      });
    if (o.scheme == MSS_CPTR3)
      fork.run(1, [&](Handle* a) {
        amg_build(a, H.amgT, N, nnzb, H.rp.p, H.ci.p, ctt.p,
                  static_cast<const float*>(o.learned_interp), cfT);
        if (times) {
          cudaStreamSynchronize(a->stream);
          tt = since();
        }
      });
    std::exception_ptr mine;
    try {
      if (ordering) bilu_setup(h);                // last stage
      else bilu_refactor(h);
      if (times) {
        cudaStreamSynchronize(H.stream);
        tb = since();
      }
    } catch (...) {
      mine = std::current_exception();
    }
    fork.join();                                  // rethrows a worker's error
    if (mine) std::rethrow_exception(mine);
    if (times)
      std::fprintf(stderr, "mss setup: P hierarchy %.2f, T hierarchy %.2f, last stage %.2f, "
                           "join %.2f ms after the fork\n", tp, tt, tb, since());
  }
  if (H.rT.n != (size_t)N) {
    H.rT.reset(h, N);
    H.xT.reset(h, N);
    H.zP.reset(h, N);
    H.vP.reset(h, N);
    H.w.reset(h, (size_t)N * H.nb);
  }
  if (o.scheme == MSS_CPTR && H.rE.n != (size_t)2 * N) {
    H.rE.reset(h, (size_t)2 * N);
    H.xE.reset(h, (size_t)2 * N);
  }
  if (o.precision == MSS_MIXED) {
    // reduced-precision copies of everything the preconditioner reads
    TraceScope ts(h, TR_SETUP_BILU);
    if (H.amgP.present()) pack_hierarchy_mixed(h, H.amgP);
    if (H.amgT.present()) pack_hierarchy_mixed(h, H.amgT);
    if (o.scheme == MSS_CPTR3) {
      H.aptf.reset(h, nnzb);
      to_float(h, H.apt.p, H.aptf.p, nnzb);
      H.atpf.reset(h, nnzb);
      to_float(h, H.atp.p, H.atpf.p, nnzb);
    }
    pack_last_stage_mixed(h);
    if (H.rTf.n != (size_t)N) {
      H.rTf.reset(h, N);
      H.xTf.reset(h, N);
      H.zPf.reset(h, N);
      H.vPf.reset(h, N);
    }
    if (o.scheme == MSS_CPTR && H.rEf.n != (size_t)2 * N) {
      H.rEf.reset(h, (size_t)2 * N);
      H.xEf.reset(h, (size_t)2 * N);
    }
  }
  if (H.amgT.present()) prepare_tail(h, H.amgT);
  if (H.amgP.present()) prepare_tail(h, H.amgP);
  MSS_CK(cudaStreamSynchronize(H.stream));
}

void do_setup(Handle& H, const mss_bsr* J, int nb, mss_layout layout, const mss_options* opt) {
  auto t0 = std::chrono::steady_clock::now();
  if (!J || !J->row_ptr || !J->col_idx || !J->vals) fail(MSS_ERR_INVALID_ARG, "null matrix");
  if (J->n_rows < 1 || J->nnzb < J->n_rows) fail(MSS_ERR_INVALID_ARG, "bad matrix sizes");
  if (nb < 2 || nb > MSS_MAX_NB) fail(MSS_ERR_INVALID_ARG, "nb must be in [2, 16]");
  if (layout.p_idx < 0 || layout.p_idx >= nb || layout.t_idx < 0 || layout.t_idx >= nb ||
      layout.p_idx == layout.t_idx)
    fail(MSS_ERR_INVALID_ARG, "p_idx and t_idx must be distinct indices in [0, nb)");
  mss_options o;
  if (opt) o = *opt;
  else mss_options_default(&o);
  check_options(o);
  release_setup(H);
  H.opt = o;
  H.N = J->n_rows;
  H.nnzb = J->nnzb;
  H.nb = nb;
  H.p = layout.p_idx;
  H.t = layout.t_idx;
  H.col_major = layout.col_major_blocks != 0;
  const int N = H.N, nnzb = H.nnzb;
  Handle* h = &H;
  H.rp.reset(h, N + 1);
  H.ci.reset(h, nnzb);
  H.diag.reset(h, N);
  {
    TraceScope ts(h, TR_SETUP_SCALE);
    copy_dev(h, H.rp.p, J->row_ptr, sizeof(int) * ((size_t)N + 1));
    copy_dev(h, H.ci.p, J->col_idx, sizeof(int) * (size_t)nnzb);
    validate_pattern(h, H.rp.p, H.ci.p, N, nnzb, H.diag.p);
  }
  H.wrows.reset(h, (size_t)N * 2 * nb);
  H.abar.reset(h, (size_t)nnzb * nb * nb);
  numeric_setup(H, J->vals, true, nullptr, nullptr);
  H.J = *J;
  H.ready = true;
  H.setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0)
                   .count();
}

__global__ void k_same_pattern(int N, int nnzb, const int* __restrict__ rpa,
                               const int* __restrict__ cia, const int* __restrict__ rpb,
                               const int* __restrict__ cib, int* __restrict__ diff) {
  const long long n = (long long)(N + 1 > nnzb ? N + 1 : nnzb);
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    if (k <= N && rpa[k] != rpb[k]) *diff = 1;
    if (k < nnzb && cia[k] != cib[k]) *diff = 1;
  }
}

// New values on the set-up's pattern (Newton-loop reuse, Sec. 2.5): the
// pattern check, then the numeric set-up on the kept symbolic one (pattern,
// diagonal positions, last-stage ordering and factor pattern); with
// MSS_REUSE_COARSENING the AMG levels also keep their C/F splits.
void do_update(Handle& H, const mss_bsr* J, int reuse) {
  auto t0 = std::chrono::steady_clock::now();
  need_ready(H);
  if (!J || !J->row_ptr || !J->col_idx || !J->vals) fail(MSS_ERR_INVALID_ARG, "null matrix");
  if (reuse != MSS_REUSE_PATTERN && reuse != MSS_REUSE_COARSENING)
    fail(MSS_ERR_INVALID_ARG, "reuse must be MSS_REUSE_PATTERN or MSS_REUSE_COARSENING");
  if (J->n_rows != H.N || J->nnzb != H.nnzb)
    fail(MSS_ERR_INVALID_ARG, "the matrix sizes differ from the set-up's");
  if (reuse == MSS_REUSE_COARSENING && H.opt.scheme == MSS_CPTR)
    fail(MSS_ERR_INVALID_ARG, "MSS_REUSE_COARSENING keeps scalar AMG splits; CPTR's system "
                              "AMG is rebuilt (use MSS_REUSE_PATTERN)");
  Handle* h = &H;
  {
    DBuf<int> diff(h, 1);
    fill_int(h, diff.p, 0, 1);
    const long long n = std::max((long long)H.N + 1, (long long)H.nnzb);
    unsigned g = grid_for(n, 256);
    if (g > 4096u) g = 4096u;
    k_same_pattern<<<g, 256, 0, h->stream>>>(H.N, H.nnzb, H.rp.p, H.ci.p, J->row_ptr, J->col_idx,
                                             diff.p);
    MSS_LAUNCH_CK("k_same_pattern");
    if (read_int(h, diff.p) != 0)
      fail(MSS_ERR_INVALID_ARG, "the pattern differs from the set-up's (call mss_setup)");
  }
  H.ready = false;
  if (H.sgraph) {   // the solve graph holds pointers into the old hierarchies
    cudaGraphExecDestroy(H.sgraph);
    H.sgraph = nullptr;
  }
  std::vector<DBuf<int>> cfT, cfP;
  if (reuse == MSS_REUSE_COARSENING) {
    for (auto& L : H.amgT.lev) cfT.push_back(std::move(L.cf));
    for (auto& L : H.amgP.lev) cfP.push_back(std::move(L.cf));
  }
  // the old hierarchies came from the workers' streams: free them there only
  // after everything queued on the handle's stream
  for (auto& a : H.aux)
    if (a) order_streams(H.stream, a->stream);
  H.amgT = Hierarchy();
  H.amgP = Hierarchy();
  numeric_setup(H, J->vals, false, cfT.empty() ? nullptr : &cfT, cfP.empty() ? nullptr : &cfP);
  H.J = *J;
  H.ready = true;
  H.setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0)
                   .count();
}


Hierarchy& pick(Handle& H, int which) {
  if (which == 0 && H.amgT.present()) return H.amgT;
  if (which == 1 && H.amgP.present()) return H.amgP;
  fail(MSS_ERR_INVALID_ARG, "no AMG stage " + std::to_string(which) + " in this scheme");
}

int solve_impl(Handle& H, const mss_bsr* J, const double* b, double* x, double tol, int maxit,
               mss_result* out) {
  auto t0 = std::chrono::steady_clock::now();
  need_ready(H);
  if (!J || J->n_rows != H.J.n_rows || J->nnzb != H.J.nnzb || J->row_ptr != H.J.row_ptr ||
      J->col_idx != H.J.col_idx || J->vals != H.J.vals)
    fail(MSS_ERR_NOT_SETUP, "the matrix differs from the one passed to mss_setup");
  if (!b || !x || b == x) fail(MSS_ERR_INVALID_ARG, "b and x must be distinct device vectors");
  if (!(tol >= 0.0) || maxit < 0) fail(MSS_ERR_INVALID_ARG, "tol >= 0 and maxit >= 0 required");
  mss_result r{};
  int st = fgmres(&H, b, x, tol, maxit, &r);
  MSS_CK(cudaStreamSynchronize(H.stream));
  r.setup_ms = H.setup_ms;
  r.solve_ms =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  r.status = st;
  if (out) *out = r;
  return st;
}

}  // namespace

namespace mss {
void setup_handle(Handle& H, const mss_bsr* J, int nb, mss_layout layout,
                  const mss_options* opt) {
  do_setup(H, J, nb, layout, opt);
}
int solve_handle(Handle& H, const mss_bsr* J, const double* b, double* x, double tol, int maxit,
                 mss_result* out) {
  return solve_impl(H, J, b, x, tol, maxit, out);
}
}  // namespace mss

// The graph owns a private handle (its own stream, memory from the device
// pool), so it does not depend on the lifetime of the handle it came from.
struct mss_gnn {
  std::unique_ptr<Handle> h;
  GnnGraph* g = nullptr;
  std::string last_error;
  ~mss_gnn() {
    if (h) cudaStreamSynchronize(h->stream);
    if (g) gnn_destroy(g);
  }
};

template <class F>
static int gnn_guarded(mss_gnn* G, F&& f) {
  try {
    f();
    G->last_error.clear();
    return MSS_OK;
  } catch (const Error& e) {
    G->last_error = e.msg;
    return e.code;
  } catch (const std::bad_alloc&) {
    G->last_error = "host allocation failed";
    return MSS_ERR_OOM;
  } catch (...) {
    G->last_error = "unexpected internal error";
    return MSS_ERR_CUDA;
  }
}

extern "C" {

int mss_options_default(mss_options* o) {
  if (!o) return MSS_ERR_INVALID_ARG;
  *o = mss_options{};
  o->scheme = MSS_CPTR3;
  o->stage_order = MSS_STAGE_T_FIRST;
  o->stage3 = MSS_BILU0;
  o->ilu_order = MSS_STRIPS;
  o->ilu_strip = 32;
  o->orthog = MSS_CGS1;
  o->smoother = MSS_JACOBI;
  o->nu_pre = 2;    // HSL_MI20 defaults (Sec. 5.1): two pre- and two post-smoothing
  o->nu_post = 2;   // sweeps, Jacobi damping 0.8
  o->cheb_degree = 2;
  o->amg_max_coarse = 1000;
  o->amg_max_levels = 25;
  o->interp_max_elems = 4;
  o->restart = 30;
  o->precision = MSS_FP64;
  o->driver = MSS_DRIVER_HOST;
  o->factor_form = MSS_FACTOR_AUTO;
  o->amg_theta = 0.25;
  o->jacobi_omega = 0.8;
  o->cheb_lo_ratio = 30.0;
  o->cheb_hi_factor = 1.0;
  o->seed = 0x5eedULL;
  o->learned_interp = nullptr;
  return MSS_OK;
}

int mss_create(mss_handle** out, void* cuda_stream, mss_alloc_fn alloc, mss_free_fn free_fn,
               void* alloc_ctx) {
  if (!out) return MSS_ERR_INVALID_ARG;
  *out = nullptr;
  if ((alloc == nullptr) != (free_fn == nullptr)) return MSS_ERR_INVALID_ARG;
  mss_handle* hh = new (std::nothrow) mss_handle();
  if (!hh) return MSS_ERR_OOM;
  int st = guarded(hh, [&] {
    Handle& H = hh->h;
    H.stream = static_cast<cudaStream_t>(cuda_stream);
    H.alloc = alloc;
    H.free_fn = free_fn;
    H.ctx = alloc_ctx;
    MSS_CK(cudaGetDevice(&H.device));
    MSS_CK(cudaDeviceGetAttribute(&H.num_sms, cudaDevAttrMultiProcessorCount, H.device));
    mss_options_default(&H.opt);
  });
  if (st != MSS_OK) {
    delete hh;
    return st;
  }
  *out = hh;
  return MSS_OK;
}

void mss_destroy(mss_handle* hh) {
  if (!hh) return;
  cudaStreamSynchronize(hh->h.stream);
  delete hh;
  trim_pools();
}

int mss_setup(mss_handle* hh, const mss_bsr* J, int nb, mss_layout layout,
              const mss_options* opt) {
  if (!hh) return MSS_ERR_INVALID_ARG;
  return guarded(hh, [&] { do_setup(hh->h, J, nb, layout, opt); });
}

int mss_update_values(mss_handle* hh, const mss_bsr* J, int reuse) {
  if (!hh) return MSS_ERR_INVALID_ARG;
  return guarded(hh, [&] { do_update(hh->h, J, reuse); });
}

int mss_scale_rhs(mss_handle* hh, const double* b, double* bbar) {
  if (!hh) return MSS_ERR_INVALID_ARG;
  return guarded(hh, [&] {
    need_ready(hh->h);
    if (!b || !bbar) fail(MSS_ERR_INVALID_ARG, "null vector");
    scale_vector(&hh->h, b, bbar);
    MSS_LAUNCH_CK("mss_scale_rhs");
  });
}

int mss_spmv(mss_handle* hh, const double* x, double* y) {
  if (!hh) return MSS_ERR_INVALID_ARG;
  return guarded(hh, [&] {
    need_ready(hh->h);
    if (!x || !y || x == y) fail(MSS_ERR_INVALID_ARG, "x and y must be distinct");
    bsr_spmv(&hh->h, x, y);
  });
}

int mss_apply(mss_handle* hh, const double* r, double* y) {
  if (!hh) return MSS_ERR_INVALID_ARG;
  return guarded(hh, [&] {
    need_ready(hh->h);
    if (!r || !y || r == y) fail(MSS_ERR_INVALID_ARG, "r and y must be distinct");
    precond_apply(&hh->h, r, y);
    check_tail(&hh->h, hh->h.amgT);
    check_tail(&hh->h, hh->h.amgP);
  });
}

int mss_stage_apply(mss_handle* hh, int which, const double* r, double* y) {
  if (!hh) return MSS_ERR_INVALID_ARG;
  return guarded(hh, [&] {
    Handle& H = hh->h;
    need_ready(H);
    if (!r || !y || r == y) fail(MSS_ERR_INVALID_ARG, "r and y must be distinct");
    if (which == 2) {
      last_stage_apply(&H, r, (const double*)nullptr, (const double*)nullptr, y);
      return;
    }
    Hierarchy& A = pick(H, which);
    if (A.bs == 2) {   // CPTR's first stage (Eq. CPTRM1) on (P, T)
      gather_pair(&H, r, H.rE.p);
      vcycle(&H, A, H.rE.p, H.xE.p);
      scatter_pair_zero(&H, H.xE.p, y);
      return;
    }
    int var = which == 0 ? H.t : H.p;
    gather_var(&H, r, var, H.rT.p);
    vcycle(&H, A, H.rT.p, H.xT.p);
    scatter_var_zero(&H, H.xT.p, var, y);
    check_tail(&H, A);
  });
}

int mss_fgmres_solve(mss_handle* hh, const mss_bsr* J, const double* b, double* x, double tol,
                     int maxit, mss_result* out) {
  if (!hh) return MSS_ERR_INVALID_ARG;
  int st = MSS_OK;
  int g = guarded(hh, [&] { st = solve_impl(hh->h, J, b, x, tol, maxit, out); });
  if (g != MSS_OK) {
    if (out) out->status = g;
    return g;
  }
  if (st != MSS_OK) hh->h.last_error = mss_status_string(st);
  return st;
}

int mss_solve_host(mss_handle* hh, const mss_bsr* Jh, int nb, mss_layout layout,
                   const mss_options* opt, const double* b_host, double* x_host, double tol,
                   int maxit, mss_result* out) {
  if (!hh) return MSS_ERR_INVALID_ARG;
  int st = MSS_OK;
  int g = guarded(hh, [&] {
    Handle& H = hh->h;
    Handle* h = &H;
    if (!Jh || !Jh->row_ptr || !Jh->col_idx || !Jh->vals || !b_host || !x_host)
      fail(MSS_ERR_INVALID_ARG, "null host pointer");
    if (Jh->n_rows < 1 || Jh->nnzb < Jh->n_rows || nb < 2 || nb > MSS_MAX_NB)
      fail(MSS_ERR_INVALID_ARG, "bad sizes");
    const size_t N = (size_t)Jh->n_rows, nnzb = (size_t)Jh->nnzb, nb2 = (size_t)nb * nb;
    if (H.host_rp.n < N + 1) H.host_rp.reset(h, N + 1);
    if (H.host_ci.n < nnzb) H.host_ci.reset(h, nnzb);
    if (H.host_b.n < N * nb) H.host_b.reset(h, N * nb);
    if (H.host_x.n < N * nb) H.host_x.reset(h, N * nb);
    MSS_CK(cudaMemcpyAsync(H.host_rp.p, Jh->row_ptr, sizeof(int) * (N + 1),
                           cudaMemcpyHostToDevice, H.stream));
    MSS_CK(cudaMemcpyAsync(H.host_ci.p, Jh->col_idx, sizeof(int) * nnzb, cudaMemcpyHostToDevice,
                           H.stream));
    // The block values are read once, by the scaling kernels: when they sit in
    // pinned host memory that the device can address, those kernels read them
    // in place over the host link instead of after a staging copy.
    const double* vals = nullptr;
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, Jh->vals) == cudaSuccess && at.type == cudaMemoryTypeHost &&
        at.devicePointer != nullptr) {
      vals = static_cast<const double*>(at.devicePointer);
    } else {
      cudaGetLastError();   // pageable memory: not an error, copy it
      if (H.host_vals.n < nnzb * nb2) H.host_vals.reset(h, nnzb * nb2);
      MSS_CK(cudaMemcpyAsync(H.host_vals.p, Jh->vals, sizeof(double) * nnzb * nb2,
                             cudaMemcpyHostToDevice, H.stream));
      vals = H.host_vals.p;
    }
    MSS_CK(cudaMemcpyAsync(H.host_b.p, b_host, sizeof(double) * N * nb, cudaMemcpyHostToDevice,
                           H.stream));
    mss_bsr Jd{Jh->n_rows, Jh->nnzb, H.host_rp.p, H.host_ci.p, vals};
    do_setup(H, &Jd, nb, layout, opt);
    st = solve_impl(H, &Jd, H.host_b.p, H.host_x.p, tol, maxit, out);
    MSS_CK(cudaMemcpyAsync(x_host, H.host_x.p, sizeof(double) * N * nb, cudaMemcpyDeviceToHost,
                           H.stream));
    MSS_CK(cudaStreamSynchronize(H.stream));
  });
  if (g != MSS_OK) {
    if (out) out->status = g;
    return g;
  }
  return st;
}

int mss_condense(mss_handle* hh, const mss_full* J, const double* r1, const double* r2,
                 double* a, double* b) {
  if (!hh) return MSS_ERR_INVALID_ARG;
  return guarded(hh, [&] { condense(&hh->h, J, r1, r2, a, b); });
}

int mss_recover(mss_handle* hh, const mss_full* J, const double* r2, const double* d1,
                double* d2) {
  if (!hh) return MSS_ERR_INVALID_ARG;
  return guarded(hh, [&] { recover(&hh->h, J, r2, d1, d2); });
}

int mss_residual_norm(mss_handle* hh, const mss_bsr* J, int nb, const double* b, const double* x,
                      double* norms) {
  if (!hh) return MSS_ERR_INVALID_ARG;
  return guarded(hh, [&] { residual_norm(&hh->h, J, nb, b, x, norms); });
}

int mss_residual_norm_noalloc(mss_handle* hh, const mss_bsr* J, int nb, const double* b,
                              const double* x, double* norms) {
  if (!hh) return MSS_ERR_INVALID_ARG;
  return guarded(hh, [&] { residual_norm_noalloc(&hh->h, J, nb, b, x, norms); });
}

int mss_get_scaled(mss_handle* hh, double* abar) {
  if (!hh) return MSS_ERR_INVALID_ARG;
  return guarded(hh, [&] {
    Handle& H = hh->h;
    need_ready(H);
    if (!abar) fail(MSS_ERR_INVALID_ARG, "null output");
    copy_dev(&H, abar, H.abar.p, sizeof(double) * H.abar.n);
    MSS_CK(cudaStreamSynchronize(H.stream));
  });
}

int mss_amg_num_levels(mss_handle* hh, int which) {
  if (!hh || !hh->h.ready) return 0;
  if (which == 0) return (int)hh->h.amgT.lev.size();
  if (which == 1) return (int)hh->h.amgP.lev.size();
  return 0;
}

int mss_amg_level_sizes(mss_handle* hh, int which, int level, int32_t* sizes) {
  if (!hh) return MSS_ERR_INVALID_ARG;
  return guarded(hh, [&] {
    Handle& H = hh->h;
    need_ready(H);
    Hierarchy& A = pick(H, which);
    if (level < 0 || level >= (int)A.lev.size() || !sizes)
      fail(MSS_ERR_INVALID_ARG, "bad level");
    const Level& L = A.lev[level];
    bool last = level == (int)A.lev.size() - 1;
    sizes[0] = L.n;
    sizes[1] = L.nnz;
    sizes[2] = last ? 0 : L.nnzP;
  });
}

int mss_amg_level_copy(mss_handle* hh, int which, int level, int32_t* arp, int32_t* aci,
                       double* av, int32_t* cf, int32_t* prp, int32_t* pci, double* pv) {
  if (!hh) return MSS_ERR_INVALID_ARG;
  return guarded(hh, [&] {
    Handle& H = hh->h;
    need_ready(H);
    Hierarchy& A = pick(H, which);
    if (level < 0 || level >= (int)A.lev.size()) fail(MSS_ERR_INVALID_ARG, "bad level");
    const Level& L = A.lev[level];
    bool last = level == (int)A.lev.size() - 1;
    if (!arp || !aci || !av) fail(MSS_ERR_INVALID_ARG, "null output");
    copy_dev(&H, arp, L.rp.p, sizeof(int) * ((size_t)L.n + 1));
    copy_dev(&H, aci, L.ci.p, sizeof(int) * (size_t)L.nnz);
    copy_dev(&H, av, L.v.p, sizeof(double) * (size_t)L.nnz);
    if (!last) {
      if (!cf || !prp || !pci || !pv) fail(MSS_ERR_INVALID_ARG, "null output");
      copy_dev(&H, cf, L.cf.p, sizeof(int) * (size_t)L.n);
      copy_dev(&H, prp, L.prp.p, sizeof(int) * ((size_t)L.n + 1));
      copy_dev(&H, pci, L.pci.p, sizeof(int) * (size_t)L.nnzP);
      copy_dev(&H, pv, L.pv.p, sizeof(double) * (size_t)L.nnzP);
    }
    MSS_CK(cudaStreamSynchronize(H.stream));
  });
}

int mss_bilu_num_colours(mss_handle* hh, int32_t* ncolours) {
  if (!hh || !ncolours) return MSS_ERR_INVALID_ARG;
  return guarded(hh, [&] {
    need_ready(hh->h);
    *ncolours = hh->h.ncol;
  });
}

int mss_bilu_ordering(mss_handle* hh, int32_t* colour, int32_t* perm) {
  if (!hh) return MSS_ERR_INVALID_ARG;
  return guarded(hh, [&] {
    Handle& H = hh->h;
    need_ready(H);
    if (colour) copy_dev(&H, colour, H.colour.p, sizeof(int) * (size_t)H.N);
    if (perm) copy_dev(&H, perm, H.perm.p, sizeof(int) * (size_t)H.N);
    MSS_CK(cudaStreamSynchronize(H.stream));
  });
}

int mss_bilu_factors(mss_handle* hh, double* fv, double* fdinv) {
  if (!hh) return MSS_ERR_INVALID_ARG;
  return guarded(hh, [&] {
    Handle& H = hh->h;
    need_ready(H);
    if (H.opt.stage3 == MSS_BLOCK_JACOBI)
      fail(MSS_ERR_INVALID_ARG, "block Jacobi has no ILU factors");
    if (fv) copy_dev(&H, fv, H.fv.p, sizeof(double) * H.fv.n);
    if (fdinv) copy_dev(&H, fdinv, H.fdinv.p, sizeof(double) * H.fdinv.n);
    MSS_CK(cudaStreamSynchronize(H.stream));
  });
}

long long mss_kernel_launches(int reset) { return launch_count(reset != 0); }

int mss_probe_wait_limit(mss_handle* hh, int32_t* timed_out) {
  if (!hh || !timed_out) return MSS_ERR_INVALID_ARG;
  return guarded(hh, [&] { *timed_out = wait_limit_probe(&hh->h) != 0 ? 1 : 0; });
}

int mss_trace_enable(mss_handle* hh, int enable) {
  if (!hh) return MSS_ERR_INVALID_ARG;
  return guarded(hh, [&] {
    Handle& H = hh->h;
    trace_drain(&H);
    H.trace = enable != 0;
  });
}

int mss_trace_read(mss_handle* hh, int kind, int64_t* launches, double* ms, int reset) {
  if (!hh || kind < 0 || kind >= TR_KINDS) return MSS_ERR_INVALID_ARG;
  return guarded(hh, [&] {
    Handle& H = hh->h;
    trace_drain(&H);
    if (launches) *launches = H.trace_n[kind];
    if (ms) *ms = H.trace_ms[kind];
    if (reset) {
      H.trace_n[kind] = 0;
      H.trace_ms[kind] = 0.0;
    }
  });
}

const char* mss_status_string(int s) {
  switch (s) {
    case MSS_OK: return "MSS_OK";
    case MSS_ERR_INVALID_ARG: return "MSS_ERR_INVALID_ARG";
    case MSS_ERR_SINGULAR_BLOCK: return "MSS_ERR_SINGULAR_BLOCK";
    case MSS_ERR_NOT_CONVERGED: return "MSS_ERR_NOT_CONVERGED";
    case MSS_ERR_BREAKDOWN: return "MSS_ERR_BREAKDOWN";
    case MSS_ERR_CUDA: return "MSS_ERR_CUDA";
    case MSS_ERR_OOM: return "MSS_ERR_OOM";
    case MSS_ERR_AMG: return "MSS_ERR_AMG";
    case MSS_ERR_NOT_SETUP: return "MSS_ERR_NOT_SETUP";
    default: return "MSS_ERR_UNKNOWN";
  }
}

const char* mss_last_error(const mss_handle* hh) {
  if (!hh) return "null handle";
  return hh->h.last_error.c_str();
}


/* ---- learned temperature interpolation ------------------------------------ */
int mss_gnn_num_params(void) { return gnn_num_params(); }

int mss_gnn_create(mss_handle* hh, mss_gnn** out) {
  if (!hh || !out) return MSS_ERR_INVALID_ARG;
  *out = nullptr;
  return guarded(hh, [&] {
    Handle& H = hh->h;
    need_ready(H);
    if (!H.amgT.present() || H.amgT.lev.size() < 2)
      fail(MSS_ERR_INVALID_ARG, "the set-up has no coarsened temperature hierarchy (CPTR3)");
    Level& L = H.amgT.lev[0];
    std::unique_ptr<mss_gnn> G(new mss_gnn());
    G->h.reset(new Handle());
    Handle& P = *G->h;
    P.device = H.device;
    P.num_sms = H.num_sms;
    MSS_CK(cudaStreamCreateWithFlags(&P.owned.s, cudaStreamNonBlocking));
    P.stream = P.owned.s;
    order_streams(H.stream, P.stream);   // the hierarchy is complete before the copy
    G->g = gnn_create(&P, L.n, L.rp.p, L.ci.p, L.v.p, L.cf.p, L.prp.p, L.pci.p, L.pv.p, L.nnz);
    MSS_CK(cudaStreamSynchronize(P.stream));   // nothing of h is read after this
    *out = G.release();
  });
}

void mss_gnn_destroy(mss_gnn* g) { delete g; }

int mss_gnn_info(const mss_gnn* g, int32_t* n, int32_t* m, int32_t* t) {
  if (!g) return MSS_ERR_INVALID_ARG;
  if (n) *n = gnn_nodes(g->g);
  if (m) *m = gnn_edges(g->g);
  if (t) *t = gnn_entries(g->g);
  return MSS_OK;
}

int mss_gnn_set_vectors(mss_gnn* g, int K, const double* starts, int nu, double omega,
                        int norm) {
  if (!g || !starts) return MSS_ERR_INVALID_ARG;
  return gnn_guarded(g, [&] {
    MSS_CK(cudaDeviceSynchronize());   // starts may come from any stream
    gnn_set_vectors(g->g, K, starts, nu, omega, norm);
    MSS_CK(cudaStreamSynchronize(g->h->stream));
  });
}

int mss_gnn_weights(mss_gnn* g, const float* params, double* w) {
  if (!g || !params || !w) return MSS_ERR_INVALID_ARG;
  return gnn_guarded(g, [&] {
    MSS_CK(cudaDeviceSynchronize());
    gnn_weights(g->g, params, w);
    MSS_CK(cudaStreamSynchronize(g->h->stream));
  });
}

int mss_gnn_loss_grad(mss_gnn* g, const float* params, double* loss, float* grad) {
  if (!g || !params) return MSS_ERR_INVALID_ARG;
  return gnn_guarded(g, [&] {
    MSS_CK(cudaDeviceSynchronize());
    const double L = gnn_loss_grad(g->g, params, grad);
    MSS_CK(cudaStreamSynchronize(g->h->stream));
    if (loss) *loss = L;
  });
}

int mss_gnn_adam(mss_gnn* g, float* params, float* m1, float* m2, const float* grad, int step,
                 float lr, float beta1, float beta2, float eps) {
  if (!g || !params || !m1 || !m2 || !grad) return MSS_ERR_INVALID_ARG;
  return gnn_guarded(g, [&] {
    gnn_adam(g->h.get(), params, m1, m2, grad, step, lr, beta1, beta2, eps);
    MSS_CK(cudaStreamSynchronize(g->h->stream));
  });
}

const char* mss_gnn_last_error(const mss_gnn* g) {
  return g ? g->last_error.c_str() : "null graph";
}

}  // extern "C"
