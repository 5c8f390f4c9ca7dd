// fused.cu -- the fused schedule of batched solves (not in the paper).
//
// A group of independent systems that share the block size and the options
// is solved in lock step: every launch of the restarted FGMRES (Sec. 5.1)
// with its multi-stage preconditioner (Algorithms 1 and 2) serves all systems
// of the group at once. A launch walks a list of tiles; a tile is a run of
// blocks of one system's own launch of that kernel (the blocks the system's
// one-system launch would have), and the launch's CTAs stay resident and take
// tile after tile (grid-stride over the list). Every tile runs the same device
// body as the one-system kernel with the block index and grid size of the
// system's own launch, so each system computes exactly the values of its own
// solve.
//
// The whole group solve is one CUDA graph with the nested while loops of the
// one-system graph (restart cycles, Arnoldi steps): each system keeps its own
// solve state; after every step a control kernel marks the systems that take
// another step and continues the loop while any does. Systems that have
// stopped skip their tiles (a flag read per tile).
//
// The AMG V-cycles of the group go level by level: the down-sweep steps of
// every depth in order, then the coarse solves, then the up-sweep steps from
// the deepest level back; each system takes part at the depths it has, which
// keeps every system's own order of operations.
//
// Tile size (blocks per tile) and residency (CTAs per SM) of the launches are
// picked by an autotuner on the group's first preconditioner application and
// matrix-vector product; no result depends on them.
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "bilu_sweeps.cuh"
#include "common.cuh"
#include "krylov_kernels.cuh"
#include "vcycle_rows.cuh"
#include "vec_rows.cuh"

namespace mss {
namespace {

// blocks [b0, b1) of system s's own launch of G blocks
struct MTile {
  int s, b0, b1, G;
};

// The tile walker: body B on every tile of the list, tiles of systems whose
// live flag is 0 skipped (live == null: every system takes part).
template <class B>
__global__ void k_multi(const typename B::P* __restrict__ prm, const MTile* __restrict__ tiles,
                        int ntiles, const int* __restrict__ live) {
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const MTile tl = tiles[t];
    if (live && live[tl.s] == 0) continue;
    const typename B::P& p = prm[tl.s];
    for (int vb = tl.b0; vb < tl.b1; ++vb) {
      B::run(p, vb, tl.G);
      __syncthreads();   // the next block reuses the body's shared memory
    }
  }
}

// ---- bodies ------------------------------------------------------------------
// Each body's P holds the arguments of one system's launch; run() is the
// one-system kernel's code with vb for blockIdx.x and G for gridDim.x.

// row operations of the stages before the last one (V-cycles and the
// kernels that form their right-hand sides)
enum VKind { V_JACOBI, V_RESIDUAL, V_RESTRICT, V_PROLONG, V_GEMV, V_COPY, V_GATHER, V_PATSUB };

struct BVOp {
  struct P {
    int kind, n, nb, var;
    const int *rp, *ci;
    const double *v, *dinv, *b, *xin, *xc;
    const double* r;    // the block residual (gather, pattern subtraction)
    double omega;
    double *xout, *x1;
  };
  static __device__ __forceinline__ void run(const P& p, int vb, int) {
    const int i = vb * blockDim.x + threadIdx.x;
    switch (p.kind) {
      case V_JACOBI:
        if (i < p.n)
          dev::jacobi_row<double, double, dev::LdPlain>(i, i, p.rp, p.ci, p.v, p.dinv, p.b, p.omega,
                                                        p.xin, p.xout);
        break;
      case V_RESIDUAL:
        if (i < p.n) dev::residual_row<double, double, dev::LdPlain>(i, i, p.rp, p.ci, p.v, p.b,
                                                                     p.xin, p.xout);
        break;
      case V_RESTRICT:
        if (i < p.n)
          dev::restrict_row<double, double, dev::LdPlain>(i, i, p.rp, p.ci, p.v, p.xin, p.xout,
                                                          p.dinv, p.omega, p.x1);
        break;
      case V_PROLONG:
        if (i < p.n) dev::prolong_row<double, double, dev::LdPlain>(i, i, p.rp, p.ci, p.v, p.xc,
                                                                    p.xin, p.xout);
        break;
      case V_GEMV: {
        const int row = i >> 5, lane = threadIdx.x & 31;
        if (row < p.n) {
          const double s = dev::gemv_row<double, dev::LdPlain>(p.v + (size_t)row * p.n, lane,
                                                               p.n, p.b);
          if (lane == 0) p.xout[row] = s;
        }
        break;
      }
      case V_COPY:
        if (i < p.n) p.xout[i] = p.xin[i];
        break;
      case V_GATHER:
        dev::gather_var_row<double>(i, p.n, p.nb, p.r, p.var, p.xout, p.dinv, p.omega, p.x1);
        break;
      case V_PATSUB:
        dev::pattern_sub_row<double>(i, p.n, p.nb, p.rp, p.ci, p.v, p.xin, p.r, p.var, p.xout,
                                     p.dinv, p.omega, p.x1);
        break;
    }
  }
};

// the last stage's sweeps
enum BKind { B_FWD_PAR, B_FWD_CHAIN, B_BWD_PAR, B_BWD_CHAIN };

template <int NB, int MODE>
struct BLast {
  struct P {
    int kind, q0, q1, s0, s1, lower, p, t;
    const int *perm, *frp, *fslo, *fshi, *fdp, *fpos, *fcell, *st_first, *st_len, *cflag;
    const double *fv, *fcs, *fdinv, *cL, *cG, *r, *xT, *vP;
    double *w, *y;
  };
  static __device__ __forceinline__ void run(const P& p, int vb, int) {
    const long long warp = ((long long)vb * blockDim.x + threadIdx.x) >> 5;
    switch (p.kind) {
      case B_FWD_PAR:
        dev::fwd_par<NB, MODE, double, double>(warp, p.q0, p.q1, p.perm, p.frp, p.fslo, p.fpos,
                                               p.fcell, p.fv, p.fcs, p.r, p.xT, p.vP, p.w,
                                               p.lower, 1);
        break;
      case B_FWD_CHAIN:
        dev::fwd_chain<NB, double, double>(warp, p.s0, p.s1, p.st_first, p.st_len, p.fslo, p.fdp,
                                           p.fpos, p.fv, p.cL, p.cflag, p.w);
        break;
      case B_BWD_PAR:
        dev::bwd_par<NB, double, double>(warp, p.q0, p.q1, p.frp, p.fshi, p.fpos, p.fv, p.fdinv,
                                         p.w);
        break;
      case B_BWD_CHAIN:
        dev::bwd_chain<NB, double, double>(warp, p.s0, p.s1, p.st_first, p.st_len, p.fdp,
                                           p.fshi, p.fpos, p.fv, p.fdinv, p.cG, p.cflag, p.w,
                                           p.lower, p.perm, p.xT, p.vP, p.p, p.t, p.y);
        break;
    }
  }
};

template <int NB>
struct BSpmv {
  struct P {
    int N;
    const int *rp, *ci;
    const double *vals, *x;
    double* y;
  };
  static __device__ __forceinline__ void run(const P& p, int vb, int) {
    dev::bsr_spmv_rows<NB>(((long long)vb * blockDim.x + threadIdx.x) >> 5, p.N, p.rp, p.ci,
                           p.vals, p.x, p.y);
  }
};

template <int NB>
struct BScale {
  struct P {
    int N, p, t, scheme;
    const double *b, *wrows;
    double* out;
  };
  static __device__ __forceinline__ void run(const P& p, int vb, int) {
    dev::scale_vec_entry<NB>((long long)vb * blockDim.x + threadIdx.x, p.b, p.N, p.p, p.t,
                             p.scheme, p.wrows, p.out);
  }
};

// Krylov kernels: one body type with a kind, the arguments of every kind in
// one record (fields a kind does not use stay zero)
enum KKind {
  K_FILL, K_COPY, K_SQNORM, K_REDUCE, K_SOLVE_INIT, K_CYCLE_HEAD, K_INIT_G, K_STORE_Z, K_MDOT,
  K_UPDATE, K_ARNOLDI_FINISH, K_NORMALIZE, K_STEP_CONTROL, K_BACKSOLVE, K_XUPDATE, K_RESID_NORM,
  K_CYCLE_CONTROL
};

struct BKry {
  struct P {
    int kind, m, mode, rG;
    long long n, chunk, ld;
    GState* st;
    const double *a, *b, *c;   // inputs (meaning per kind)
    double *out, *out2, *H, *cs, *sn, *g, *ks;
    double value;
  };
  static __device__ __forceinline__ void run(const P& p, int vb, int G) {
    switch (p.kind) {
      case K_FILL: {   // as k_fill_double (grid-stride)
        long long i = (long long)vb * blockDim.x + threadIdx.x;
        const long long stride = (long long)G * blockDim.x;
        for (; i < p.n; i += stride) p.out[i] = p.value;
        break;
      }
      case K_COPY: {
        long long i = (long long)vb * blockDim.x + threadIdx.x;
        const long long stride = (long long)G * blockDim.x;
        for (; i < p.n; i += stride) p.out[i] = p.a[i];
        break;
      }
      case K_SQNORM: dev::sqnorm(p.n, p.chunk, p.a, p.out, vb); break;
      case K_REDUCE: dev::reduce(p.rG, p.a, p.out, p.st, p.mode, vb); break;
      case K_SOLVE_INIT: dev::solve_init(p.ks, p.st, 0, 0); break;
      case K_CYCLE_HEAD: dev::cycle_head(p.n, p.a, p.out, p.out2, p.st, vb, G); break;
      case K_INIT_G: dev::init_g(p.m, p.g, p.st, 0, 0, vb); break;
      case K_STORE_Z: dev::store_z(p.n, p.a, p.out, p.ld, p.st, vb, G); break;
      case K_MDOT: dev::mdot(p.n, p.chunk, p.a, p.ld, p.st, p.b, p.mode, p.out, vb, G); break;
      case K_UPDATE:
        dev::update(p.n, p.chunk, p.a, p.ld, p.st, p.b, p.out, p.mode, p.out2, vb, G);
        break;
      case K_ARNOLDI_FINISH:
        dev::arnoldi_finish(p.m, p.a, p.b, p.c, p.H, p.cs, p.sn, p.g, p.ks, p.st);
        break;
      case K_NORMALIZE: dev::normalize_store(p.n, p.a, p.ks, p.out, p.ld, p.st, p.out2, vb, G); break;
      case K_STEP_CONTROL: dev::step_control(p.m, p.ks, p.st, 0, 0); break;
      case K_BACKSOLVE: dev::backsolve(p.m, p.H, p.g, p.out, p.st); break;
      case K_XUPDATE: dev::xupdate(p.n, p.a, p.ld, p.b, p.out, p.st, vb, G); break;
      case K_RESID_NORM: dev::resid_norm(p.n, p.chunk, p.a, p.out, p.out2, vb); break;
      case K_CYCLE_CONTROL: dev::cycle_control(p.ks, p.st, 0, 0); break;
    }
  }
};

// Group control after a phase: live[s] = the system's go_outer (which = 0) or
// go_inner (which = 1); the loop's condition is whether any system is live.
// *count counts the control launches (the loop trips, for the launch count).
__global__ void k_group_control(int ns, GState* const* __restrict__ st, int* __restrict__ live,
                                int which, int* __restrict__ any, int* __restrict__ count,
                                cudaGraphConditionalHandle c, int use) {
  __shared__ int anyl;
  if (threadIdx.x == 0) anyl = 0;
  __syncthreads();
  for (int s = threadIdx.x; s < ns; s += blockDim.x) {
    const int v = which == 0 ? st[s]->go_outer : st[s]->go_inner;
    live[s] = v;
    if (v) atomicOr(&anyl, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    *any = anyl;
    *count += 1;
    if (use) cudaGraphSetConditional(c, anyl ? 1u : 0u);
  }
}

__global__ void k_gather_states(int ns, GState* const* __restrict__ st, GState* __restrict__ out) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < ns; s += gridDim.x * blockDim.x)
    out[s] = *st[s];
}

// ---- plan: the launches of the group solve -----------------------------------
enum Phase { PH_INIT, PH_HEAD, PH_STEP, PH_TAIL, PH_N };

using LaunchFn = void (*)(const unsigned char* prm, const MTile* tiles, int ntiles,
                          const int* live, unsigned grid, unsigned threads, cudaStream_t s);

template <class B>
void launch_site(const unsigned char* prm, const MTile* tiles, int ntiles, const int* live,
                 unsigned grid, unsigned threads, cudaStream_t s) {
  k_multi<B><<<grid, threads, 0, s>>>(reinterpret_cast<const typename B::P*>(prm), tiles, ntiles,
                                      live);
  MSS_LAUNCH_CK("k_multi");
}

// One launch of the group: the body, every system's arguments, every
// system's own grid (0: the system has no such launch) and the block size.
struct Site {
  LaunchFn launch = nullptr;
  size_t prm_off = 0;
  std::vector<int> vgrid;
  unsigned threads = 256;
  bool tune = false;          // part of the timed application and product
  size_t tile_off = 0;
  int ntiles = 0;
  unsigned grid = 0;
};

struct Plan {
  int ns = 0;
  std::vector<unsigned char> prm;
  std::vector<Site> site[PH_N];
  int phase = PH_INIT;
  bool tune = false;
  template <class B>
  void add(const std::vector<typename B::P>& p, const std::vector<int>& vgrid, unsigned threads) {
    bool any = false;
    for (int g : vgrid) any |= g > 0;
    if (!any) return;
    const size_t off = (prm.size() + 15) / 16 * 16;
    prm.resize(off + sizeof(typename B::P) * (size_t)ns);
    std::memcpy(prm.data() + off, p.data(), sizeof(typename B::P) * (size_t)ns);
    Site s;
    s.launch = &launch_site<B>;
    s.prm_off = off;
    s.vgrid = vgrid;
    s.threads = threads;
    s.tune = tune;
    site[phase].push_back(std::move(s));
  }
};

// A launch of one system, kept until the launches of all systems are merged
// by key: systems' launches with the same key become one group launch.
template <class P>
struct Rec {
  std::vector<int> key;
  int s;
  P p;
  int vgrid;
  unsigned threads;
};

template <class B>
void add_merged(Plan& plan, std::vector<Rec<typename B::P>>& recs) {
  std::stable_sort(recs.begin(), recs.end(),
                   [](const Rec<typename B::P>& a, const Rec<typename B::P>& b) {
                     return a.key < b.key;
                   });
  size_t i = 0;
  while (i < recs.size()) {
    size_t j = i;
    std::vector<typename B::P> p((size_t)plan.ns);
    std::memset(p.data(), 0, sizeof(typename B::P) * p.size());
    std::vector<int> vg((size_t)plan.ns, 0);
    while (j < recs.size() && recs[j].key == recs[i].key) {
      p[recs[j].s] = recs[j].p;
      vg[recs[j].s] = recs[j].vgrid;
      ++j;
    }
    plan.add<B>(p, vg, recs[i].threads);
    i = j;
  }
  recs.clear();
}

struct SysRef {
  Handle* h;
  Krylov K;
  const double* b;
  double* x;
};

bool first_sweep(const Hierarchy& H, const mss_options& o, int l) {
  return H.bs == 1 && o.smoother == MSS_JACOBI && l < (int)H.lev.size() - 1;
}

// The V-cycle of one system as keyed records, in the order of the one-system
// V-cycle with Jacobi smoothing whose level vectors hold the first sweep from
// zero (keys: down-sweep (0, depth, step), coarse solve (1, depth), up-sweep
// (2, -depth, step)).
void plan_vcycle_level(Handle* h, Hierarchy& H, int l, const double* b, double* out, int s,
                       unsigned T, std::vector<Rec<BVOp::P>>& recs) {
  const mss_options& o = h->opt;
  Level& L = H.lev[l];
  const int nl = (int)H.lev.size();
  auto rec = [&](std::vector<int> key, BVOp::P p, long long rows, bool warp_rows) {
    const int vg = (int)grid_for(warp_rows ? rows * 32 : rows, (int)T);
    recs.push_back({std::move(key), s, p, vg, T});
  };
  if (l == nl - 1) {
    BVOp::P p{};
    p.kind = V_GEMV;
    p.n = L.n;
    p.v = H.coarse_inv.p;
    p.b = b;
    p.xout = out;
    rec({1, l}, p, L.n, true);
    return;
  }
  Level& Cl = H.lev[l + 1];
  double* cb = Cl.b.p;
  double* cx = Cl.x.p;
  double* cur = out;
  double* alt = L.x2.p;
  const double om = o.jacobi_omega;
  auto jacobi = [&](std::vector<int> key, double* xin, double* xout) {
    BVOp::P p{};
    p.kind = V_JACOBI;
    p.n = L.n;
    p.rp = L.rp.p;
    p.ci = L.ci.p;
    p.v = L.v.p;
    p.dinv = L.dinv.p;
    p.b = b;
    p.omega = om;
    p.xin = xin;
    p.xout = xout;
    rec(std::move(key), p, L.n, false);
  };
  int k = 0;
  for (int q = 1; q < o.nu_pre; ++q) {
    jacobi({0, l, k++}, cur, alt);
    std::swap(cur, alt);
  }
  {
    BVOp::P p{};
    p.kind = V_RESIDUAL;
    p.n = L.n;
    p.rp = L.rp.p;
    p.ci = L.ci.p;
    p.v = L.v.p;
    p.b = b;
    p.xin = cur;
    p.xout = L.r.p;
    rec({0, l, k++}, p, L.n, false);
  }
  {
    BVOp::P p{};
    p.kind = V_RESTRICT;
    p.n = L.nc;
    p.rp = L.rrp.p;
    p.ci = L.rci.p;
    p.v = L.rv.p;
    p.xin = L.r.p;
    p.xout = cb;
    p.dinv = Cl.dinv.p;
    p.omega = om;
    p.x1 = first_sweep(H, o, l + 1) ? cx : nullptr;
    rec({0, l, k++}, p, L.nc, false);
  }
  plan_vcycle_level(h, H, l + 1, cb, cx, s, T, recs);
  double* target = o.nu_post % 2 == 0 ? out : L.x2.p;
  {
    BVOp::P p{};
    p.kind = V_PROLONG;
    p.n = L.n;
    p.rp = L.prp.p;
    p.ci = L.pci.p;
    p.v = L.pv.p;
    p.xc = cx;
    p.xin = cur;
    p.xout = target;
    rec({2, -l, 0}, p, L.n, false);
  }
  cur = target;
  alt = target == out ? L.x2.p : out;
  k = 1;
  for (int q = 0; q < o.nu_post; ++q) {
    jacobi({2, -l, k++}, cur, alt);
    std::swap(cur, alt);
  }
  if (cur != out) {
    BVOp::P p{};
    p.kind = V_COPY;
    p.n = L.n;
    p.xin = cur;
    p.xout = out;
    rec({2, -l, k++}, p, L.n, false);
  }
}

void plan_vcycle(Plan& plan, std::vector<SysRef>& S, Hierarchy Handle::*which,
                 const std::vector<const double*>& b, const std::vector<double*>& x, unsigned T) {
  std::vector<Rec<BVOp::P>> recs;
  for (int s = 0; s < plan.ns; ++s) {
    Handle* h = S[s].h;
    plan_vcycle_level(h, h->*which, 0, b[s], x[s], s, T, recs);
  }
  add_merged<BVOp>(plan, recs);
}

// the right-hand side of a V-cycle: the stage's variable of r (gather) or
// r minus the coupling to the previous stage's result (pattern subtraction),
// with the V-cycle's first sweep from zero where the hierarchy has one
void plan_rhs(Plan& plan, std::vector<SysRef>& S, int kind, Hierarchy Handle::*next,
              const std::vector<int>& var, const std::vector<const double*>& coup,
              const std::vector<const double*>& xprev, const std::vector<double*>& out,
              const std::vector<double*>& x1, unsigned T) {
  std::vector<BVOp::P> p((size_t)plan.ns);
  std::vector<int> vg((size_t)plan.ns);
  for (int s = 0; s < plan.ns; ++s) {
    Handle* h = S[s].h;
    Hierarchy& H = h->*next;
    BVOp::P q{};
    q.kind = kind;
    q.n = h->N;
    q.nb = h->nb;
    q.var = var[s];
    q.r = S[s].K.rfix;
    q.xout = out[s];
    if (kind == V_PATSUB) {
      q.rp = h->rp.p;
      q.ci = h->ci.p;
      q.v = coup[s];
      q.xin = xprev[s];
    }
    if (first_sweep(H, h->opt, 0)) {
      q.dinv = H.lev[0].dinv.p;
      q.omega = h->opt.jacobi_omega;
      q.x1 = x1[s];
    }
    p[s] = q;
    vg[s] = (int)grid_for(h->N, (int)T);
  }
  plan.add<BVOp>(p, vg, T);
}

constexpr unsigned kChainT = 64;   // block size of the chain passes (as the one-system kernels)

// the last stage: keys forward (0, colour, part), backward (1, -colour, part)
template <int NB, int MODE>
void plan_last_nb(Plan& plan, std::vector<SysRef>& S, const std::vector<const double*>& xT,
                  const std::vector<const double*>& vP, unsigned T) {
  using BL = BLast<NB, MODE>;
  constexpr int RPW = 32 / NB;
  std::vector<Rec<typename BL::P>> recs;
  for (int s = 0; s < plan.ns; ++s) {
    Handle* h = S[s].h;
    const bool bjac = h->opt.stage3 == MSS_BLOCK_JACOBI;
    const bool chains = !bjac &&
                        (h->opt.ilu_order == MSS_STRIPS || h->opt.ilu_order == MSS_STRIPS_JP) &&
                        h->opt.ilu_strip > 1;
    typename BL::P base{};
    base.perm = h->perm.p;
    base.frp = h->frp.p;
    base.fslo = h->fslo.p;
    base.fshi = h->fshi.p;
    base.fdp = h->fdp.p;
    base.fpos = h->fpos.p;
    base.fcell = h->fcell.p;
    base.st_first = h->st_first.p;
    base.st_len = h->st_len.p;
    base.cflag = h->cflag.p;
    base.fv = h->fv.p;
    base.fcs = h->fcs.p;
    base.fdinv = h->fdinv.p;
    base.cL = h->cL.p;
    base.cG = h->cG.p;
    base.r = S[s].K.rfix;
    base.xT = xT[s];
    base.vP = vP[s];
    base.w = h->w.p;
    base.y = S[s].K.zfix;
    base.p = h->p;
    base.t = h->t;
    auto rec = [&](std::vector<int> key, int kind, int c, long long units, unsigned thr) {
      typename BL::P q = base;
      q.kind = kind;
      q.q0 = h->cstart[c];
      q.q1 = h->cstart[c + 1];
      q.s0 = h->sc_start[c];
      q.s1 = h->sc_start[c + 1];
      q.lower = bjac ? 0 : 1;
      if (kind == B_BWD_CHAIN) {
        q.xT = (MODE & 1) ? xT[s] : nullptr;
        q.vP = (MODE & 2) ? vP[s] : nullptr;
      }
      const long long warps = (units + RPW - 1) / RPW;
      recs.push_back({std::move(key), s, q, (int)grid_for(warps * 32, (int)thr), thr});
    };
    for (int c = 0; c < h->ncol; ++c) {
      const int q0 = h->cstart[c], q1 = h->cstart[c + 1];
      const int s0 = h->sc_start[c], s1 = h->sc_start[c + 1];
      if (q1 <= q0) continue;
      rec({0, c, 0}, B_FWD_PAR, c, q1 - q0, T);
      if (chains) rec({0, c, 1}, B_FWD_CHAIN, c, s1 - s0, kChainT);
    }
    for (int c = h->ncol - 1; c >= 0; --c) {
      const int q0 = h->cstart[c], q1 = h->cstart[c + 1];
      const int s0 = h->sc_start[c], s1 = h->sc_start[c + 1];
      if (q1 <= q0) continue;
      if (!bjac) rec({1, -c, 0}, B_BWD_PAR, c, q1 - q0, T);
      rec({1, -c, 1}, B_BWD_CHAIN, c, s1 - s0, kChainT);
    }
  }
  add_merged<BL>(plan, recs);
}

template <int NB>
void plan_last(Plan& plan, std::vector<SysRef>& S, const std::vector<const double*>& xT,
               const std::vector<const double*>& vP, unsigned T) {
  // ILU alone: no earlier stage; CPR: v_P only; CPTR3: x_T and v_P
  const int mode = (xT[0] ? 1 : 0) | (vP[0] ? 2 : 0);
  switch (mode) {
    case 0: plan_last_nb<NB, 0>(plan, S, xT, vP, T); break;
    case 2: plan_last_nb<NB, 2>(plan, S, xT, vP, T); break;
    case 3: plan_last_nb<NB, 3>(plan, S, xT, vP, T); break;
    default: fail(MSS_ERR_INVALID_ARG, "no fused last stage for this combination of stages");
  }
}

// z = M^{-1} v for every system: the stages of Algorithm 2 (CPTR3), Algorithm
// 1 (CPR) or the last stage alone, as precond_apply runs them
template <int NB>
void plan_apply(Plan& plan, std::vector<SysRef>& S, unsigned T) {
  const int ns = plan.ns;
  const mss_options& o = S[0].h->opt;
  std::vector<const double*> none((size_t)ns, nullptr), xTc(ns), vPc(ns);
  std::vector<double*> rT(ns), xT(ns), zP(ns), vP(ns);
  std::vector<const double*> crT(ns), czP(ns), apt(ns), atp(ns);
  std::vector<int> vp(ns), vt(ns);
  for (int s = 0; s < ns; ++s) {
    Handle* h = S[s].h;
    rT[s] = h->rT.p;
    xT[s] = h->xT.p;
    zP[s] = h->zP.p;
    vP[s] = h->vP.p;
    crT[s] = h->rT.p;
    czP[s] = h->zP.p;
    xTc[s] = h->xT.p;
    vPc[s] = h->vP.p;
    apt[s] = h->apt.p;
    atp[s] = h->atp.p;
    vp[s] = h->p;
    vt[s] = h->t;
  }
  if (o.scheme == MSS_ILU0) {
    plan_last<NB>(plan, S, none, none, T);
    return;
  }
  if (o.scheme == MSS_CPR) {
    plan_rhs(plan, S, V_GATHER, &Handle::amgP, vp, none, none, rT, vP, T);
    plan_vcycle(plan, S, &Handle::amgP, crT, vP, T);
    plan_last<NB>(plan, S, none, vPc, T);
    return;
  }
  if (o.stage_order == MSS_STAGE_T_FIRST) {
    plan_rhs(plan, S, V_GATHER, &Handle::amgT, vt, none, none, rT, xT, T);
    plan_vcycle(plan, S, &Handle::amgT, crT, xT, T);
    plan_rhs(plan, S, V_PATSUB, &Handle::amgP, vp, apt, xTc, zP, vP, T);
    plan_vcycle(plan, S, &Handle::amgP, czP, vP, T);
  } else {
    plan_rhs(plan, S, V_GATHER, &Handle::amgP, vp, none, none, rT, vP, T);
    plan_vcycle(plan, S, &Handle::amgP, crT, vP, T);
    plan_rhs(plan, S, V_PATSUB, &Handle::amgT, vt, atp, vPc, zP, xT, T);
    plan_vcycle(plan, S, &Handle::amgT, czP, xT, T);
  }
  plan_last<NB>(plan, S, xTc, vPc, T);
}

template <int NB>
void plan_spmv(Plan& plan, std::vector<SysRef>& S, bool x_is_solution, unsigned T) {
  constexpr int RPW = 32 / NB;
  std::vector<typename BSpmv<NB>::P> p((size_t)plan.ns);
  std::vector<int> vg((size_t)plan.ns);
  for (int s = 0; s < plan.ns; ++s) {
    Handle* h = S[s].h;
    const long long warps = (h->N + RPW - 1) / RPW;
    p[s] = {h->N, h->rp.p, h->ci.p, h->abar.p, x_is_solution ? S[s].x : S[s].K.zfix,
            x_is_solution ? h->res.p : S[s].K.wfix};
    vg[s] = (int)grid_for(warps * 32, (int)T);
  }
  plan.add<BSpmv<NB>>(p, vg, T);
}

// one Krylov launch kind for every system; f fills the system's record and
// returns its grid
template <class F>
void plan_kry(Plan& plan, std::vector<SysRef>& S, unsigned threads, F&& f) {
  std::vector<BKry::P> p((size_t)plan.ns);
  std::vector<int> vg((size_t)plan.ns);
  for (int s = 0; s < plan.ns; ++s) {
    BKry::P q{};
    vg[s] = f(S[s], q);
    p[s] = q;
  }
  plan.add<BKry>(p, vg, threads);
}

// The four launch sequences of the one-system solve (krylov.cu seq_init,
// seq_head, seq_step, seq_tail) for the group, the control kernels aside.
template <int NB>
void plan_solve(Plan& plan, std::vector<SysRef>& S, unsigned T) {
  auto sgrid = [](const SysRef& r) { return (int)r.K.sgrid; };
  // ---- init: bbar = N^{-1} b, x = 0, ||bbar||, r = bbar
  plan.phase = PH_INIT;
  {
    std::vector<typename BScale<NB>::P> p((size_t)plan.ns);
    std::vector<int> vg((size_t)plan.ns);
    for (int s = 0; s < plan.ns; ++s) {
      Handle* h = S[s].h;
      p[s] = {h->N, h->p, h->t, h->opt.scheme, S[s].b, h->wrows.p, h->bbar.p};
      vg[s] = (int)grid_for((long long)h->N * NB, 256);
    }
    plan.add<BScale<NB>>(p, vg, 256);
  }
  plan_kry(plan, S, 256, [&](SysRef& r, BKry::P& q) {
    q.kind = K_FILL;
    q.n = r.K.n;
    q.out = r.x;
    q.value = 0.0;
    const unsigned g = grid_for(r.K.n, 256);
    return (int)(g > 4096 ? 4096 : g);
  });
  plan_kry(plan, S, KT, [&](SysRef& r, BKry::P& q) {
    q.kind = K_SQNORM;
    q.n = r.K.n;
    q.chunk = r.K.rs.chunk;
    q.a = r.h->bbar.p;
    q.out = r.K.part;
    return r.K.rs.G;
  });
  plan_kry(plan, S, KT, [&](SysRef& r, BKry::P& q) {
    q.kind = K_REDUCE;
    q.rG = r.K.rs.G;
    q.a = r.K.part;
    q.out = r.K.ks + 7;
    q.st = r.K.st;
    q.mode = 2;
    return 1;
  });
  plan_kry(plan, S, 32, [&](SysRef& r, BKry::P& q) {
    q.kind = K_SOLVE_INIT;
    q.ks = r.K.ks;
    q.st = r.K.st;
    return 1;
  });
  plan_kry(plan, S, 256, [&](SysRef& r, BKry::P& q) {
    q.kind = K_COPY;
    q.n = r.K.n;
    q.a = r.h->bbar.p;
    q.out = r.h->res.p;
    return (int)grid_for(r.K.n, 256);
  });
  // ---- cycle head: V_0 = r / beta, g = beta e_1
  plan.phase = PH_HEAD;
  plan_kry(plan, S, 256, [&](SysRef& r, BKry::P& q) {
    q.kind = K_CYCLE_HEAD;
    q.n = r.K.n;
    q.a = r.h->res.p;
    q.out = r.K.V;
    q.out2 = r.K.rfix;
    q.st = r.K.st;
    return sgrid(r);
  });
  plan_kry(plan, S, 128, [&](SysRef& r, BKry::P& q) {
    q.kind = K_INIT_G;
    q.m = r.K.m;
    q.g = r.K.g;
    q.st = r.K.st;
    return 1;
  });
  // ---- Arnoldi step: z_j = M^{-1} v_j, w = Abar z_j, orthogonalise, normalise
  plan.phase = PH_STEP;
  plan.tune = true;
  plan_apply<NB>(plan, S, T);
  plan.tune = false;
  plan_kry(plan, S, 256, [&](SysRef& r, BKry::P& q) {
    q.kind = K_STORE_Z;
    q.n = r.K.n;
    q.a = r.K.zfix;
    q.out = r.K.Z;
    q.ld = r.K.ld;
    q.st = r.K.st;
    return sgrid(r);
  });
  plan.tune = true;
  plan_spmv<NB>(plan, S, false, T);
  plan.tune = false;
  const bool cgs2 = S[0].h->opt.orthog == MSS_CGS2;
  auto reduce = [&](int mode, double* (*out)(SysRef&)) {
    plan_kry(plan, S, KT, [&](SysRef& r, BKry::P& q) {
      q.kind = K_REDUCE;
      q.rG = r.K.rs.G;
      q.a = r.K.part;
      q.out = out(r);
      q.st = r.K.st;
      q.mode = mode;
      return mode == 0 ? r.K.m + 1 : 1;
    });
  };
  plan_kry(plan, S, KT, [&](SysRef& r, BKry::P& q) {
    q.kind = K_MDOT;
    q.n = r.K.n;
    q.chunk = r.K.rs.chunk;
    q.a = r.K.V;
    q.ld = r.K.ld;
    q.st = r.K.st;
    q.b = r.K.wfix;
    q.mode = 1;
    q.out = r.K.part;
    return r.K.rs.G;
  });
  reduce(0, [](SysRef& r) { return r.K.h1; });
  reduce(1, [](SysRef& r) { return r.K.sq; });
  auto update = [&](int mode, bool with_h2) {
    plan_kry(plan, S, KT, [&](SysRef& r, BKry::P& q) {
      q.kind = K_UPDATE;
      q.n = r.K.n;
      q.chunk = r.K.rs.chunk;
      q.a = r.K.V;
      q.ld = r.K.ld;
      q.st = r.K.st;
      q.b = with_h2 ? r.K.h2 : r.K.h1;
      q.out = r.K.wfix;
      q.mode = mode;
      q.out2 = r.K.part;
      return r.K.rs.G;
    });
  };
  if (cgs2) {
    update(0, false);
    reduce(0, [](SysRef& r) { return r.K.h2; });
  }
  update(1, cgs2);
  reduce(2, [](SysRef& r) { return r.K.sq + 1; });
  plan_kry(plan, S, 32, [&](SysRef& r, BKry::P& q) {
    q.kind = K_ARNOLDI_FINISH;
    q.m = r.K.m;
    q.a = r.K.h1;
    q.b = cgs2 ? r.K.h2 : nullptr;
    q.c = r.K.sq;
    q.H = r.K.H;
    q.cs = r.K.cs;
    q.sn = r.K.sn;
    q.g = r.K.g;
    q.ks = r.K.ks;
    q.st = r.K.st;
    return 1;
  });
  plan_kry(plan, S, 256, [&](SysRef& r, BKry::P& q) {
    q.kind = K_NORMALIZE;
    q.n = r.K.n;
    q.a = r.K.wfix;
    q.ks = r.K.ks;
    q.out = r.K.V;
    q.ld = r.K.ld;
    q.st = r.K.st;
    q.out2 = r.K.rfix;
    return sgrid(r);
  });
  plan_kry(plan, S, 32, [&](SysRef& r, BKry::P& q) {
    q.kind = K_STEP_CONTROL;
    q.m = r.K.m;
    q.ks = r.K.ks;
    q.st = r.K.st;
    return 1;
  });
  // ---- cycle tail: x += Z_k y_k, true residual, stop or restart
  plan.phase = PH_TAIL;
  plan_kry(plan, S, 32, [&](SysRef& r, BKry::P& q) {
    q.kind = K_BACKSOLVE;
    q.m = r.K.m;
    q.H = r.K.H;
    q.g = r.K.g;
    q.out = r.K.yv;
    q.st = r.K.st;
    return 1;
  });
  plan_kry(plan, S, 256, [&](SysRef& r, BKry::P& q) {
    q.kind = K_XUPDATE;
    q.n = r.K.n;
    q.a = r.K.Z;
    q.ld = r.K.ld;
    q.b = r.K.yv;
    q.out = r.x;
    q.st = r.K.st;
    return sgrid(r);
  });
  plan_spmv<NB>(plan, S, true, T);
  plan_kry(plan, S, KT, [&](SysRef& r, BKry::P& q) {
    q.kind = K_RESID_NORM;
    q.n = r.K.n;
    q.chunk = r.K.rs.chunk;
    q.a = r.h->bbar.p;
    q.out = r.h->res.p;
    q.out2 = r.K.part;
    return r.K.rs.G;
  });
  reduce(2, [](SysRef& r) { return r.K.ks + 6; });
  plan_kry(plan, S, 32, [&](SysRef& r, BKry::P& q) {
    q.kind = K_CYCLE_CONTROL;
    q.ks = r.K.ks;
    q.st = r.K.st;
    return 1;
  });
}

// ---- execution -----------------------------------------------------------------
struct Group {
  Handle* gh = nullptr;        // the group's stream and device buffers
  int ns = 0;
  std::vector<SysRef> S;
  Plan plan;
  int tile_blocks = 1;         // blocks of a system's launch per tile
  int per_sm = 4;              // resident CTAs per SM of each launch
  std::vector<MTile> htiles;
  DBuf<unsigned char> dprm;
  DBuf<MTile> dtiles;
  DBuf<int> live;              // ns outer flags, then ns inner flags
  DBuf<int> ctl;               // any-flags (2) and control-kernel counts (2)
  DBuf<GState*> dst;
  DBuf<GState> gs;
  long long launches[PH_N] = {};
  cudaGraphExec_t exec = nullptr;
  ~Group() {
    if (exec) cudaGraphExecDestroy(exec);
  }
};

void build_tiles(Group& G, bool tune_only) {
  G.htiles.clear();
  const long long cap = (long long)G.per_sm * G.gh->num_sms;
  for (int ph = 0; ph < PH_N; ++ph)
    for (Site& s : G.plan.site[ph]) {
      if (tune_only && !s.tune) continue;
      s.tile_off = G.htiles.size();
      for (int q = 0; q < G.ns; ++q)
        for (int b0 = 0; b0 < s.vgrid[q]; b0 += G.tile_blocks)
          G.htiles.push_back({q, b0, std::min(b0 + G.tile_blocks, s.vgrid[q]), s.vgrid[q]});
      s.ntiles = (int)(G.htiles.size() - s.tile_off);
      s.grid = (unsigned)std::max(1LL, std::min<long long>(s.ntiles, cap));
    }
  if (G.dtiles.n < G.htiles.size()) G.dtiles.reset(G.gh, G.htiles.size());
  MSS_CK(cudaMemcpyAsync(G.dtiles.p, G.htiles.data(), sizeof(MTile) * G.htiles.size(),
                         cudaMemcpyHostToDevice, G.gh->stream));
  MSS_CK(cudaStreamSynchronize(G.gh->stream));
}

void run_phase(Group& G, int ph, bool tune_only = false) {
  const int* live = ph == PH_INIT ? nullptr : G.live.p + (ph == PH_STEP ? G.ns : 0);
  for (Site& s : G.plan.site[ph]) {
    if (tune_only && !s.tune) continue;
    s.launch(G.dprm.p + s.prm_off, G.dtiles.p + s.tile_off, s.ntiles, tune_only ? nullptr : live,
             s.grid, s.threads, G.gh->stream);
  }
}

void control(Group& G, int which, cudaGraphConditionalHandle c, int use) {
  k_group_control<<<1, 256, 0, G.gh->stream>>>(G.ns, G.dst.p, G.live.p + (which ? G.ns : 0),
                                                which, G.ctl.p + which, G.ctl.p + 2 + which, c,
                                                use);
  MSS_LAUNCH_CK("k_group_control");
}

// the autotuner: blocks per tile and resident CTAs per SM, timed on the
// group's preconditioner application and matrix-vector product (from a zero
// vector, every system taking part)
void tune(Group& G) {
  for (SysRef& r : G.S)
    MSS_CK(cudaMemsetAsync(r.K.rfix, 0, sizeof(double) * (size_t)r.K.n, G.gh->stream));
  cudaEvent_t a, b;
  MSS_CK(cudaEventCreate(&a));
  MSS_CK(cudaEventCreate(&b));
  float best = 1e30f;
  int bt = 1, br = 4;
  for (int tb : {1, 4, 16})
    for (int r : {4, 8}) {
      G.tile_blocks = tb;
      G.per_sm = r;
      build_tiles(G, true);
      run_phase(G, PH_STEP, true);
      MSS_CK(cudaEventRecord(a, G.gh->stream));
      for (int k = 0; k < 3; ++k) run_phase(G, PH_STEP, true);
      MSS_CK(cudaEventRecord(b, G.gh->stream));
      MSS_CK(cudaEventSynchronize(b));
      float ms = 0.f;
      MSS_CK(cudaEventElapsedTime(&ms, a, b));
      if (ms < best) {
        best = ms;
        bt = tb;
        br = r;
      }
    }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  G.tile_blocks = bt;
  G.per_sm = br;
}

void run_host(Group& G) {
  run_phase(G, PH_INIT);
  control(G, 0, 0, 0);
  while (read_int(G.gh, G.ctl.p)) {
    run_phase(G, PH_HEAD);
    control(G, 1, 0, 0);
    while (read_int(G.gh, G.ctl.p + 1)) {
      run_phase(G, PH_STEP);
      control(G, 1, 0, 0);
    }
    run_phase(G, PH_TAIL);
    control(G, 0, 0, 0);
  }
}

// init -> while (any system continues) { head -> while (any system takes a
// step) { step } -> tail }, the shape of the one-system solve graph
void build_graph(Group& G) {
  Handle* h = G.gh;
  cudaGraph_t top = nullptr;
  MSS_CK(cudaGraphCreate(&top, 0));
  try {
    cudaGraphConditionalHandle outer, inner;
    MSS_CK(cudaGraphConditionalHandleCreate(&outer, top, 0, cudaGraphCondAssignDefault));
    cudaGraphNode_t n0 = capture_into(h, top, nullptr, 0, &G.launches[PH_INIT], [&] {
      run_phase(G, PH_INIT);
      control(G, 0, outer, 1);
    });
    cudaGraphNode_t wo;
    cudaGraph_t ob = add_while(top, n0, outer, &wo);
    MSS_CK(cudaGraphConditionalHandleCreate(&inner, ob, 0, cudaGraphCondAssignDefault));
    cudaGraphNode_t n1 = capture_into(h, ob, nullptr, 0, &G.launches[PH_HEAD], [&] {
      run_phase(G, PH_HEAD);
      control(G, 1, inner, 1);
    });
    cudaGraphNode_t wi;
    cudaGraph_t ib = add_while(ob, n1, inner, &wi);
    capture_into(h, ib, nullptr, 0, &G.launches[PH_STEP], [&] {
      run_phase(G, PH_STEP);
      control(G, 1, inner, 1);
    });
    capture_into(h, ob, &wi, 1, &G.launches[PH_TAIL], [&] {
      run_phase(G, PH_TAIL);
      control(G, 0, outer, 1);
    });
    MSS_CK(cudaGraphInstantiate(&G.exec, top, 0));
  } catch (...) {
    cudaGraphDestroy(top);
    throw;
  }
  cudaGraphDestroy(top);
}

int bucket_of_rows(long long n) {
  int b = 0;
  while ((2LL << b) <= n) ++b;
  return b;
}

}  // namespace

bool fused_supported(const mss_options& o, int nb) {
  return nb >= 2 && nb <= kFusedMaxNB && o.precision == MSS_FP64 && o.smoother == MSS_JACOBI &&
         (o.scheme == MSS_CPTR3 || o.scheme == MSS_CPR || o.scheme == MSS_ILU0);
}

void fused_solve(Handle* gh, const std::vector<Handle*>& hs, const std::vector<const double*>& b,
                 const std::vector<double*>& x, double tol, int maxit, int driver,
                 FusedTuneCache* cache, std::vector<mss_result>& res, FusedInfo* info) {
  Group G;
  G.gh = gh;
  G.ns = (int)hs.size();
  G.plan.ns = G.ns;
  res.assign(hs.size(), mss_result{});
  if (G.ns == 0) return;
  const int nb = hs[0]->nb;
  long long rows = 0;
  for (int s = 0; s < G.ns; ++s) {
    Handle* h = hs[s];
    if (h->nb != nb || !fused_supported(h->opt, h->nb) || h->opt.restart != hs[0]->opt.restart ||
        h->opt.orthog != hs[0]->opt.orthog || h->opt.scheme != hs[0]->opt.scheme ||
        h->opt.stage_order != hs[0]->opt.stage_order)
      fail(MSS_ERR_INVALID_ARG, "a fused group needs one block size and one set of options");
    SysRef r{h, workspace(h), b[s], x[s]};
    G.S.push_back(r);
    rows += h->N;
  }
  // every system's state: tolerance and iteration limit, all flags zero
  for (SysRef& r : G.S) {
    GState st{};
    st.tol = tol;
    st.maxit = maxit;
    write_to_device(r.h, r.K.st, &st, sizeof(GState));
  }
  const unsigned T = 256;
  switch (nb) {   // the block sizes of the fused schedule (kFusedMaxNB)
    case 2: plan_solve<2>(G.plan, G.S, T); break;
    case 3: plan_solve<3>(G.plan, G.S, T); break;
    case 4: plan_solve<4>(G.plan, G.S, T); break;
    case 5: plan_solve<5>(G.plan, G.S, T); break;
    case 6: plan_solve<6>(G.plan, G.S, T); break;
    case 7: plan_solve<7>(G.plan, G.S, T); break;
    case 8: plan_solve<8>(G.plan, G.S, T); break;
    default: fail(MSS_ERR_INVALID_ARG, "the fused schedule takes nb <= 8");
  }
  G.dprm.reset(gh, G.plan.prm.size());
  MSS_CK(cudaMemcpyAsync(G.dprm.p, G.plan.prm.data(), G.plan.prm.size(), cudaMemcpyHostToDevice,
                         gh->stream));
  std::vector<GState*> sp;
  for (SysRef& r : G.S) sp.push_back(r.K.st);
  G.dst.reset(gh, sp.size());
  MSS_CK(cudaMemcpyAsync(G.dst.p, sp.data(), sizeof(GState*) * sp.size(), cudaMemcpyHostToDevice,
                         gh->stream));
  G.live.reset(gh, 2 * (size_t)G.ns);
  G.ctl.reset(gh, 4);
  fill_int(gh, G.ctl.p, 0, 4);
  G.gs.reset(gh, G.ns);
  MSS_CK(cudaStreamSynchronize(gh->stream));
  // tile shape: cached per (size bucket, nb), tuned on the first group
  // (no cache: the fixed shape of 1 block per tile, 4 CTAs per SM)
  const long long key = (long long)bucket_of_rows(rows) * 32 + nb;
  bool tuned = cache == nullptr;
  if (cache) {
    std::lock_guard<std::mutex> lk(cache->mu);
    auto it = cache->choice.find(key);
    if (it != cache->choice.end()) {
      G.tile_blocks = it->second.first;
      G.per_sm = it->second.second;
      tuned = true;
    }
  }
  if (!tuned) {
    tune(G);
    std::lock_guard<std::mutex> lk(cache->mu);
    cache->choice[key] = {G.tile_blocks, G.per_sm};
  }
  build_tiles(G, false);
  if (driver == MSS_DRIVER_GRAPH) {
    build_graph(G);
    MSS_CK(cudaGraphLaunch(G.exec, gh->stream));
  } else {
    run_host(G);
  }
  k_gather_states<<<1, 128, 0, gh->stream>>>(G.ns, G.dst.p, G.gs.p);
  MSS_LAUNCH_CK("k_gather_states");
  std::vector<GState> hst((size_t)G.ns);
  MSS_CK(cudaMemcpyAsync(hst.data(), G.gs.p, sizeof(GState) * hst.size(), cudaMemcpyDeviceToHost,
                         gh->stream));
  int counts[4];
  MSS_CK(cudaMemcpyAsync(counts, G.ctl.p, sizeof(counts), cudaMemcpyDeviceToHost, gh->stream));
  MSS_CK(cudaStreamSynchronize(gh->stream));
  if (driver == MSS_DRIVER_GRAPH) {
    // control launches: counts[2] after init and tails, counts[3] after heads
    // and steps
    const long long heads = counts[2] - 1, steps = counts[3] - heads;
    add_launches(G.launches[PH_INIT] + heads * (G.launches[PH_HEAD] + G.launches[PH_TAIL]) +
                 steps * G.launches[PH_STEP]);
  }
  for (int s = 0; s < G.ns; ++s) {
    const GState& st = hst[s];
    mss_result& r = res[s];
    r.iters = st.total;
    r.restarts = st.restarts;
    r.status = (st.rhs_bad || st.status == MSS_ERR_BREAKDOWN) ? MSS_ERR_BREAKDOWN : st.status;
    r.rel_res_implicit = st.rel_impl;
    r.rel_res_true = st.rel_true;
    r.setup_ms = hs[s]->setup_ms;
  }
  if (info) {
    info->tile_blocks = G.tile_blocks;
    info->per_sm = G.per_sm;
    long long sites = 0;
    for (int ph = 0; ph < PH_N; ++ph) sites += (long long)G.plan.site[ph].size();
    info->sites = sites;
    info->steps = counts[3] - (counts[2] - 1);
  }
}

}  // namespace mss
