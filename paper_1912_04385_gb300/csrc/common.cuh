// common.cuh -- internal declarations of libmss (handle, device buffers,
// errors, launchers). Not part of the public ABI; see include/mss.h.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <memory>
#include <vector>

#include "mss.h"

namespace mss {

// Internal errors travel as exceptions inside the library and become status
// codes at the C-ABI boundary.
struct Error {
  int code;
  std::string msg;
};

[[noreturn]] void fail(int code, const std::string& msg);
void check_cuda(cudaError_t e, const char* what, const char* file, int line);
void count_launch();   // process-wide count of this library's kernel launches
long long launch_count(bool reset);
void add_launches(long long n);          // launches replayed by a CUDA graph
// While a stream capture runs on this thread, launches are counted into *c
// (the captured graph's size) instead of the process-wide count.
void capture_count(long long* c);
#define MSS_CK(call) ::mss::check_cuda((call), #call, __FILE__, __LINE__)
// every kernel launch is followed by MSS_LAUNCH_CK (error check and count)
#define MSS_LAUNCH_CK(what) \
  (::mss::count_launch(), ::mss::check_cuda(cudaGetLastError(), what, __FILE__, __LINE__))

// Optional event trace of kernel classes (CUDA events on the handle's stream).
enum TraceKind {
  TR_SPMV = 0,      // BSR matrix-vector product
  TR_BILU_FWD,      // forward sweeps of the last stage (fused u)
  TR_BILU_BWD,      // backward sweeps (fused y = x + v + M3 u)
  TR_VCYCLE,        // one whole AMG V-cycle
  TR_ORTHO,         // CGS2 projections, updates and norms of one Arnoldi step
  TR_SETUP_SCALE,   // validation, scaling and extraction
  TR_SETUP_AMG,     // one AMG hierarchy set-up
  TR_SETUP_BILU,    // colouring, ordering and factorisation
  TR_APPLY,         // one whole preconditioner application
  TR_CONDENSE,      // static condensation kernel
  TR_RECOVER,       // recovery of the secondary unknowns
  TR_KINDS
};

struct Handle;
void* dev_alloc(Handle* h, size_t bytes);   // the handle's hooks, else the device pool
void dev_free(Handle* h, void* p, size_t bytes);   // bytes: as passed to dev_alloc
cudaMemPool_t device_pool(int device);      // library-owned stream-ordered pool
void trim_pools();                          // return unused pool memory

// Owning device buffer allocated through the handle's hooks.
template <class T>
struct DBuf {
  Handle* h = nullptr;
  T* p = nullptr;
  size_t n = 0;
  DBuf() = default;
  DBuf(Handle* hh, size_t nn) { reset(hh, nn); }
  void reset(Handle* hh, size_t nn) {
    release();
    h = hh;
    n = nn;
    p = nn ? static_cast<T*>(dev_alloc(hh, nn * sizeof(T))) : nullptr;
  }
  void release() {
    if (p) dev_free(h, p, n * sizeof(T));
    p = nullptr;
    n = 0;
  }
  ~DBuf() { release(); }
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  DBuf(DBuf&& o) noexcept : h(o.h), p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
  DBuf& operator=(DBuf&& o) noexcept {
    if (this != &o) {
      release();
      h = o.h; p = o.p; n = o.n;
      o.p = nullptr; o.n = 0;
    }
    return *this;
  }
  T* get() const { return p; }
};

// One level of a scalar AMG hierarchy (CSR, 0-based, ascending columns).
struct Level {
  int n = 0, nnz = 0;
  DBuf<int> rp, ci;
  DBuf<double> v, dinv;
  double lam = 0.0;           // Gershgorin bound of D^-1 A (Chebyshev)
  // transfer to the next level (absent on the coarsest level)
  int nc = 0, nnzP = 0;
  DBuf<int> cf;               // 1 = C point
  DBuf<int> prp, pci;         // P: n x nc
  DBuf<double> pv;
  DBuf<int> rrp, rci;         // R = P^T: nc x n
  DBuf<double> rv;
  // V-cycle vectors
  DBuf<double> b, x, x2, r, d;
  // mixed precision: BF16 copies of A, P, R values, FP32 D^-1 and vectors
  DBuf<__nv_bfloat16> vh, pvh, rvh;
  DBuf<float> dinvf, bf, xf, x2f, rf, df;
  // multicolour Gauss-Seidel: points in colour-major order (ascending inside
  // a colour) and the first position of each colour (host, ncolour + 1)
  int ncolour = 0;
  std::vector<int> cstart;
  DBuf<int> mcorder;
  // system AMG (2 unknowns per point): inverse 2 x 2 diagonal block per point
  DBuf<double> dinv2;
  DBuf<float> dinv2f;
};

struct Hierarchy {
  std::vector<Level> lev;
  int bs = 1;                 // unknowns per point: 1 scalar AMG, 2 the system AMG of CPTR
  DBuf<double> coarse_inv;    // dense inverse of the coarsest operator, row-major
  DBuf<float> coarse_invf;    // its FP32 copy (mixed precision)
  int nc = 0;                 // size of the coarsest level
  // fused coarse levels: the first level of the tail (-1: none), its launch
  // width and shared memory, device descriptors of the tail levels (FP64 and mixed), the grid
  // barrier's words and its error flag
  int tail = -1;
  int tail_grid = 0;
  size_t tail_smem = 0;       // dynamic shared memory of the fused launch's blocks
  DBuf<unsigned char> tdesc, tdescf;
  DBuf<unsigned> tbar;
  DBuf<int> terr;
  bool present() const { return !lev.empty(); }
};

// A stream the library created; destroyed with its owner (declared first in
// Handle, so destroyed after every member whose frees are queued on it).
struct OwnedStream {
  cudaStream_t s = nullptr;
  ~OwnedStream() {
    if (s) cudaStreamDestroy(s);
  }
};

// Page-locked staging for the host's small read-backs (flags, counts, the
// solve state). Copies to pageable memory are staged by the driver and, with
// several set-up threads, serialise behind whichever stream is the slowest to
// reach its copy; a pinned word is read with a plain stream synchronisation.
struct PinnedHost {
  void* p = nullptr;
  ~PinnedHost() {
    if (p) cudaFreeHost(p);
  }
};
constexpr size_t kPinnedBytes = 256;

// Device blocks a handle without allocation hooks has freed, kept for its
// next allocations of the same size class on the same stream (reuse on the
// stream that freed them is ordered after every earlier use there, so it needs
// no driver call; a set-up allocates and frees a few hundred buffers). Bounded
// in block size and in total; the rest goes back to the pool. Declared after
// the stream and before every buffer of the handle: the buffers' frees land
// here, and the destructor returns the blocks while the stream still exists.
struct BlockCache {
  cudaStream_t s = nullptr;                           // the stream the blocks were freed on
  std::map<size_t, std::vector<void*>> blocks;        // size class -> free blocks
  size_t bytes = 0;
  ~BlockCache();
};

struct Handle {
  OwnedStream owned;
  PinnedHost pin;
  BlockCache cache;
  // binding
  cudaStream_t stream = nullptr;
  // Worker handles of the concurrent set-up (T and P hierarchies built on
  // their own streams and threads, allocating from the device pool). Declared
  // before the hierarchies they allocate, so they are destroyed after them.
  std::unique_ptr<Handle> aux[2];
  mss_alloc_fn alloc = nullptr;
  mss_free_fn free_fn = nullptr;
  void* ctx = nullptr;
  std::string last_error;
  int device = 0;
  int num_sms = 0;
  // problem
  bool ready = false;
  int N = 0, nb = 0, nnzb = 0, p = 0, t = 1;
  bool col_major = false;      // layout of the set-up's blocks
  mss_options opt{};
  int tb = 128;                // threads per CTA of the apply-path kernels (a multiple
                               // of 32; no result depends on it); set by the autotuner
  mss_bsr J{};                 // the caller's matrix (identity check in solve)
  double setup_ms = 0.0;
  // scaled system
  DBuf<int> rp, ci, diag;      // copied pattern, diagonal block index per row
  DBuf<double> abar;           // Abar blocks, row-major
  DBuf<double> wrows;          // W rows p and t per cell: N x 2 x nb
  DBuf<double> apt;            // Abar[p][t] per block (z_P = r_P - Abar_Pt x_T)
  DBuf<double> atp;            // Abar[t][p] per block (P-first stage order)
  Hierarchy amgT, amgP;
  // last stage: multicolour block ILU(0) in colour-major positions
  int ncol = 0;
  std::vector<int> cstart;     // host: first position of each colour, ncol + 1
  DBuf<int> colour, perm, iperm;
  DBuf<int> frp, fpos, fcell;  // factor pattern: column position and cell
  DBuf<int> fdp;               // index of the diagonal block in each factor row
  DBuf<int> fsrc;              // source block (index into Abar) of each factor block
  DBuf<int> fslo, fshi;        // per row: first in-strip lower entry, end of in-strip upper
  DBuf<double> cL, cG;         // per position: L_{q,q-1} and G_{q,q+1} (zero if absent)
  DBuf<int> cflag;             // per position: bit 0 / bit 1 = other in-strip lower / upper
  // mixed precision: BF16 factor blocks, FP32 column slices and work vectors
  DBuf<__nv_bfloat16> fvh, fdinvh, cLh, cGh;
  DBuf<float> fcsf, aptf, atpf;
  DBuf<float> rTf, xTf, zPf, vPf, wf;
  DBuf<int> st_first, st_len;  // strips in colour-major order: first position, length
  std::vector<int> sc_start;   // host: first strip of each colour, ncol + 1
  DBuf<double> fv;             // L (strictly lower) / U (strictly upper) blocks
  DBuf<double> fdinv;          // inverse of U's diagonal block, per position
  DBuf<double> fcs;            // Abar column slices [t | p] per factor block (2 nb)
  // preconditioner work vectors
  DBuf<double> rT, xT, zP, vP, w;
  DBuf<double> rE, xE;         // CPTR: the (P, T) pair of every cell, interleaved
  DBuf<float> rEf, xEf;
  // Krylov workspace
  int m = 0;
  DBuf<double> V, Z, bbar, res, hbuf, part;
  DBuf<double> kscal;          // device scalars of the Givens recurrence
  DBuf<double> gst;            // device solve state (step, counts, status, norms)
  DBuf<double> rfix, zfix, wfix;   // fixed-address Arnoldi vectors (v_j, z_j, w)
  // device-driven solve: the whole restarted FGMRES as one CUDA graph with
  // two nested while-loop conditional nodes, built on first use
  bool capturing = false;
  cudaGraphExec_t sgraph = nullptr;
  int sg_m = 0;
  long long sg_n = 0;
  long long sg_launch[4] = {};  // kernels in: init, cycle head, Arnoldi step, cycle tail
  DBuf<double> gb, gx;          // the graph's own copies of b and x
  DBuf<int> kflag;
  // end-to-end host solve copies
  DBuf<int> host_rp, host_ci;
  DBuf<double> host_vals, host_b, host_x;
  // scratch for reductions and flags
  DBuf<int> iflag;
  DBuf<double> dscr;
  // event trace
  struct TraceRec {
    int kind;
    cudaEvent_t a, b;
  };
  bool trace = false;
  std::vector<cudaEvent_t> ev_free;
  std::vector<TraceRec> ev_pending;
  double trace_ms[TR_KINDS] = {};
  long long trace_n[TR_KINDS] = {};
  Handle() = default;
  Handle(const Handle&) = delete;
  Handle& operator=(const Handle&) = delete;
  ~Handle();
};

// Records an event pair around its lifetime when tracing is on, and always
// an NVTX range named after the kind (outside stream capture).
struct TraceScope {
  Handle* h;
  int kind;
  cudaEvent_t a = nullptr;
  bool ranged = false;        // an NVTX range was pushed
  TraceScope(Handle* hh, int k);
  ~TraceScope();
};
void trace_drain(Handle* h);   // synchronises and accumulates finished pairs

// SplitMix64 (Steele, Lea, Flood 2014) as a counter-based generator: the
// value for counter k is the (k+1)-th output of the stream seeded with seed.
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t k) {
  uint64_t z = seed + (k + 1ULL) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// Load-and-convert to the compute type C (FP64, FP32, BF16 storage).
template <class C>
__device__ __forceinline__ C cvt(double x) { return (C)x; }
template <class C>
__device__ __forceinline__ C cvt(float x) { return (C)x; }
template <class C>
__device__ __forceinline__ C cvt(__nv_bfloat16 x) { return (C)__bfloat162float(x); }

// ---- launch helpers --------------------------------------------------------
// Dispatch a call templated on the block size NB (2..MSS_MAX_NB).
#define MSS_NB_DISPATCH(NBV, CALL)                                     \
  switch (NBV) {                                                       \
    case 2: { constexpr int NB = 2; CALL; } break;                     \
    case 3: { constexpr int NB = 3; CALL; } break;                     \
    case 4: { constexpr int NB = 4; CALL; } break;                     \
    case 5: { constexpr int NB = 5; CALL; } break;                     \
    case 6: { constexpr int NB = 6; CALL; } break;                     \
    case 7: { constexpr int NB = 7; CALL; } break;                     \
    case 8: { constexpr int NB = 8; CALL; } break;                     \
    case 9: { constexpr int NB = 9; CALL; } break;                     \
    case 10: { constexpr int NB = 10; CALL; } break;                   \
    case 11: { constexpr int NB = 11; CALL; } break;                   \
    case 12: { constexpr int NB = 12; CALL; } break;                   \
    case 13: { constexpr int NB = 13; CALL; } break;                   \
    case 14: { constexpr int NB = 14; CALL; } break;                   \
    case 15: { constexpr int NB = 15; CALL; } break;                   \
    case 16: { constexpr int NB = 16; CALL; } break;                   \
    default: fail(MSS_ERR_INVALID_ARG, "nb must be in [2, 16]");       \
  }

inline unsigned grid_for(long long n, int threads) {
  long long g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > 2147483647LL) g = 2147483647LL;
  return static_cast<unsigned>(g);
}

// util.cu
void exclusive_scan(Handle* h, const int* in, int* out, int n);   // out has n + 1 entries
// bytes <= kPinnedBytes from device memory to dst through the pinned staging
// word; synchronises the handle's stream
void read_back(Handle* h, void* dst, const void* dptr, size_t bytes);
// bytes <= kPinnedBytes from src to device memory through the staging word;
// synchronises the handle's stream
void write_to_device(Handle* h, void* dptr, const void* src, size_t bytes);
int read_int(Handle* h, const int* dptr);                         // synchronises
// count ints from device addresses dptrs[k] into out[k], one synchronisation
void read_ints(Handle* h, const int* const* dptrs, int* out, int count);
double read_double(Handle* h, const double* dptr);
void fill_int(Handle* h, int* p, int value, long long n);
void fill_double(Handle* h, double* p, double value, long long n);
void copy_dev(Handle* h, void* dst, const void* src, size_t bytes);

// setup_scale.cu
void validate_pattern(Handle* h, const int* rp, const int* ci, int N, int nnzb, int* diag);
// entries of the scaled blocks written beside Abar, one per block (any
// pointer may be null): pp = Abar[p][p] (B_PP), tt = Abar[t][t] (C_TT),
// pt = Abar[p][t], tp = Abar[t][p]
struct Extract {
  double* pp = nullptr;
  double* tt = nullptr;
  double* pt = nullptr;
  double* tp = nullptr;
};
void build_scaling(Handle* h, const double* vals, bool col_major, const Extract& ex = Extract{});
void scale_vector(Handle* h, const double* b, double* bbar);
// B_ee of CPTR: the 2 x 2 block Abar[(p, t), (p, t)] of every block (4 per block)
void extract_pair(Handle* h, double* out);

// amg_setup.cu
// level 0: the n0-row CSR (rp0, ci0, vals0), read on h's stream. frozen_cf
// (optional): C/F splits of an earlier hierarchy of a matrix with the same
// pattern, moved into the levels they fit instead of running PMIS.
void amg_build(Handle* h, Hierarchy& H, int n0, int nnz0, const int* rp0, const int* ci0,
               const double* vals0, const float* learned = nullptr,
               std::vector<DBuf<int>>* frozen_cf = nullptr);

// the system AMG of CPTR on np points of 2 x 2 blocks (bv: 4 per block)
void amg_build_system(Handle* h, Hierarchy& H, int np, int nnzb, const int* rp, const int* ci,
                      const double* bv);

// amg_cycle.cu
// The first Jacobi sweep from zero on level 0 of a hierarchy, x = omega D^-1 b,
// written by the kernel that forms b (x == nullptr: not used, because the
// smoother is not Jacobi or level 0 is the coarsest level).
template <class C>
struct Sweep0 {
  const C* dinv = nullptr;
  C omega = 0;
  C* x = nullptr;
};
Sweep0<double> sweep0(Handle* h, Hierarchy& H, double* x);
Sweep0<float> sweep0_mixed(Handle* h, Hierarchy& H, float* x);
// x_has_sweep0: x already holds sweep0's result for this b
void vcycle(Handle* h, Hierarchy& H, const double* b, double* x, bool x_has_sweep0 = false);
void vcycle_mixed(Handle* h, Hierarchy& H, const float* b, float* x,   // BF16 / FP32
                  bool x_has_sweep0 = false);
void pack_hierarchy_mixed(Handle* h, Hierarchy& H);
// the fused coarse-level launch's descriptors (after the set-up and, for the
// mixed form, after pack_hierarchy_mixed); no tail when it would not pay
void prepare_tail(Handle* h, Hierarchy& H);
// fails with MSS_ERR_CUDA if a grid barrier of the fused coarse levels gave up
void check_tail(Handle* h, Hierarchy& H);
// runs one grid-barrier wait that cannot complete; returns its error flag
int wait_limit_probe(Handle* h);
void gather_var(Handle* h, const double* v, int var, double* out, Sweep0<double> s0 = {});
void gather_var(Handle* h, const double* v, int var, float* out, Sweep0<float> s0 = {});
void scatter_var_zero(Handle* h, const double* s, int var, double* out);
// CPTR: the (P, T) pair of every cell to an interleaved vector and back
void gather_pair(Handle* h, const double* v, double* out);
void gather_pair(Handle* h, const double* v, float* out);
template <class C>
void split_pair(Handle* h, const C* pair, C* vP, C* xT);
void scatter_pair_zero(Handle* h, const double* pair, double* out);
void csr_block_pattern_spmv_sub(Handle* h, const double* vals, const double* x,
                                const double* r, int var, double* out, Sweep0<double> s0 = {});
void csr_block_pattern_spmv_sub(Handle* h, const float* vals, const float* x, const double* r,
                                int var, float* out, Sweep0<float> s0 = {});
void to_float(Handle* h, const double* in, float* out, long long n);
void to_bf16(Handle* h, const double* in, __nv_bfloat16* out, long long n);

// bilu.cu
// Jones-Plassmann colouring of the points of a structurally symmetric CSR
// graph (the priorities of the point-multicolour ILU order); returns the
// number of colours
int colour_points(Handle* h, int n, const int* rp, const int* ci, uint64_t seed, int* colour);
void bilu_setup(Handle* h);
// the numeric part alone (new values of Abar, same pattern and ordering)
void bilu_refactor(Handle* h);
// fused last stage: u = r - Abar[:,t] xT - Abar[:,p] vP (terms absent when the
// pointer is NULL), y = xadd + M3 u where xadd puts xT at t and vP at p.
void last_stage_apply(Handle* h, const double* r, const double* xT, const double* vP,
                      double* y);
// mixed form: BF16 factor blocks, FP32 sweeps, FP64 r and y
void last_stage_apply(Handle* h, const double* r, const float* xT, const float* vP, double* y);
void pack_last_stage_mixed(Handle* h);

// gnn.cu: learned interpolation for the temperature AMG (level 0)
struct GnnGraph;
int gnn_num_params();
GnnGraph* gnn_create(Handle* h, int n, const int* rp, const int* ci, const double* a,
                     const int* cf, const int* prp, const int* pci, const double* pv, int nnz);
void gnn_destroy(GnnGraph* g);
int gnn_entries(const GnnGraph* g);
int gnn_nodes(const GnnGraph* g);
int gnn_edges(const GnnGraph* g);
void gnn_weights(GnnGraph* g, const float* params, double* w);
void gnn_apply_to_p(GnnGraph* g, const float* params, double* pv);
void gnn_set_vectors(GnnGraph* g, int K, const double* starts, int nu, double omega, int norm);
double gnn_loss_grad(GnnGraph* g, const float* params, float* grad);
void gnn_adam(Handle* h, float* params, float* m1, float* m2, const float* grad, int step,
              float lr, float b1, float b2, float eps);

// fused.cu: lock-step solves of a group of set-up systems (one block size,
// one set of options) through multi-system launches; the tile shape of the
// launches is tuned once per (size bucket, nb) and cached (cache == null: a
// fixed shape); driver MSS_DRIVER_GRAPH runs the group solve as one graph
struct FusedTuneCache {
  std::mutex mu;
  std::map<long long, std::pair<int, int>> choice;   // key -> (blocks per tile, CTAs per SM)
};
struct FusedInfo {
  int tile_blocks = 0, per_sm = 0;
  long long sites = 0;   // multi-system launches in the init, head, step and tail sequences
  int steps = 0;         // Arnoldi steps of the group (the longest system's count)
};
// the fused schedule covers FP64 solves with Jacobi-smoothed V-cycles (CPTR3,
// CPR or the last stage alone) and block sizes up to kFusedMaxNB
constexpr int kFusedMaxNB = 8;
bool fused_supported(const mss_options& o, int nb);
void fused_solve(Handle* gh, const std::vector<Handle*>& hs, const std::vector<const double*>& b,
                 const std::vector<double*>& x, double tol, int maxit, int driver,
                 FusedTuneCache* cache, std::vector<mss_result>& res, FusedInfo* info);

// condense.cu: static condensation and recovery of the secondary unknowns
void condense(Handle* h, const mss_full* J, const double* r1, const double* r2, double* a,
              double* b);
void recover(Handle* h, const mss_full* J, const double* r2, const double* d1, double* d2);

// residual.cu
void check_residual_args(const mss_bsr* J, int nb, const double* b, const double* x,
                         const double* norms);
void residual_norms(cudaStream_t s, const mss_bsr* J, int nb, const double* b, const double* x,
                    double* scratch, double* norms);   // scratch: 2 n_rows doubles
void residual_norm(Handle* h, const mss_bsr* J, int nb, const double* b, const double* x,
                   double* norms);
// noalloc.cu
void residual_norm_noalloc(Handle* h, const mss_bsr* J, int nb, const double* b, const double* x,
                           double* norms);

// krylov.cu
void bsr_spmv(Handle* h, const double* x, double* y);
void precond_apply(Handle* h, const double* r, double* y);
// api.cu: the set-up and solve behind mss_setup / mss_fgmres_solve (throw Error)
void setup_handle(Handle& H, const mss_bsr* J, int nb, mss_layout layout,
                  const mss_options* opt);
int solve_handle(Handle& H, const mss_bsr* J, const double* b, double* x, double tol, int maxit,
                 mss_result* out);
int fgmres(Handle* h, const double* b, double* x, double tol, int maxit, mss_result* out);

}  // namespace mss
