/*
 * mss.h -- C-ABI of the multi-stage preconditioned FGMRES library for GB300
 * (libmss.so, CUDA, sm_103a).
 *
 * Method: Cremon, Castelletto, White, "Multi-Stage Preconditioners for
 * Thermal-Compositional-Reactive Flow in Porous Media" (arXiv:1912.04385).
 * The library solves the primary (statically condensed) system A x = b of
 * Sec. 3, Eq. reduced, by split preconditioning (Sec. 4, Eqs. splitPrec1 and
 * splitPrec2): the left scaling N^{-1} (Eq. CPR for CPR, Eqs. CPTR31 and
 * CPTR32 for CPTR3) is applied once, then right-preconditioned FGMRES
 * (Sec. 5.1) applies the multi-stage operator M^{-1} of Eq. multistageprec in
 * the form of Algorithm 1 (CPR) or Algorithm 2 (CPTR3) every iteration.
 *
 * Conventions shared by every entry point
 *   - A is cell-blocked BSR: row_ptr[n_rows+1] and col_idx[nnzb] (int32,
 *     columns strictly ascending within a row, diagonal block present,
 *     pattern structurally symmetric as for any finite-volume cell graph),
 *     vals[nnzb * nb * nb] (float64). Blocks are row-major unless
 *     mss_layout.col_major_blocks is set. Vectors are cell-interleaved:
 *     unknown k of cell i lives at i*nb + k.
 *   - Every pointer argument named as "device" is device memory of the
 *     current CUDA device; "host" pointers are ordinary host memory.
 *     Caller-owned arrays are only read (inputs) or written (outputs), never
 *     retained after the call returns unless stated.
 *   - All device work is enqueued on the handle's stream. Calls that return
 *     results to the host synchronise that stream.
 *   - Every function returns an int status: MSS_OK (0) or a negative
 *     MSS_ERR_* code; no exception crosses the ABI. mss_last_error() gives a
 *     message for the last failing call on a handle.
 */
#ifndef MSS_H
#define MSS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define MSS_OK 0
#define MSS_ERR_INVALID_ARG (-1)    /* bad size, pointer, pattern or option */
#define MSS_ERR_SINGULAR_BLOCK (-2) /* zero pivot in a cell block (no pivoting, Sec. 3) */
#define MSS_ERR_NOT_CONVERGED (-3)  /* maxit reached; x holds the last iterate */
#define MSS_ERR_BREAKDOWN (-4)      /* non-finite value in the Krylov recurrence */
#define MSS_ERR_CUDA (-5)           /* a CUDA runtime call failed */
#define MSS_ERR_OOM (-6)            /* device allocation failed */
#define MSS_ERR_AMG (-7)            /* AMG set-up failed (coarsest level too large, ...) */
#define MSS_ERR_NOT_SETUP (-8)      /* handle has no set-up, or another matrix was passed */

/* Largest cell block size nb the library takes (the paper's primary systems
 * have 14 unknowns per cell, Sec. 5.1). */
#define MSS_MAX_NB 16

/* ---- option values ------------------------------------------------------ */
enum { MSS_CPTR3 = 0, MSS_CPR = 1, MSS_ILU0 = 2, MSS_CPTR = 3 }; /* preconditioner scheme */
enum { MSS_STAGE_T_FIRST = 0, MSS_STAGE_P_FIRST = 1 }; /* CPTR3 stage order */
enum { MSS_BILU0 = 0, MSS_BLOCK_JACOBI = 1 };        /* last stage */
enum { MSS_MULTICOLOR = 0, MSS_STRIPS = 2, MSS_STRIPS_JP = 3 }; /* block ILU(0) ordering */
enum { MSS_JACOBI = 0, MSS_CHEBYSHEV = 1, MSS_MCSGS = 3 }; /* AMG smoother (2: lexicographic
                                                       symmetric Gauss-Seidel, sequential,
                                                       has no GPU form) */
enum { MSS_FP64 = 0, MSS_MIXED = 1 };                /* preconditioner arithmetic */
enum { MSS_CGS1 = 0, MSS_CGS2 = 1 };                 /* Arnoldi orthogonalisation */
enum { MSS_DRIVER_HOST = 0, MSS_DRIVER_GRAPH = 1 };  /* who runs the FGMRES loop */
enum { MSS_FACTOR_AUTO = 0, MSS_FACTOR_WARP = 1, MSS_FACTOR_LANES = 2 }; /* ILU(0) kernel */

/* A BSR matrix; the arrays are device memory owned by the caller. */
typedef struct {
  int32_t n_rows;           /* number of cells N */
  int32_t nnzb;             /* number of stored blocks */
  const int32_t* row_ptr;   /* device, N + 1 entries, row_ptr[0] = 0 */
  const int32_t* col_idx;   /* device, nnzb entries */
  const double* vals;       /* device, nnzb * nb * nb entries */
} mss_bsr;

/* Position of pressure and temperature inside a cell block (the paper's
 * [s, P, T] partition, Sec. 4; any order is accepted). */
typedef struct {
  int32_t p_idx;            /* index of the pressure unknown, 0 <= p_idx < nb */
  int32_t t_idx;            /* index of the temperature unknown, != p_idx */
  int32_t col_major_blocks; /* 1 if vals blocks are stored column-major */
} mss_layout;

typedef struct {
  int32_t scheme;           /* MSS_CPTR3 (default; Sec. 4.3) | MSS_CPR (Sec. 4.1) |
                               MSS_ILU0 (no scaling, the last stage alone) |
                               MSS_CPTR (Sec. 4.2, Eqs. CPTRinit, CPTR1, CPTRM1): the
                               scaling N1 of Eq. CPTR31 alone, then two stages: a
                               system AMG for the 2 x 2 block B_ee on (P, T) --
                               nodal coarsening (PMIS on the Frobenius norms of the
                               blocks), classical interpolation per unknown on the
                               common split, Galerkin products of the coupled
                               system, damped 2 x 2 block Jacobi with jacobi_omega,
                               nu_pre, nu_post (the smoother option is not used) --
                               and the last stage. */
  int32_t stage_order;      /* MSS_STAGE_T_FIRST (Algorithm 2, default) | P first */
  int32_t stage3;           /* MSS_BILU0 (default) | MSS_BLOCK_JACOBI */
  int32_t ilu_order;        /* MSS_STRIPS (default): strips of ilu_strip consecutive
                               cells, coloured first-fit in strip order (each
                               strip the smallest colour none of its lower-index
                               adjacent strips has: two colours on a structured
                               grid), colour-major, natural order inside a strip;
                               MSS_STRIPS_JP: the same strips coloured by
                               Jones-Plassmann (SplitMix64 priorities, `seed`);
                               MSS_MULTICOLOR: every cell coloured on its own
                               (Jones-Plassmann) */
  int32_t smoother;         /* MSS_JACOBI (default) | MSS_CHEBYSHEV | MSS_MCSGS:
                               symmetric Gauss-Seidel, the smoother of the paper's
                               AMG (Sec. 5.1), in multicolour form: per level the
                               points are coloured (Jones-Plassmann, `seed`), one
                               application sweeps the colours in order and then
                               in reverse, a colour's points updated at once */
  int32_t nu_pre, nu_post;  /* smoothing sweeps per V-cycle leg (2, 2: HSL_MI20's defaults,
                               which Sec. 5.1 names) */
  int32_t cheb_degree;      /* Chebyshev polynomial degree (2) */
  int32_t amg_max_coarse;   /* direct solve at or below this size (1000, Sec. 5.1) */
  int32_t amg_max_levels;   /* at most this many levels (25) */
  int32_t interp_max_elems; /* interpolation row truncation, 0 = none (4) */
  int32_t restart;          /* FGMRES restart length m (30) */
  int32_t precision;        /* MSS_FP64 (default): every stage in float64.
                               MSS_MIXED: the preconditioner M^{-1} (Algorithms
                               1/2) keeps BF16 copies of the AMG operators,
                               interpolation/restriction and the block ILU(0)
                               factors, and FP32 copies of the scaled coupling
                               blocks; its sweeps run in FP32. The scaling, the
                               outer matvec, Arnoldi, Givens rotations and the
                               true residual stay float64, so FGMRES (Sec. 5.1,
                               flexible in the preconditioner) still converges
                               to the float64 tolerance; the iteration count
                               may differ from the float64 run. Not in the
                               paper, which computes in float64 throughout. */
  int32_t ilu_strip;        /* strip length in cells for MSS_STRIPS (32), 1..1024 */
  int32_t orthog;           /* Arnoldi: MSS_CGS1 (default) | MSS_CGS2 */
  int32_t driver;           /* MSS_DRIVER_HOST: the host reads the solve state back
                               after every Arnoldi step and decides;
                               MSS_DRIVER_GRAPH: the whole restarted solve is one
                               CUDA graph (two nested while-loop conditional
                               nodes, the decisions taken by device kernels),
                               launched once per solve and read back once. Same
                               kernels, same order, same results. */
  int32_t factor_form;      /* which kernel factors a colour of the block ILU(0):
                               MSS_FACTOR_AUTO (default) picks per colour by its
                               size (a warp per strip for colours too small to
                               fill the SMs, nb lanes per strip otherwise);
                               MSS_FACTOR_WARP / MSS_FACTOR_LANES force one form
                               for every colour. Both perform the same operations
                               in the same order, so the factors are the same
                               bits whichever form runs. */
  double amg_theta;         /* strength threshold (0.25) */
  double jacobi_omega;      /* Jacobi damping (0.8, HSL_MI20's default) */
  double cheb_lo_ratio;     /* Chebyshev interval [bound/ratio, factor*bound] (30) */
  double cheb_hi_factor;    /* (1.0) */
  uint64_t seed;            /* PMIS measure and colouring priorities */
  const void* learned_interp; /* NULL: classical interpolation everywhere (default).
                               Else a device pointer to mss_gnn_num_params()
                               floats: the network below predicts level 0's
                               interpolation weights of the temperature
                               hierarchy (CPTR3 only). Read during mss_setup. */
} mss_options;

typedef struct {
  int32_t iters;            /* FGMRES inner iterations in total */
  int32_t restarts;         /* completed restart cycles */
  int32_t status;           /* same as the return value */
  int32_t pad_;
  double rel_res_implicit;  /* |g_{k+1}| / ||bbar|| from the Givens recurrence */
  double rel_res_true;      /* ||bbar - Abar x|| / ||bbar|| at return */
  double setup_ms;          /* wall time of the last mss_setup */
  double solve_ms;          /* wall time of this solve */
} mss_result;

typedef struct mss_handle mss_handle;

/* Device memory hooks. alloc returns device memory of at least `bytes`
 * bytes (aligned to 256 bytes) or NULL; free releases it. Both are called
 * only from mss_* calls on the host thread that makes them. Memory passed
 * to free may still be in use by work already enqueued on the handle's
 * stream, so the hooks must be stream-ordered on that stream (as a caching
 * allocator bound to the stream is) or synchronous like cudaFree. */
typedef void* (*mss_alloc_fn)(size_t bytes, void* ctx);
typedef void (*mss_free_fn)(void* ptr, void* ctx);

/* Fill `opt` with the defaults listed above. Errors: INVALID_ARG if NULL. */
int mss_options_default(mss_options* opt);

/* Create a handle bound to the current CUDA device and `cuda_stream`
 * (a cudaStream_t, NULL = legacy default stream). alloc/free_fn may both be
 * NULL, in which case cudaMalloc/cudaFree are used; the handle owns every
 * buffer it allocates and frees it in mss_destroy. Errors: INVALID_ARG,
 * OOM. */
int mss_create(mss_handle** h, void* cuda_stream, mss_alloc_fn alloc, mss_free_fn free_fn,
               void* alloc_ctx);

/* Release the handle and everything it owns (NULL is ignored). */
void mss_destroy(mss_handle* h);

/* Set-up for the matrix J (Sec. 4): validates the pattern; builds the cell
 * scaling W_i = N^{-1} restricted to cell i from the diagonal block
 * (Eq. CPR, or Eqs. CPTR31 and CPTR32; identity for MSS_ILU0) and the scaled
 * blocks Abar_ij = W_i J_ij (Eq. splitPrec1); extracts B_PP and C_TT
 * (Eqs. CPR, CPTR31, CPTR32) and builds an AMG hierarchy for each
 * (Eqs. CPRM1, CPTR3M1, CPTRM2; classical AMG, coarse size <= 1000, Sec.
 * 5.1); and factors the last stage, block ILU(0) of Abar (Eq. CPTR3M3) in a
 * colour-major ordering of strips (or of single cells). J's arrays are
 * copied or consumed during the call;
 * the caller may free them afterwards, except that mss_fgmres_solve checks
 * that it receives the same mss_bsr (pointers and sizes). `opt` may be NULL
 * (defaults). nb in [2, MSS_MAX_NB]. Errors: INVALID_ARG (bad
 * sizes, pattern, layout or option), SINGULAR_BLOCK (a cell block needs
 * pivoting), AMG, OOM, CUDA. */
int mss_setup(mss_handle* h, const mss_bsr* J, int nb, mss_layout layout,
              const mss_options* opt);

/* New values of the same matrix pattern, as in a Newton loop (Sec. 2.5: the
 * Jacobian is re-evaluated at every Newton iteration and time step on a fixed
 * grid, so its block pattern does not change). J has the set-up's n_rows,
 * nnzb and pattern (checked on the device: INVALID_ARG otherwise; the
 * arrays may be other copies); its values replace the set-up's. The
 * symbolic set-up is kept -- the validated pattern, the diagonal positions,
 * the last stage's colouring, ordering and factor pattern -- and the rest is
 * recomputed: the scaling, B_PP and C_TT, the AMG hierarchies, the
 * factorisation and the reduced-precision copies.
 *   reuse = MSS_REUSE_PATTERN: the result is the one mss_setup gives for J,
 *           bit for bit (every kept part depends on the pattern only);
 *   reuse = MSS_REUSE_COARSENING: every AMG level also keeps its C/F split,
 *           so strength, interpolation weights and the Galerkin operators are
 *           recomputed on the earlier coarse grids (an F point left without
 *           a strong C point interpolates nothing).
 * Options are the set-up's (a learned_interp pointer must still be valid).
 * Afterwards mss_fgmres_solve takes J (not the set-up's mss_bsr). Errors:
 * NOT_SETUP, INVALID_ARG, SINGULAR_BLOCK, AMG, OOM, CUDA; after an error the
 * handle needs mss_setup again. */
enum { MSS_REUSE_PATTERN = 0, MSS_REUSE_COARSENING = 1 };
int mss_update_values(mss_handle* h, const mss_bsr* J, int reuse);

/* bbar = N^{-1} b (Eq. splitPrec1), device vectors of length N*nb.
 * Errors: NOT_SETUP, INVALID_ARG. */
int mss_scale_rhs(mss_handle* h, const double* b, double* bbar);

/* y = Abar x for the scaled matrix (the FGMRES matrix-vector product),
 * device vectors of length N*nb. Errors: NOT_SETUP, INVALID_ARG. */
int mss_spmv(mss_handle* h, const double* x, double* y);

/* y = M^{-1} r on the scaled system: Algorithm 2 for CPTR3, Algorithm 1
 * for CPR, the last stage alone for MSS_ILU0. r, y: device, length N*nb,
 * distinct. Errors: NOT_SETUP, INVALID_ARG. */
int mss_apply(mss_handle* h, const double* r, double* y);

/* One stage operator alone, for testing the composition of Eq.
 * multistageprec: which = 0 temperature AMG stage (Eq. CPTR3M1), 1 pressure
 * AMG stage (Eq. CPTRM2 / CPRM1; for MSS_CPTR the system AMG stage on
 * (P, T), Eq. CPTRM1), 2 last stage (block ILU(0) or block Jacobi of Abar). The result is zero outside the stage's unknowns. Always
 * float64, whatever mss_options.precision (mss_apply follows precision).
 * Errors: NOT_SETUP, INVALID_ARG (stage absent in the scheme). */
int mss_stage_apply(mss_handle* h, int which, const double* r, double* y);

/* Solve A x = b: bbar = N^{-1} b, then right-preconditioned restarted
 * FGMRES(m) on Abar from x = 0 (Sec. 5.1; restart is a reading; classical
 * Gram-Schmidt once or twice per step, opt.orthog) until the
 * implicit residual |g|/||bbar|| <= tol and the true residual
 * ||bbar - Abar x||/||bbar|| <= tol, or maxit inner iterations. J must be
 * the mss_bsr passed to mss_setup. b, x: device, length N*nb; x is written
 * with the last iterate even on NOT_CONVERGED. `out` (host, may be NULL)
 * receives iteration counts, residuals and timings. Synchronises the
 * stream. Errors: NOT_SETUP, INVALID_ARG, NOT_CONVERGED, BREAKDOWN, CUDA. */
int mss_fgmres_solve(mss_handle* h, const mss_bsr* J, const double* b, double* x, double tol,
                     int maxit, mss_result* out);

/* End-to-end solve from HOST buffers: copies J's pattern (host arrays in an
 * mss_bsr) and b to the device, runs mss_setup and mss_fgmres_solve, and
 * copies x back to the host. When J's values are in pinned host memory the
 * device can address (cudaHostAlloc, cudaHostRegister), the set-up's scaling
 * kernels read them in place over the host link, without a staging copy; the
 * host arrays must then stay unchanged until the call returns. Device copies
 * are owned by the handle and released at the next call or in mss_destroy.
 * Errors: as mss_setup and mss_fgmres_solve. */
int mss_solve_host(mss_handle* h, const mss_bsr* J_host, int nb, mss_layout layout,
                   const mss_options* opt, const double* b_host, double* x_host, double tol,
                   int maxit, mss_result* out);

/* Residual check of the unscaled system for a given x: norms[0] =
 * ||b - J x||_2, norms[1] = ||b||_2 (Eq. reduced; the solver itself stops on
 * the scaled residual, Sec. 5.1). Any BSR matrix with row-major blocks; no
 * set-up is needed, the handle supplies the stream and the allocation hooks.
 * J, b, x: device, as in mss_setup; norms: device, 2 doubles, written in
 * stream order (the call does not synchronise). Scratch of 2 * n_rows
 * doubles is allocated through the handle's hooks for the call. The sums run
 * in a fixed order, so the result does not depend on the launch shape.
 * Errors: INVALID_ARG, OOM, CUDA. */
int mss_residual_norm(mss_handle* h, const mss_bsr* J, int nb, const double* b, const double* x,
                      double* norms);

/* mss_residual_norm without any device allocation. The paper has no
 * counterpart: this is a library convenience for callers that cannot call
 * cudaMalloc at the point of the call -- a process whose device memory pool
 * is wholly reserved by another framework, code inside a region where an
 * allocation call is not allowed (it would break a stream capture or
 * synchronise the device), or a latency-bound loop that must not enter the
 * allocator. Same kernels, arguments, result and errors as
 * mss_residual_norm, but the scratch (2 * n_rows doubles) lives in a static
 * device array sized for MSS_NOALLOC_MAX_CELLS cells (16 MiB), which every
 * GPU that loads the library holds until the process exits; n_rows above
 * the limit returns MSS_ERR_INVALID_ARG. No cudaMalloc, cudaFree or
 * allocating routine is called and the handle's hooks are not used. The
 * first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, on the current device, which must be the handle's);
 * make that first call before any stream capture. All calls share the array,
 * which keeps the last call's contents: each call writes every entry it reads
 * before reading it, but calls whose GPU work overlaps (on other streams or
 * from other threads) race on the array and must be serialised by the
 * caller. */
#define MSS_NOALLOC_MAX_CELLS (1 << 20)
int mss_residual_norm_noalloc(mss_handle* h, const mss_bsr* J, int nb, const double* b,
                              const double* x, double* norms);

/* ---- static condensation (Sec. 3, Eqs. global and reduced) ---------------
 * The simulator's global system [J11 J12; J21 J22] [d1; d2] = -[r1; r2] has
 * n1 primary and n2 secondary unknowns per cell, the secondary ones coupled
 * only inside their cell, so J12 and J22 are one block per cell. Eliminating
 * them gives the primary system A d1 = b that mss_setup takes:
 *   A = J11 - J12 J22^{-1} J21,  b = -r1 + J12 J22^{-1} r2,
 * with the cell graph's block pattern; afterwards the secondary unknowns are
 *   d2 = J22^{-1} (-r2 - J21 d1).
 * J22 is inverted per cell without pivoting (Sec. 3 aligns the secondary
 * equations with unknowns so that its pivots are nonzero). */
#define MSS_CONDENSE_MAX_UNKNOWNS 16
typedef struct {
  int32_t n_rows;           /* cells N */
  int32_t nnzb;             /* blocks of the cell graph */
  const int32_t* row_ptr;   /* device, N + 1 (as mss_bsr) */
  const int32_t* col_idx;   /* device, nnzb */
  int32_t n1;               /* primary unknowns per cell, 1..16 */
  int32_t n2;               /* secondary unknowns per cell, 0..16 */
  const double* j11;        /* device, nnzb blocks n1 x n1, row-major */
  const double* j21;        /* device, nnzb blocks n2 x n1 (secondary rows, primary columns) */
  const double* j12;        /* device, N blocks n1 x n2 (cell-local) */
  const double* j22;        /* device, N blocks n2 x n2 (cell-local) */
} mss_full;

/* a (device, nnzb * n1 * n1) receives A's blocks on J's pattern, b (device,
 * N * n1) the reduced right-hand side; r1 (N * n1) and r2 (N * n2, may be
 * NULL when n2 = 0) are device vectors, cell-interleaved. One pass, one warp
 * per cell, on the handle's stream; the call synchronises it to report
 * errors. Errors: INVALID_ARG (sizes, null pointers, a row_ptr entry outside
 * [0, nnzb]), SINGULAR_BLOCK (a J22 block needs pivoting), OOM, CUDA. */
int mss_condense(mss_handle* h, const mss_full* J, const double* r1, const double* r2,
                 double* a, double* b);

/* d2 (device, N * n2) = J22^{-1} (-r2 - J21 d1) per cell, for the primary
 * solution d1 (device, N * n1). Synchronises the handle's stream. Errors:
 * as mss_condense, and INVALID_ARG for a col_idx entry outside [0, N) or a
 * row of more than 64 blocks. */
int mss_recover(mss_handle* h, const mss_full* J, const double* r2, const double* d1,
                double* d2);

/* ---- introspection (tests) --------------------------------------------- */
/* Copy the scaled blocks Abar (device, nnzb*nb*nb, row-major) into `abar`
 * (device, caller-owned). */
int mss_get_scaled(mss_handle* h, double* abar);

/* Number of AMG levels of stage `which` (0 = C_TT, 1 = B_PP, or B_ee for
 * MSS_CPTR, whose levels are read in the scalar form with the (P, T) pair of
 * a point interleaved and the point split repeated per unknown); 0 if the
 * scheme has no such stage. */
int mss_amg_num_levels(mss_handle* h, int which);

/* sizes[0] = rows, sizes[1] = nnz(A_l), sizes[2] = nnz(P_l) (0 on the
 * coarsest level); host array of 3. */
int mss_amg_level_sizes(mss_handle* h, int which, int level, int32_t* sizes);

/* Copy level `level` of stage `which` into caller-owned device arrays sized
 * from mss_amg_level_sizes: A_l (rp, ci, v), the C/F split (1 = C), and the
 * interpolation P_l (rp, ci, v). cf and P are not written on the coarsest
 * level. */
int mss_amg_level_copy(mss_handle* h, int which, int level, int32_t* arp, int32_t* aci,
                       double* av, int32_t* cf, int32_t* prp, int32_t* pci, double* pv);

/* Number of colours of the block ILU(0) ordering (host int). */
int mss_bilu_num_colours(mss_handle* h, int32_t* ncolours);

/* Copy the cell colours and the ordering (perm[k] = cell at position k)
 * into caller-owned device arrays of N entries. */
int mss_bilu_ordering(mss_handle* h, int32_t* colour, int32_t* perm);

/* Copy the block ILU(0) factors of Eq. CPTR3M3 (the CPR second stage) in
 * colour-major positions: fv (device, nnzb*nb*nb, row-major blocks, rows in
 * position order, blocks of a row in ascending column position) holds the
 * strictly lower blocks L_qk (unit diagonal implied), the pivot block U_qq
 * and the upper blocks U_qj, except that the upper blocks coupling two cells
 * of one strip hold U_qq^{-1} U_qj (the form the strip chains read);
 * fdinv (device, N*nb*nb) holds U_qq^{-1} per position. Either pointer may
 * be NULL. Errors: NOT_SETUP; INVALID_ARG for block Jacobi (no factors). */
int mss_bilu_factors(mss_handle* h, double* fv, double* fdinv);

/* Runs, on the handle's stream, one wait of the grid barrier used by the
 * fused coarse V-cycle levels that can never complete (it expects a block
 * that is not launched). The wait gives up after its poll limit (well under
 * a second), sets the barrier's error flag and the kernel returns, leaving
 * the context usable. *timed_out (host) = 1 when that happened. */
int mss_probe_wait_limit(mss_handle* h, int32_t* timed_out);

/* ---- measurement --------------------------------------------------------- */
/* Number of kernel launches made by this library in this process since the
 * last call with reset != 0 (the count before the reset is returned). */
long long mss_kernel_launches(int reset);

/* Event trace of kernel classes: when enabled, CUDA events recorded on the
 * handle's stream bracket every BSR matrix-vector product (kind 0), every
 * forward (1) and backward (2) last-stage sweep launch, every V-cycle (3),
 * every Arnoldi orthogonalisation step (4), the set-up phases: scaling
 * (5), the span in which the two AMG hierarchies are built on worker streams
 * while the last stage is ordered and factorised (6), that ordering and
 * factorisation alone (7), every whole preconditioner application (8), and
 * the kernels of mss_condense (9) and mss_recover (10).
 * Solves run with MSS_DRIVER_GRAPH record no events (a graph holds none). */
int mss_trace_enable(mss_handle* h, int enable);

/* Totals for one kind since the last reset: number of bracketed regions
 * and their summed elapsed GPU time in ms (host pointers, may be NULL).
 * Synchronises the stream. reset != 0 zeroes the kind's totals after
 * reading. Errors: INVALID_ARG for an unknown kind. */
int mss_trace_read(mss_handle* h, int kind, int64_t* launches, double* ms, int reset);

/* ---- batched solves (not in the paper) ------------------------------------
 * Many independent systems of different sizes, set up and solved
 * concurrently: a pool of `lanes` host worker threads, each driving its own
 * handle on its own CUDA stream (memory from the library's stream-ordered
 * device pool), takes the systems largest first. Every system is set up and
 * solved exactly as by mss_setup + mss_fgmres_solve with the given options,
 * so its solution is the one a single handle gives, bit for bit.
 *
 * Autotuner (autotune != 0): the first system of each size bucket
 * (floor(log2 N), nb) is used to time the preconditioner application and the
 * matrix-vector product at 64, 128, 256 and 512 threads per CTA (the result
 * does not depend on it) and one solve with each driver (host loop, or the
 * CUDA graph including its capture); the fastest choice is cached in the
 * batch object for later systems of the bucket. With autotune == 0 every
 * system uses 256 threads and the driver in the options.
 *
 * Fused schedule (mss_batch_set_schedule(b, MSS_SCHEDULE_FUSED)): the lanes
 * set the systems up, each on a handle of its own; then the systems of each
 * block size are solved in lock step as one group: every kernel launch of the
 * restarted FGMRES and of the preconditioner serves all systems of the group.
 * A launch walks a list of tiles (runs of blocks of one system's own launch of
 * that kernel) with CTAs that stay resident and take tile after tile, and the
 * whole group solve is one CUDA graph whose loops run while any system takes
 * another step. Each system still computes exactly the values of its own
 * solve (same kernels' bodies, same launch shapes per system), so solutions
 * and iteration counts equal the lanes schedule's bit for bit. The tile shape
 * (blocks per tile, resident CTAs per SM) is tuned on the group's first
 * preconditioner application and product and cached per (floor(log2 of the
 * group's rows), nb) (fixed at 1 block and 4 CTAs with autotune == 0). It
 * covers FP64 solves with Jacobi smoothing (CPTR3, CPR, ILU0) and nb <= 8;
 * other systems take the lanes schedule. Every system of a group finishes with
 * the group: latency is traded for throughput.
 *
 * Both schedules keep many streams busy at once; a process that sets
 * CUDA_DEVICE_MAX_CONNECTIONS (e.g. 32) before CUDA starts gives them more
 * hardware work queues than the default 8 (streams sharing a queue wait on
 * each other's work). */
enum { MSS_SCHEDULE_LANES = 0, MSS_SCHEDULE_FUSED = 1 };

typedef struct {
  mss_bsr J;                /* device arrays, as for mss_setup */
  int32_t nb;
  mss_layout layout;
  const double* b;          /* device, n_rows * nb */
  double* x;                /* device, n_rows * nb: the solution (x0 = 0) */
} mss_system;

typedef struct {
  int32_t bucket;           /* floor(log2(n_rows)) */
  int32_t threads;          /* threads per CTA used */
  int32_t driver;           /* MSS_DRIVER_* used */
  int32_t lane;             /* worker that solved it (fused: the worker that set it up) */
  double latency_ms;        /* host clock: start of its set-up to end of its solve */
  double finish_ms;         /* host clock: start of the batch call to end of its solve */
  int32_t schedule;         /* MSS_SCHEDULE_* that solved it */
  int32_t group;            /* fused: its group (systems of one nb); lanes: -1 */
  int32_t tile_blocks;      /* fused: blocks of a system's launch per tile */
  int32_t per_sm;           /* fused: resident CTAs per SM of each launch */
} mss_batch_info;

typedef struct mss_batch mss_batch;

/* lanes: worker threads, 1..64. Handles are created on the current device.
 * Errors: INVALID_ARG, CUDA, OOM. */
int mss_batch_create(mss_batch** b, int lanes, int autotune);
void mss_batch_destroy(mss_batch* b);

/* MSS_SCHEDULE_LANES (default) or MSS_SCHEDULE_FUSED for later
 * mss_batch_solve calls. Errors: INVALID_ARG. */
int mss_batch_set_schedule(mss_batch* b, int schedule);

/* Sets up and solves the n systems (tol, maxit as for mss_fgmres_solve; opt
 * NULL = defaults). The device is synchronised first, so inputs written on
 * any stream are complete; every solution is complete on return.
 * results[i] (host, n entries) is system i's outcome (status per system: one
 * failing system does not stop the others); info (host, n entries, may be
 * NULL) its schedule. Returns MSS_OK when every system converged, else the
 * first non-OK system status; INVALID_ARG for bad arguments. */
int mss_batch_solve(mss_batch* b, int n, const mss_system* sys, const mss_options* opt,
                    double tol, int maxit, mss_result* results, mss_batch_info* info);

/* The autotuner's cache: up to cap entries of 4 int32 each (bucket, nb,
 * threads, driver) written to out (host); returns the number of entries. */
int mss_batch_tuned(mss_batch* b, int cap, int32_t* out);

/* Message for the last failing call on `b`. */
const char* mss_batch_last_error(const mss_batch* b);

/* ---- learned temperature interpolation (not in the paper) -----------------
 * The paper's temperature stage is classical AMG (Sec. 5.1). Here a
 * message-passing network of width 32 on the graph of the level-0 temperature
 * operator A = C_TT predicts a relative correction s_ij of every classical
 * interpolation weight p_ij (F point i, C point j): w_ij = p_ij (1 + s_ij),
 * so a network with a zero read-out is classical interpolation exactly.
 *   x_i  = [a_ii / mean a_kk, sum_j a_ij / a_ii]                (node input)
 *   e_ij = [a_ij/a_ii, a_ji/a_jj, |a_ij| / max_k|a_ik|, cf_i, cf_j] (edge input)
 *   H0 = relu(X Wn + bn), G = relu(E We + be)
 *   l = 1..3: M_i = sum_j G_ij * H_j, H^l = relu([H^{l-1} | M] W_l + b_l)
 *   z = relu([H3_i | H3_j | G_ij] Wo + bo), s_ij = z . wr + br
 * Training loss on test vectors e_k (nu damped-Jacobi sweeps on A e = 0 from
 * given starts) with the defect d_k = e_k - P e_k|C (zero at C points):
 * norm 0: L = sum_k ||A d_k||^2 / sum_k ||A e_k||^2 (residual);
 * norm 1: L = sum_k sum_i |a_ii| d_ki^2 / sum_k sum_i |a_ii| e_ki^2 (the
 * least-squares interpolation criterion of bootstrap AMG).
 * Parameters: one float vector, in order Wn 2x32, bn 32, We 5x32, be 32,
 * W1 64x32, b1 32, W2 64x32, b2 32, W3 64x32, b3 32, Wo 96x32, bo 32, wr 32,
 * br 1 (matrices row-major [in x out]). Dense layers run on BF16 tensor cores
 * with FP32 accumulation; the loss is FP64. */
int mss_gnn_num_params(void);

typedef struct mss_gnn mss_gnn;

/* A training graph from h's current set-up (CPTR3 with at least two
 * temperature levels): level 0's operator, C/F split and classical
 * interpolation are copied, so neither later set-ups nor the destruction of
 * h affect it. The graph has its own stream and takes memory from the
 * library's device pool. The calls below synchronise the device on entry
 * (their inputs may come from any stream) and the graph's stream on return.
 * Errors: NOT_SETUP, INVALID_ARG (no such hierarchy; a pattern without one
 * diagonal per row or not structurally symmetric). */
int mss_gnn_create(mss_handle* h, mss_gnn** g);
void mss_gnn_destroy(mss_gnn* g);

/* nodes n, off-diagonal edges m, interpolation entries t of F rows (host
 * pointers, may be NULL). */
int mss_gnn_info(const mss_gnn* g, int32_t* n, int32_t* m, int32_t* t);

/* Test vectors: starts (device, n x K row-major, K in [1, 64]) smoothed by nu
 * damped-Jacobi sweeps with weight omega; norm selects the loss (0 or 1). */
int mss_gnn_set_vectors(mss_gnn* g, int K, const double* starts, int nu, double omega,
                        int norm);

/* w (device, t doubles): the learned weights, entries in row order of P. */
int mss_gnn_weights(mss_gnn* g, const float* params, double* w);

/* loss (host, may be NULL) and its gradient (device, mss_gnn_num_params()
 * floats, may be NULL) for params (device). Errors: NOT_SETUP without test
 * vectors. */
int mss_gnn_loss_grad(mss_gnn* g, const float* params, double* loss, float* grad);

/* One Adam step (Kingma and Ba) on device arrays of mss_gnn_num_params()
 * floats, on g's stream; step counts from 1. */
int mss_gnn_adam(mss_gnn* g, float* params, float* m1, float* m2, const float* grad, int step,
                 float lr, float beta1, float beta2, float eps);

/* Message for the last failing call on `g`. */
const char* mss_gnn_last_error(const mss_gnn* g);

/* Human-readable name of a status code (static string). */
const char* mss_status_string(int status);

/* Message for the last failing call on `h` (valid until the next call). */
const char* mss_last_error(const mss_handle* h);

#ifdef __cplusplus
}
#endif

#endif /* MSS_H */
