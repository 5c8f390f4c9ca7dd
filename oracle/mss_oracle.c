/*
 * mss_oracle.c -- plain, slow FP64 CPU oracle for the multi-stage CPR / CPTR3
 * preconditioner inside right-preconditioned FGMRES (arXiv:1912.04385).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load this library. It shares no code, header
 * or constant with the CUDA library; the two meet only through the seeded
 * synthetic inputs.
 *
 * Every routine follows the paper's statement of the method step by step:
 *   - split preconditioning and left scaling ........ Sec. 4, Eqs. splitPrec1/2
 *   - CPR decoupling ................................ Sec. 4.1, Eq. CPR
 *   - CPTR3 decoupling N1, N2 ....................... Sec. 4.3, Eqs. CPTR31, CPTR32
 *   - cell-local ("diag") Schur approximations ...... Sec. 4.1, Remark 3
 *   - stage operators ............................... Eqs. CPRM1, CPTR3M1, CPTRM2, CPTR3M3
 *   - stage application ............................. Algorithms 1 and 2
 *   - multi-stage composition ....................... Eq. multistageprec
 *   - exact sub-solvers ............................. Sec. 5.1 (direct-solver study)
 *   - classical AMG, V-cycle, coarse <= 1000 ........ Sec. 5.1 (HSL_MI20 settings)
 *   - GMRES, right-preconditioned, relative tol ..... Sec. 5.1
 * Where the paper is silent (PMIS coarsening, interpolation formula,
 * smoothers, block ILU ordering, restarted FGMRES) the routine states the
 * reading it implements.
 *
 * Conventions: BSR blocks are row-major nb x nb, cell-interleaved vectors
 * (cell i, unknown k at i*nb + k). Columns ascend within every row.
 * Build with FMA contraction disabled (-ffp-contract=off) so that every
 * floating-point operation rounds exactly as written.
 *
 * Parity status per function is stated where the function is defined.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_ARG (-1)
#define OR_ERR_SINGULAR (-2)
#define OR_ERR_NOT_CONVERGED (-3)
#define OR_ERR_BREAKDOWN (-4)
#define OR_ERR_MEM (-5)
#define OR_ERR_AMG (-6)

#define OR_MAXLEV 25
#define OR_MAX_DENSE 8192

/* ------------------------------------------------------------------------ */
/* options                                                                  */
/* ------------------------------------------------------------------------ */
typedef struct {
  int scheme;        /* 0 CPTR3 (three stages), 1 CPR (two stages), 2 ILU only,
                        3 CPTR (two stages, system AMG on the 2 x 2 block B_ee) */
  int stage_order;   /* 0: T stage then P stage (Alg. 2 order); 1: P then T */
  int exact_sub;     /* 1: M_TT = C_TT^-1 and M_PP = B_PP^-1 by dense LU */
  int stage3;        /* 0: block ILU(0) of the scaled matrix, 1: block Jacobi */
  int ilu_order;     /* 0: multicolour (Jones-Plassmann), 1: natural, 2: strips
                        coloured first-fit in strip order, 3: strips coloured by
                        Jones-Plassmann */
  int smoother;      /* 0: damped Jacobi, 1: Chebyshev, 2: symmetric Gauss-Seidel,
                        3: multicolour symmetric Gauss-Seidel */
  int nu_pre, nu_post;
  int cheb_degree;
  int max_coarse, max_levels, interp_max;
  int restart;
  int ilu_strip;     /* strip length (cells) of the strip ordering */
  double theta, omega, cheb_lo_ratio, cheb_hi_factor;
  uint64_t seed;
} or_opts;

typedef struct {
  int iters, restarts, status, pad_;
  double rel_res_implicit, rel_res_true;
} or_result;

void or_opts_default(or_opts* o) {
  memset(o, 0, sizeof(*o));
  o->scheme = 0;
  o->stage_order = 0;
  o->exact_sub = 0;
  o->stage3 = 0;
  o->ilu_order = 2;      /* strips of ilu_strip cells (reading) */
  o->smoother = 0;
  o->nu_pre = 2;          /* HSL_MI20 defaults (Sec. 5.1): 2 pre-, 2 post-sweeps */
  o->nu_post = 2;
  o->cheb_degree = 2;
  o->max_coarse = 1000;   /* Sec. 5.1: maximum coarse problem size 1000 */
  o->max_levels = 25;
  o->interp_max = 4;
  o->restart = 30;
  o->ilu_strip = 32;
  o->theta = 0.25;
  o->omega = 0.8;          /* HSL_MI20's default Jacobi damping */
  o->cheb_lo_ratio = 30.0;
  o->cheb_hi_factor = 1.0;
  o->seed = 0x5eedULL;
}

/* ------------------------------------------------------------------------ */
/* small helpers                                                            */
/* ------------------------------------------------------------------------ */
typedef struct { int n, m, nnz; int* rp; int* ci; double* v; } csr_t;

static void csr_free(csr_t* a) {
  free(a->rp); free(a->ci); free(a->v);
  memset(a, 0, sizeof(*a));
}

static int csr_alloc(csr_t* a, int n, int m, int nnz) {
  a->n = n; a->m = m; a->nnz = nnz;
  a->rp = (int*)calloc((size_t)n + 1, sizeof(int));
  a->ci = (int*)malloc(sizeof(int) * (size_t)(nnz > 0 ? nnz : 1));
  a->v = (double*)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
  return (a->rp && a->ci && a->v) ? OR_OK : OR_ERR_MEM;
}

/* SplitMix64 (Steele, Lea, Flood 2014) as a counter-based generator: the
 * value for counter k is the (k+1)-th output of the sequence seeded with
 * `seed`, i.e. mix(seed + (k+1) * golden_gamma). */
static uint64_t or_splitmix(uint64_t seed, uint64_t k) {
  uint64_t z = seed + (k + 1ULL) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* uniform double in [0, 1) from the top 53 bits */
static double or_unit(uint64_t h) { return (double)(h >> 11) * (1.0 / 9007199254740992.0); }

static double dot(int n, const double* a, const double* b) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

static double nrm2(int n, const double* a) { return sqrt(dot(n, a, a)); }

/* Gauss-Jordan inverse without pivoting (the paper's orderings keep the
 * cell blocks invertible without pivoting, Sec. 3). a, inv: m x m row-major.
 * The eliminations use IEEE fused multiply-adds (one rounding per update),
 * as do the scaling's dot products below. */
static int gj_inverse_nopiv(int m, const double* a_in, double* inv) {
  double a[32 * 32];
  if (m > 32) return OR_ERR_ARG;
  memcpy(a, a_in, sizeof(double) * (size_t)m * m);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) inv[i * m + j] = (i == j) ? 1.0 : 0.0;
  for (int k = 0; k < m; ++k) {
    double piv = a[k * m + k];
    if (piv == 0.0 || !isfinite(piv)) return OR_ERR_SINGULAR;
    double rpiv = 1.0 / piv;     /* the pivot row is scaled by the reciprocal */
    for (int j = 0; j < m; ++j) {
      a[k * m + j] = a[k * m + j] * rpiv;
      inv[k * m + j] = inv[k * m + j] * rpiv;
    }
    for (int i = 0; i < m; ++i) {
      if (i == k) continue;
      double f = a[i * m + k];
      for (int j = 0; j < m; ++j) {
        a[i * m + j] = fma(-f, a[k * m + j], a[i * m + j]);
        inv[i * m + j] = fma(-f, inv[k * m + j], inv[i * m + j]);
      }
    }
  }
  return OR_OK;
}

/* Solve a x = b (m x m, no pivoting) by Gaussian elimination; x holds b on
 * entry. */
static int ge_solve_nopiv(int m, const double* a_in, double* x) {
  double a[32 * 32];
  if (m > 32) return OR_ERR_ARG;
  memcpy(a, a_in, sizeof(double) * (size_t)m * m);
  for (int k = 0; k < m; ++k) {
    double piv = a[k * m + k];
    if (piv == 0.0 || !isfinite(piv)) return OR_ERR_SINGULAR;
    for (int i = k + 1; i < m; ++i) {
      double f = a[i * m + k] / piv;
      for (int j = k; j < m; ++j) a[i * m + j] -= f * a[k * m + j];
      x[i] -= f * x[k];
    }
  }
  for (int k = m - 1; k >= 0; --k) {
    double s = x[k];
    for (int j = k + 1; j < m; ++j) s -= a[k * m + j] * x[j];
    x[k] = s / a[k * m + k];
  }
  return OR_OK;
}

/* Dense LU with partial pivoting (row-major n x n), in place. */
static int lu_factor(int n, double* a, int* piv) {
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = fabs(a[(size_t)k * n + k]);
    for (int i = k + 1; i < n; ++i) {
      double v = fabs(a[(size_t)i * n + k]);
      if (v > best) { best = v; p = i; }
    }
    piv[k] = p;
    if (best == 0.0 || !isfinite(best)) return OR_ERR_SINGULAR;
    if (p != k)
      for (int j = 0; j < n; ++j) {
        double t = a[(size_t)k * n + j];
        a[(size_t)k * n + j] = a[(size_t)p * n + j];
        a[(size_t)p * n + j] = t;
      }
    double d = a[(size_t)k * n + k];
    for (int i = k + 1; i < n; ++i) {
      double f = a[(size_t)i * n + k] / d;
      a[(size_t)i * n + k] = f;
      if (f != 0.0)
        for (int j = k + 1; j < n; ++j) a[(size_t)i * n + j] -= f * a[(size_t)k * n + j];
    }
  }
  return OR_OK;
}

static void lu_solve(int n, const double* lu, const int* piv, double* x) {
  for (int k = 0; k < n; ++k) {
    int p = piv[k];
    if (p != k) { double t = x[k]; x[k] = x[p]; x[p] = t; }
  }
  for (int i = 0; i < n; ++i) {
    double s = x[i];
    for (int j = 0; j < i; ++j) s -= lu[(size_t)i * n + j] * x[j];
    x[i] = s;
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = x[i];
    for (int j = i + 1; j < n; ++j) s -= lu[(size_t)i * n + j] * x[j];
    x[i] = s / lu[(size_t)i * n + i];
  }
}

/* y = A x for a scalar CSR matrix */
static void csr_mv(const csr_t* a, const double* x, double* y) {
  for (int i = 0; i < a->n; ++i) {
    double s = 0.0;
    for (int e = a->rp[i]; e < a->rp[i + 1]; ++e) s += a->v[e] * x[a->ci[e]];
    y[i] = s;
  }
}

/* C = A * B by rows (Gustavson): for row i, contributions a_ik * b_kj are
 * accumulated in ascending k, then ascending j within row k; the output row
 * is sorted by column. */
static int csr_matmul(const csr_t* A, const csr_t* B, csr_t* C) {
  int n = A->n, m = B->m;
  int* mark = (int*)malloc(sizeof(int) * (size_t)(m > 0 ? m : 1));
  double* acc = (double*)calloc((size_t)(m > 0 ? m : 1), sizeof(double));
  int* cols = (int*)malloc(sizeof(int) * (size_t)(m > 0 ? m : 1));
  int* rp = (int*)calloc((size_t)n + 1, sizeof(int));
  if (!mark || !acc || !cols || !rp) return OR_ERR_MEM;
  for (int j = 0; j < m; ++j) mark[j] = -1;
  /* symbolic */
  for (int i = 0; i < n; ++i) {
    int cnt = 0;
    for (int e = A->rp[i]; e < A->rp[i + 1]; ++e) {
      int k = A->ci[e];
      for (int f = B->rp[k]; f < B->rp[k + 1]; ++f) {
        int j = B->ci[f];
        if (mark[j] != i) { mark[j] = i; ++cnt; }
      }
    }
    rp[i + 1] = rp[i] + cnt;
  }
  if (csr_alloc(C, n, m, rp[n]) != OR_OK) return OR_ERR_MEM;
  memcpy(C->rp, rp, sizeof(int) * ((size_t)n + 1));
  for (int j = 0; j < m; ++j) mark[j] = -1;
  for (int i = 0; i < n; ++i) {
    int cnt = 0;
    for (int e = A->rp[i]; e < A->rp[i + 1]; ++e) {
      int k = A->ci[e];
      double aik = A->v[e];
      for (int f = B->rp[k]; f < B->rp[k + 1]; ++f) {
        int j = B->ci[f];
        if (mark[j] != i) { mark[j] = i; acc[j] = 0.0; cols[cnt++] = j; }
        acc[j] = acc[j] + aik * B->v[f];
      }
    }
    /* insertion sort of the touched columns */
    for (int a = 1; a < cnt; ++a) {
      int c = cols[a], b = a - 1;
      while (b >= 0 && cols[b] > c) { cols[b + 1] = cols[b]; --b; }
      cols[b + 1] = c;
    }
    for (int a = 0; a < cnt; ++a) {
      C->ci[rp[i] + a] = cols[a];
      C->v[rp[i] + a] = acc[cols[a]];
    }
  }
  free(mark); free(acc); free(cols); free(rp);
  return OR_OK;
}

/* B = A^T, rows sorted by column */
static int csr_transpose(const csr_t* A, csr_t* B) {
  if (csr_alloc(B, A->m, A->n, A->nnz) != OR_OK) return OR_ERR_MEM;
  for (int e = 0; e < A->nnz; ++e) B->rp[A->ci[e] + 1]++;
  for (int j = 0; j < A->m; ++j) B->rp[j + 1] += B->rp[j];
  int* fill = (int*)malloc(sizeof(int) * (size_t)(A->m > 0 ? A->m : 1));
  if (!fill) return OR_ERR_MEM;
  for (int j = 0; j < A->m; ++j) fill[j] = B->rp[j];
  for (int i = 0; i < A->n; ++i)          /* ascending i -> sorted rows */
    for (int e = A->rp[i]; e < A->rp[i + 1]; ++e) {
      int j = A->ci[e];
      B->ci[fill[j]] = i;
      B->v[fill[j]] = A->v[e];
      fill[j]++;
    }
  free(fill);
  return OR_OK;
}

static int csr_diag_pos(const csr_t* a, int i) {
  for (int e = a->rp[i]; e < a->rp[i + 1]; ++e)
    if (a->ci[e] == i) return e;
  return -1;
}

/* ------------------------------------------------------------------------ */
/* left scaling N^{-1} (Sec. 4, Eqs. CPR, CPTR31, CPTR32)                   */
/* ------------------------------------------------------------------------ */
/* Builds the cell scaling matrix W = N^{-1} restricted to one cell from the
 * cell's diagonal block D. The "diag" approximations D_xy of Remark 3 are the
 * cell-local parts of the diagonal block (our reading: dense sub-blocks of
 * the nb x nb cell block, not scalar diagonals).
 *
 * CPTR3 (Eq. CPTR31 then CPTR32):
 *   N1^{-1}: row P <- row P - D_Ps D_ss^{-1} (rows s); same for row T.
 *   N2^{-1}: row T <- row T - D_Tp D_PP^{-1} (row P), where D_Tp and D_PP are
 *            entries of the once-scaled block N1^{-1} D (the B blocks).
 *   W = N2^{-1} N1^{-1}.
 * CPR (Eq. CPR): h = all unknowns but P; row P <- row P - D_Ph D_hh^{-1} (rows h).
 * CPTR (Eq. CPTR1): e = {P, T}; rows e <- rows e - D_es D_ss^{-1} (rows s), which
 *   is N1 of CPTR3 alone.
 * ILU only: W = I (no decoupling for the single-stage baseline).
 * Parity: pinned (tests check the zero pattern of W D, det W = 1 and the
 * invariance of the solution).
 */
static int build_scaling(int nb, int p, int t, int scheme, const double* D, double* W) {
  double n1[32 * 32];
  for (int i = 0; i < nb; ++i)
    for (int j = 0; j < nb; ++j) W[i * nb + j] = (i == j) ? 1.0 : 0.0;
  if (scheme == 2) return OR_OK;
  if (scheme == 1) {
    int h[32], nh = 0;
    for (int k = 0; k < nb; ++k) if (k != p) h[nh++] = k;
    double Dhh[32 * 32], inv[32 * 32];
    for (int a = 0; a < nh; ++a)
      for (int b = 0; b < nh; ++b) Dhh[a * nh + b] = D[h[a] * nb + h[b]];
    int st = gj_inverse_nopiv(nh, Dhh, inv);
    if (st) return st;
    for (int b = 0; b < nh; ++b) {
      double w = 0.0;
      for (int a = 0; a < nh; ++a) w = fma(D[p * nb + h[a]], inv[a * nh + b], w);
      W[p * nb + h[b]] = -w;
    }
    return OR_OK;
  }
  /* CPTR3 */
  int s[32], ns = 0;
  for (int k = 0; k < nb; ++k) if (k != p && k != t) s[ns++] = k;
  for (int i = 0; i < nb * nb; ++i) n1[i] = W[i];
  if (ns > 0) {
    double Dss[32 * 32], inv[32 * 32];
    for (int a = 0; a < ns; ++a)
      for (int b = 0; b < ns; ++b) Dss[a * ns + b] = D[s[a] * nb + s[b]];
    int st = gj_inverse_nopiv(ns, Dss, inv);
    if (st) return st;
    for (int b = 0; b < ns; ++b) {
      double wp = 0.0, wt = 0.0;
      for (int a = 0; a < ns; ++a) {
        wp = fma(D[p * nb + s[a]], inv[a * ns + b], wp);
        wt = fma(D[t * nb + s[a]], inv[a * ns + b], wt);
      }
      n1[p * nb + s[b]] = -wp;
      n1[t * nb + s[b]] = -wt;
    }
  }
  if (scheme == 3) {   /* CPTR (Eq. CPTR1): the lower block factor of [s | e] only */
    for (int k = 0; k < nb * nb; ++k) W[k] = n1[k];
    return OR_OK;
  }
  /* once-scaled entries B_PP and B_Tp of N1^{-1} D */
  double bpp = 0.0, btp = 0.0;
  for (int k = 0; k < nb; ++k) {
    bpp = fma(n1[p * nb + k], D[k * nb + p], bpp);
    btp = fma(n1[t * nb + k], D[k * nb + p], btp);
  }
  if (bpp == 0.0 || !isfinite(bpp)) return OR_ERR_SINGULAR;
  double c = btp / bpp;
  for (int k = 0; k < nb * nb; ++k) W[k] = n1[k];
  for (int k = 0; k < nb; ++k) W[t * nb + k] = fma(-c, n1[p * nb + k], n1[t * nb + k]);
  return OR_OK;
}

/* out = W in  (nb x nb blocks, row-major), accumulation over ascending k with
 * fused multiply-adds */
static void block_left_mul(int nb, const double* W, const double* in, double* out) {
  for (int r = 0; r < nb; ++r)
    for (int c = 0; c < nb; ++c) {
      double acc = 0.0;
      for (int k = 0; k < nb; ++k) acc = fma(W[r * nb + k], in[k * nb + c], acc);
      out[r * nb + c] = acc;
    }
}

static void block_vec_left_mul(int nb, const double* W, const double* in, double* out) {
  for (int r = 0; r < nb; ++r) {
    double acc = 0.0;
    for (int k = 0; k < nb; ++k) acc = fma(W[r * nb + k], in[k], acc);
    out[r] = acc;
  }
}

/* ------------------------------------------------------------------------ */
/* classical AMG setup (Sec. 5.1 settings; coarsening reading: PMIS)        */
/* ------------------------------------------------------------------------ */
typedef struct {
  csr_t A;
  unsigned char* strong;   /* per nonzero of A */
  int* cf;                 /* 1 C point, 0 F point */
  int* cidx;               /* coarse index of C points, -1 for F */
  csr_t P, R;
  double* dinv;
  double lam_max;
  double *b, *x, *r, *t1, *t2;
  int nc;
  int ncolour;             /* multicolour Gauss-Seidel: colours of A's graph */
  int* cstart;             /* colour c holds mcorder[cstart[c] .. cstart[c + 1]) */
  int* mcorder;            /* points in colour-major order, ascending inside a colour */
  double* dinv2;           /* system AMG: inverse of each point's 2 x 2 diagonal block */
} level_t;

typedef struct {
  int nlev;
  level_t lev[OR_MAXLEV];
  double* lu;
  int* piv;
  or_opts o;
  int bs;                  /* unknowns per point: 1 scalar AMG, 2 system AMG (CPTR) */
} amg_t;

/* Strength of connection, sign-aware classical rule (reading): j is strong
 * for i if -sgn(a_ii) a_ij >= theta * max_{k != i} (-sgn(a_ii) a_ik) and that
 * maximum is positive. Parity: pinned through the 1D / 2D Poisson tests. */
static void amg_strength(const csr_t* A, double theta, unsigned char* strong) {
  for (int i = 0; i < A->n; ++i) {
    int d = csr_diag_pos(A, i);
    double aii = d >= 0 ? A->v[d] : 0.0;
    double sg = aii < 0.0 ? 1.0 : -1.0;     /* -sgn(a_ii) */
    double mx = -INFINITY;
    for (int e = A->rp[i]; e < A->rp[i + 1]; ++e)
      if (A->ci[e] != i) {
        double v = sg * A->v[e];
        if (v > mx) mx = v;
      }
    double thr = theta * mx;
    for (int e = A->rp[i]; e < A->rp[i + 1]; ++e) {
      strong[e] = 0;
      if (A->ci[e] != i && mx > 0.0 && sg * A->v[e] >= thr) strong[e] = 1;
    }
  }
}

/* PMIS coarsening (De Sterck, Yang, Heys 2006), synchronous rounds.
 * measure lambda_i = |S_i^T| + u_i, u_i = uniform(seed, level, i);
 * points that influence nobody start as F; per round every undecided point
 * whose (lambda, index) exceeds that of all undecided strong neighbours (in
 * either direction) becomes C, then undecided points that depend strongly on
 * a new C point become F. Afterwards an F point that depends strongly on some
 * point but on no C point is made C. pre / rnd (may be NULL) receive the
 * split before that fix-up (1 C, 0 F) and the round in which each point was
 * decided (0: influences nobody, F from the start). Parity: index work, compared bit-exactly;
 * pinned by the split invariants and the Poisson convergence tests. */
static int amg_pmis(const csr_t* A, const unsigned char* strong, uint64_t seed, int level,
                    int* cf, int* pre, int* rnd) {
  int n = A->n;
  int* cnt = (int*)calloc((size_t)(n > 0 ? n : 1), sizeof(int));
  double* lam = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  int* state = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));  /* -1 undecided, 0 F, 1 C */
  int* newc = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  /* transposed strength graph */
  csr_t S, ST;
  if (!cnt || !lam || !state || !newc) return OR_ERR_MEM;
  int ns = 0;
  for (int e = 0; e < A->nnz; ++e) ns += strong[e];
  if (csr_alloc(&S, n, n, ns) != OR_OK) return OR_ERR_MEM;
  for (int i = 0, q = 0; i < n; ++i) {
    for (int e = A->rp[i]; e < A->rp[i + 1]; ++e)
      if (strong[e]) { S.ci[q] = A->ci[e]; S.v[q] = 1.0; ++q; }
    S.rp[i + 1] = q;
  }
  if (csr_transpose(&S, &ST) != OR_OK) return OR_ERR_MEM;
  for (int i = 0; i < n; ++i) {
    cnt[i] = ST.rp[i + 1] - ST.rp[i];
    uint64_t key = ((uint64_t)(unsigned)level << 32) | (uint64_t)(unsigned)i;
    lam[i] = (double)cnt[i] + or_unit(or_splitmix(seed, key));
    state[i] = cnt[i] == 0 ? 0 : -1;
    if (rnd) rnd[i] = 0;
  }
  int round = 0;
#define OR_GT(a, b) (lam[a] > lam[b] || (lam[a] == lam[b] && (a) > (b)))
  for (;;) {
    int undecided = 0;
    for (int i = 0; i < n; ++i) undecided += state[i] == -1;
    if (!undecided) break;
    ++round;
    for (int i = 0; i < n; ++i) {
      newc[i] = 0;
      if (state[i] != -1) continue;
      int ismax = 1;
      for (int e = S.rp[i]; e < S.rp[i + 1] && ismax; ++e) {
        int j = S.ci[e];
        if (state[j] == -1 && OR_GT(j, i)) ismax = 0;
      }
      for (int e = ST.rp[i]; e < ST.rp[i + 1] && ismax; ++e) {
        int j = ST.ci[e];
        if (state[j] == -1 && OR_GT(j, i)) ismax = 0;
      }
      newc[i] = ismax;
    }
    for (int i = 0; i < n; ++i)
      if (newc[i]) {
        state[i] = 1;
        if (rnd) rnd[i] = round;
      }
    for (int i = 0; i < n; ++i) {
      if (state[i] != -1) continue;
      for (int e = S.rp[i]; e < S.rp[i + 1]; ++e)
        if (newc[S.ci[e]]) {
          state[i] = 0;
          if (rnd) rnd[i] = round;
          break;
        }
    }
  }
#undef OR_GT
  if (pre) for (int i = 0; i < n; ++i) pre[i] = state[i];
  /* F points with strong dependencies but no strong C point become C */
  for (int i = 0; i < n; ++i) {
    newc[i] = 0;
    if (state[i] != 0 || S.rp[i + 1] == S.rp[i]) continue;
    int hasc = 0;
    for (int e = S.rp[i]; e < S.rp[i + 1]; ++e) hasc |= state[S.ci[e]] == 1;
    newc[i] = !hasc;
  }
  for (int i = 0; i < n; ++i) cf[i] = (state[i] == 1 || newc[i]) ? 1 : 0;
  csr_free(&S); csr_free(&ST);
  free(cnt); free(lam); free(state); free(newc);
  return OR_OK;
}

/* Classical (Ruge-Stueben direct, with distribution of strong F couplings)
 * interpolation, sign-aware (reading). For an F point i with strong C set
 * C_i, weak set W_i and strong F set F_i:
 *   d_i   = a_ii + sum_{j in W_i} a_ij  (+ a_ik for k in F_i with sigma_k = 0)
 *   sigma_k = sum_{m in C_i, sgn(a_km) != sgn(a_kk)} a_km
 *   w_ij  = -( a_ij + sum_{k in F_i, sigma_k != 0} a_ik a_kj' / sigma_k ) / d_i,
 * a_kj' = a_kj if its sign is opposite to a_kk's, else 0. Rows are truncated
 * to the `maxel` largest |w| (ties: smaller column) and rescaled to keep the
 * row sum. C points interpolate by injection. Parity: pinned (1D Poisson
 * weights 1/2, constant reproduction on zero-row-sum rows). */
static int amg_interp(const csr_t* A, const unsigned char* strong, const int* cf,
                      const int* cidx, int nc, int maxel, csr_t* P) {
  int n = A->n;
  int* rowlen = (int*)calloc((size_t)n + 1, sizeof(int));
  int maxrow = 1;
  if (!rowlen) return OR_ERR_MEM;
  for (int i = 0; i < n; ++i) if (A->rp[i + 1] - A->rp[i] > maxrow) maxrow = A->rp[i + 1] - A->rp[i];
  int* cset = (int*)malloc(sizeof(int) * (size_t)maxrow);
  double* num = (double*)malloc(sizeof(double) * (size_t)maxrow);
  int* keep = (int*)malloc(sizeof(int) * (size_t)maxrow);
  /* row results are staged per row in a growing buffer */
  int cap = n * 4 + 16, used = 0;
  int* oc = (int*)malloc(sizeof(int) * (size_t)cap);
  double* ov = (double*)malloc(sizeof(double) * (size_t)cap);
  if (!cset || !num || !keep || !oc || !ov) return OR_ERR_MEM;
  for (int i = 0; i < n; ++i) {
    if (used + maxrow + 1 > cap) {
      cap = 2 * cap + maxrow + 1;
      oc = (int*)realloc(oc, sizeof(int) * (size_t)cap);
      ov = (double*)realloc(ov, sizeof(double) * (size_t)cap);
      if (!oc || !ov) return OR_ERR_MEM;
    }
    if (cf[i]) {
      oc[used] = cidx[i]; ov[used] = 1.0; ++used;
      rowlen[i] = 1;
      continue;
    }
    int nC = 0;
    double aii = 0.0;
    for (int e = A->rp[i]; e < A->rp[i + 1]; ++e) {
      int j = A->ci[e];
      if (j == i) aii = A->v[e];
      else if (strong[e] && cf[j]) { cset[nC] = j; num[nC] = A->v[e]; ++nC; }
    }
    if (nC == 0) { rowlen[i] = 0; continue; }
    double d = aii;
    for (int e = A->rp[i]; e < A->rp[i + 1]; ++e) {
      int j = A->ci[e];
      if (j == i) continue;
      if (strong[e] && cf[j]) continue;
      if (strong[e] && !cf[j]) {
        int k = j;
        double aik = A->v[e];
        int dk = csr_diag_pos(A, k);
        double akk = dk >= 0 ? A->v[dk] : 0.0;
        double sigma = 0.0;
        for (int f = A->rp[k]; f < A->rp[k + 1]; ++f) {
          int m = A->ci[f];
          double akm = A->v[f];
          if (m == k) continue;
          int inC = 0;
          for (int q = 0; q < nC; ++q) if (cset[q] == m) { inC = 1; break; }
          if (inC && ((akk < 0.0) ? (akm > 0.0) : (akm < 0.0))) sigma = sigma + akm;
        }
        if (sigma == 0.0) {
          d = d + aik;
        } else {
          for (int f = A->rp[k]; f < A->rp[k + 1]; ++f) {
            int m = A->ci[f];
            double akm = A->v[f];
            if (m == k) continue;
            if (!((akk < 0.0) ? (akm > 0.0) : (akm < 0.0))) continue;
            for (int q = 0; q < nC; ++q)
              if (cset[q] == m) {
                double tq = aik * akm;
                tq = tq / sigma;
                num[q] = num[q] + tq;
                break;
              }
          }
        }
      } else {
        d = d + A->v[e];   /* weak connection lumped into the diagonal */
      }
    }
    if (d == 0.0 || !isfinite(d)) { rowlen[i] = 0; continue; }
    for (int q = 0; q < nC; ++q) num[q] = -num[q] / d;
    for (int q = 0; q < nC; ++q) keep[q] = 1;
    if (maxel > 0 && nC > maxel) {
      double total = 0.0;
      for (int q = 0; q < nC; ++q) total = total + num[q];
      for (int q = 0; q < nC; ++q) keep[q] = 0;
      for (int r = 0; r < maxel; ++r) {     /* pick the largest remaining |w| */
        int best = -1;
        for (int q = 0; q < nC; ++q) {
          if (keep[q]) continue;
          if (best < 0 || fabs(num[q]) > fabs(num[best])) best = q;
        }
        keep[best] = 1;
      }
      double kept = 0.0;
      for (int q = 0; q < nC; ++q) if (keep[q]) kept = kept + num[q];
      if (kept != 0.0) {
        double sc = total / kept;
        for (int q = 0; q < nC; ++q) if (keep[q]) num[q] = num[q] * sc;
      }
    }
    int len = 0;
    for (int q = 0; q < nC; ++q)
      if (keep[q]) { oc[used + len] = cidx[cset[q]]; ov[used + len] = num[q]; ++len; }
    used += len;
    rowlen[i] = len;
  }
  if (csr_alloc(P, n, nc, used) != OR_OK) return OR_ERR_MEM;
  P->rp[0] = 0;
  for (int i = 0; i < n; ++i) P->rp[i + 1] = P->rp[i] + rowlen[i];
  memcpy(P->ci, oc, sizeof(int) * (size_t)used);
  memcpy(P->v, ov, sizeof(double) * (size_t)used);
  free(rowlen); free(cset); free(num); free(keep); free(oc); free(ov);
  return OR_OK;
}

static void level_free(level_t* L) {
  csr_free(&L->A); csr_free(&L->P); csr_free(&L->R);
  free(L->strong); free(L->cf); free(L->cidx); free(L->dinv);
  free(L->b); free(L->x); free(L->r); free(L->t1); free(L->t2);
  free(L->cstart); free(L->mcorder); free(L->dinv2);
  memset(L, 0, sizeof(*L));
}

void or_amg_free(amg_t* h) {
  if (!h) return;
  for (int l = 0; l < h->nlev; ++l) level_free(&h->lev[l]);
  free(h->lu); free(h->piv);
  free(h);
}

static int level_vectors(level_t* L) {
  int n = L->A.n > 0 ? L->A.n : 1;
  L->b = (double*)calloc((size_t)n, sizeof(double));
  L->x = (double*)calloc((size_t)n, sizeof(double));
  L->r = (double*)calloc((size_t)n, sizeof(double));
  L->t1 = (double*)calloc((size_t)n, sizeof(double));
  L->t2 = (double*)calloc((size_t)n, sizeof(double));
  L->dinv = (double*)calloc((size_t)n, sizeof(double));
  if (!L->b || !L->x || !L->r || !L->t1 || !L->t2 || !L->dinv) return OR_ERR_MEM;
  for (int i = 0; i < L->A.n; ++i) {
    int d = csr_diag_pos(&L->A, i);
    if (d < 0 || L->A.v[d] == 0.0) return OR_ERR_SINGULAR;
    L->dinv[i] = 1.0 / L->A.v[d];
  }
  return OR_OK;
}

/* Upper bound of the spectrum of D^{-1} A for the Chebyshev interval: the
 * Gershgorin bound max_i sum_j |a_ij| / |a_ii| (row entries summed in
 * ascending column order). Reading: a power iteration started from the ones
 * vector barely sees the oscillatory modes of a Laplacian and underestimates
 * the top of the spectrum, which makes the Chebyshev smoother diverge. */
static double spectrum_bound(level_t* L) {
  double lam = 0.0;
  for (int i = 0; i < L->A.n; ++i) {
    double s = 0.0;
    for (int e = L->A.rp[i]; e < L->A.rp[i + 1]; ++e) s = s + fabs(L->A.v[e]);
    s = s * fabs(L->dinv[i]);
    if (s > lam) lam = s;
  }
  return lam;
}

static int jp_colour(int n, const int* rp, const int* ci, uint64_t seed, int* colour,
                     int* ncol_out);

/* Colour-major order of a level's points for multicolour Gauss-Seidel: the
 * Jones-Plassmann colouring of A's graph (the same routine and priorities as
 * the point-multicolour ILU order), points ascending inside each colour. */
static int level_colours(level_t* L, uint64_t seed) {
  int n = L->A.n;
  int* col = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  if (!col) return OR_ERR_MEM;
  int ncol = 0, st = jp_colour(n, L->A.rp, L->A.ci, seed, col, &ncol);
  if (st != OR_OK) { free(col); return st; }
  L->ncolour = ncol;
  L->cstart = (int*)calloc((size_t)ncol + 1, sizeof(int));
  L->mcorder = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  if (!L->cstart || !L->mcorder) { free(col); return OR_ERR_MEM; }
  for (int i = 0; i < n; ++i) L->cstart[col[i] + 1] += 1;
  for (int c = 0; c < ncol; ++c) L->cstart[c + 1] += L->cstart[c];
  int* fill = (int*)malloc(sizeof(int) * (size_t)(ncol > 0 ? ncol : 1));
  if (!fill) { free(col); return OR_ERR_MEM; }
  for (int c = 0; c < ncol; ++c) fill[c] = L->cstart[c];
  for (int i = 0; i < n; ++i) L->mcorder[fill[col[i]]++] = i;
  free(fill);
  free(col);
  return OR_OK;
}

/* Build the hierarchy for a scalar CSR matrix (copied). With `frozen` (a
 * hierarchy of an earlier matrix with the same pattern; NULL otherwise) every
 * level that frozen coarsened keeps frozen's C/F split instead of running
 * PMIS: strength, interpolation and the Galerkin products are recomputed from
 * the new values (Newton-loop reuse, reading of Sec. 2.5). */
static int amg_build(int n, const int* rp, const int* ci, const double* v, const or_opts* o,
                     const amg_t* frozen, amg_t** out) {
  amg_t* h = (amg_t*)calloc(1, sizeof(amg_t));
  if (!h) return OR_ERR_MEM;
  h->o = *o;
  int st = OR_OK;
  level_t* L = &h->lev[0];
  if (csr_alloc(&L->A, n, n, rp[n]) != OR_OK) { free(h); return OR_ERR_MEM; }
  memcpy(L->A.rp, rp, sizeof(int) * ((size_t)n + 1));
  memcpy(L->A.ci, ci, sizeof(int) * (size_t)rp[n]);
  memcpy(L->A.v, v, sizeof(double) * (size_t)rp[n]);
  h->nlev = 1;
  for (int l = 0;; ++l) {
    L = &h->lev[l];
    if ((st = level_vectors(L)) != OR_OK) goto fail;
    if (o->smoother == 1) L->lam_max = spectrum_bound(L);
    if (o->smoother == 3 && (st = level_colours(L, o->seed)) != OR_OK) goto fail;
    if (L->A.n <= o->max_coarse || l + 1 >= o->max_levels || l + 1 >= OR_MAXLEV) break;
    L->strong = (unsigned char*)malloc((size_t)(L->A.nnz > 0 ? L->A.nnz : 1));
    L->cf = (int*)malloc(sizeof(int) * (size_t)L->A.n);
    L->cidx = (int*)malloc(sizeof(int) * (size_t)L->A.n);
    if (!L->strong || !L->cf || !L->cidx) { st = OR_ERR_MEM; goto fail; }
    amg_strength(&L->A, o->theta, L->strong);
    if (frozen && l < frozen->nlev && frozen->lev[l].cf && frozen->lev[l].A.n == L->A.n)
      memcpy(L->cf, frozen->lev[l].cf, sizeof(int) * (size_t)L->A.n);
    else if ((st = amg_pmis(&L->A, L->strong, o->seed, l, L->cf, NULL, NULL)) != OR_OK)
      goto fail;
    int nc = 0;
    for (int i = 0; i < L->A.n; ++i) L->cidx[i] = L->cf[i] ? nc++ : -1;
    L->nc = nc;
    if (nc == 0 || nc == L->A.n) {   /* coarsening stalled: this is the coarsest level */
      free(L->strong); free(L->cf); free(L->cidx);
      L->strong = NULL; L->cf = NULL; L->cidx = NULL; L->nc = 0;
      break;
    }
    if ((st = amg_interp(&L->A, L->strong, L->cf, L->cidx, nc, o->interp_max, &L->P)) != OR_OK)
      goto fail;
    if ((st = csr_transpose(&L->P, &L->R)) != OR_OK) goto fail;
    csr_t AP;
    if ((st = csr_matmul(&L->A, &L->P, &AP)) != OR_OK) goto fail;
    if ((st = csr_matmul(&L->R, &AP, &h->lev[l + 1].A)) != OR_OK) goto fail;
    csr_free(&AP);
    h->nlev = l + 2;
  }
  {
    level_t* C = &h->lev[h->nlev - 1];
    int nc = C->A.n;
    if (nc > OR_MAX_DENSE) { st = OR_ERR_AMG; goto fail; }
    h->lu = (double*)calloc((size_t)nc * nc + 1, sizeof(double));
    h->piv = (int*)malloc(sizeof(int) * (size_t)(nc + 1));
    if (!h->lu || !h->piv) { st = OR_ERR_MEM; goto fail; }
    for (int i = 0; i < nc; ++i)
      for (int e = C->A.rp[i]; e < C->A.rp[i + 1]; ++e)
        h->lu[(size_t)i * nc + C->A.ci[e]] = C->A.v[e];
    if ((st = lu_factor(nc, h->lu, h->piv)) != OR_OK) goto fail;
  }
  *out = h;
  return OR_OK;
fail:
  or_amg_free(h);
  return st;
}

/* ------------------------------------------------------------------------ */
/* system AMG for the 2 x 2 block B_ee of CPTR (Sec. 4.2, Eq. CPTRM1)         */
/* ------------------------------------------------------------------------ */
/* The paper names system AMG (SAMG, BoomerAMG) for B_ee without fixing one.
 * Reading: nodal coarsening with unknown-wise interpolation. A level is a
 * matrix of 2 x 2 blocks on a point graph (unknowns [P, T] of a point
 * interleaved in the scalar form). Per level:
 *   - norm matrix: |B_ij|_F off the diagonal with a negative sign, |B_ii|_F
 *     on it (Frobenius norms summed in the order b00, b01, b10, b11);
 *   - strength on it (the scalar rule) and PMIS -> one C/F split of points;
 *   - for each unknown k, classical interpolation of the scalar matrix of
 *     the (k, k) entries with its own strength and the common split;
 *   - P interleaved: P[2i+k][2J+k] = w^k_iJ (no cross-unknown weights);
 *   - A_c = P^T A P on the scalar interleaved form (coupled P-T entries
 *     kept), read back as 2 x 2 blocks on the union of each point's columns
 *     (absent entries zero).
 * The smoother is damped 2 x 2 block Jacobi, the coarsest level a dense
 * solve. Parity: pinned (2 x 2 block-diagonal systems reduce to two
 * decoupled scalar hierarchies; Galerkin products against dense P^T A P). */
static int bcsr2_to_scalar(int np, const int* rp, const int* ci, const double* bv, csr_t* S) {
  if (csr_alloc(S, 2 * np, 2 * np, 4 * rp[np]) != OR_OK) return OR_ERR_MEM;
  int q = 0;
  S->rp[0] = 0;
  for (int i = 0; i < np; ++i)
    for (int k = 0; k < 2; ++k) {
      for (int e = rp[i]; e < rp[i + 1]; ++e)
        for (int l = 0; l < 2; ++l) {
          S->ci[q] = 2 * ci[e] + l;
          S->v[q] = bv[(size_t)4 * e + 2 * k + l];
          ++q;
        }
      S->rp[2 * i + k + 1] = q;
    }
  return OR_OK;
}

/* 2 x 2 blocks of a scalar interleaved matrix: block row I holds every point
 * J with an entry in row 2I or 2I+1; absent entries are zero. */
static int scalar_to_bcsr2(const csr_t* S, int** rp_out, int** ci_out, double** bv_out) {
  int np = S->n / 2;
  int* rp = (int*)malloc(sizeof(int) * ((size_t)np + 1));
  if (!rp) return OR_ERR_MEM;
  rp[0] = 0;
  for (int pass = 0; pass < 2; ++pass) {
    int* ci = pass ? *ci_out : NULL;
    double* bv = pass ? *bv_out : NULL;
    for (int I = 0; I < np; ++I) {
      int a = S->rp[2 * I], ae = S->rp[2 * I + 1];
      int b = S->rp[2 * I + 1], be = S->rp[2 * I + 2];
      int q = pass ? rp[I] : 0, last = -1;
      while (a < ae || b < be) {
        int ja = a < ae ? S->ci[a] / 2 : 0x7fffffff;
        int jb = b < be ? S->ci[b] / 2 : 0x7fffffff;
        int j = ja < jb ? ja : jb;
        if (j != last) {
          if (pass) {
            ci[q] = j;
            for (int t = 0; t < 4; ++t) bv[(size_t)4 * q + t] = 0.0;
          }
          ++q;
          last = j;
        }
        if (ja == j) {
          if (pass) bv[(size_t)4 * (q - 1) + (S->ci[a] & 1)] = S->v[a];
          ++a;
        } else {
          if (pass) bv[(size_t)4 * (q - 1) + 2 + (S->ci[b] & 1)] = S->v[b];
          ++b;
        }
      }
      if (!pass) rp[I + 1] = rp[I] + q;
    }
    if (!pass) {
      *ci_out = (int*)malloc(sizeof(int) * (size_t)(rp[np] > 0 ? rp[np] : 1));
      *bv_out = (double*)malloc(sizeof(double) * 4 * (size_t)(rp[np] > 0 ? rp[np] : 1));
      if (!*ci_out || !*bv_out) return OR_ERR_MEM;
    }
  }
  *rp_out = rp;
  return OR_OK;
}

static int amg_build_system(int np0, const int* rp0, const int* ci0, const double* bv0,
                            const or_opts* o, amg_t** out) {
  amg_t* h = (amg_t*)calloc(1, sizeof(amg_t));
  if (!h) return OR_ERR_MEM;
  h->o = *o;
  h->bs = 2;
  int st = OR_OK, np = np0;
  int* brp = (int*)malloc(sizeof(int) * ((size_t)np + 1));
  int* bci = (int*)malloc(sizeof(int) * (size_t)(rp0[np] > 0 ? rp0[np] : 1));
  double* bv = (double*)malloc(sizeof(double) * 4 * (size_t)(rp0[np] > 0 ? rp0[np] : 1));
  int *cfp = NULL, *cidx = NULL;
  unsigned char *sn = NULL, *sk = NULL;
  csr_t Nm = {0}, Ak = {0}, Pk[2] = {{0}, {0}};
  if (!brp || !bci || !bv) { st = OR_ERR_MEM; goto fail; }
  memcpy(brp, rp0, sizeof(int) * ((size_t)np + 1));
  memcpy(bci, ci0, sizeof(int) * (size_t)rp0[np]);
  memcpy(bv, bv0, sizeof(double) * 4 * (size_t)rp0[np]);
  h->nlev = 1;
  for (int l = 0;; ++l) {
    level_t* L = &h->lev[l];
    int nnzb = brp[np];
    if ((st = bcsr2_to_scalar(np, brp, bci, bv, &L->A)) != OR_OK) goto fail;
    if ((st = level_vectors(L)) != OR_OK) goto fail;
    L->dinv2 = (double*)malloc(sizeof(double) * 4 * (size_t)(np > 0 ? np : 1));
    if (!L->dinv2) { st = OR_ERR_MEM; goto fail; }
    for (int i = 0; i < np; ++i)
      for (int e = brp[i]; e < brp[i + 1]; ++e)
        if (bci[e] == i && (st = gj_inverse_nopiv(2, &bv[(size_t)4 * e], &L->dinv2[(size_t)4 * i])) != OR_OK)
          goto fail;
    if (np <= o->max_coarse || l + 1 >= o->max_levels || l + 1 >= OR_MAXLEV) break;
    /* norm matrix, strength, PMIS on points */
    if (csr_alloc(&Nm, np, np, nnzb) != OR_OK) { st = OR_ERR_MEM; goto fail; }
    memcpy(Nm.rp, brp, sizeof(int) * ((size_t)np + 1));
    memcpy(Nm.ci, bci, sizeof(int) * (size_t)nnzb);
    for (int i = 0; i < np; ++i)
      for (int e = brp[i]; e < brp[i + 1]; ++e) {
        const double* q = &bv[(size_t)4 * e];
        double f = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        Nm.v[e] = bci[e] == i ? f : -f;
      }
    sn = (unsigned char*)malloc((size_t)(nnzb > 0 ? nnzb : 1));
    sk = (unsigned char*)malloc((size_t)(nnzb > 0 ? nnzb : 1));
    cfp = (int*)malloc(sizeof(int) * (size_t)(np > 0 ? np : 1));
    cidx = (int*)malloc(sizeof(int) * (size_t)(np > 0 ? np : 1));
    if (!sn || !sk || !cfp || !cidx) { st = OR_ERR_MEM; goto fail; }
    amg_strength(&Nm, o->theta, sn);
    if ((st = amg_pmis(&Nm, sn, o->seed, l, cfp, NULL, NULL)) != OR_OK) goto fail;
    int ncp = 0;
    for (int i = 0; i < np; ++i) cidx[i] = cfp[i] ? ncp++ : -1;
    if (ncp == 0 || ncp == np) break;   /* coarsening stalled: the coarsest level */
    /* unknown-wise classical interpolation on the common split */
    for (int k = 0; k < 2; ++k) {
      if (csr_alloc(&Ak, np, np, nnzb) != OR_OK) { st = OR_ERR_MEM; goto fail; }
      memcpy(Ak.rp, brp, sizeof(int) * ((size_t)np + 1));
      memcpy(Ak.ci, bci, sizeof(int) * (size_t)nnzb);
      for (int e = 0; e < nnzb; ++e) Ak.v[e] = bv[(size_t)4 * e + 3 * k];
      amg_strength(&Ak, o->theta, sk);
      if ((st = amg_interp(&Ak, sk, cfp, cidx, ncp, o->interp_max, &Pk[k])) != OR_OK) goto fail;
      csr_free(&Ak);
    }
    /* interleaved P, the split per unknown, and the Galerkin product */
    if (csr_alloc(&L->P, 2 * np, 2 * ncp, Pk[0].nnz + Pk[1].nnz) != OR_OK) { st = OR_ERR_MEM; goto fail; }
    L->cf = (int*)malloc(sizeof(int) * (size_t)2 * np);
    L->cidx = (int*)malloc(sizeof(int) * (size_t)2 * np);
    if (!L->cf || !L->cidx) { st = OR_ERR_MEM; goto fail; }
    {
      int q = 0;
      L->P.rp[0] = 0;
      for (int i = 0; i < np; ++i)
        for (int k = 0; k < 2; ++k) {
          for (int e = Pk[k].rp[i]; e < Pk[k].rp[i + 1]; ++e) {
            L->P.ci[q] = 2 * Pk[k].ci[e] + k;
            L->P.v[q] = Pk[k].v[e];
            ++q;
          }
          L->P.rp[2 * i + k + 1] = q;
          L->cf[2 * i + k] = cfp[i];
          L->cidx[2 * i + k] = cfp[i] ? 2 * cidx[i] + k : -1;
        }
    }
    L->nc = 2 * ncp;
    csr_free(&Pk[0]); csr_free(&Pk[1]); csr_free(&Nm);
    free(sn); free(sk); free(cfp); free(cidx);
    sn = sk = NULL; cfp = cidx = NULL;
    if ((st = csr_transpose(&L->P, &L->R)) != OR_OK) goto fail;
    csr_t AP, Ac;
    if ((st = csr_matmul(&L->A, &L->P, &AP)) != OR_OK) goto fail;
    if ((st = csr_matmul(&L->R, &AP, &Ac)) != OR_OK) goto fail;
    csr_free(&AP);
    free(brp); free(bci); free(bv);
    brp = NULL; bci = NULL; bv = NULL;
    st = scalar_to_bcsr2(&Ac, &brp, &bci, &bv);
    csr_free(&Ac);
    if (st != OR_OK) goto fail;
    np = ncp;
    h->nlev = l + 2;
  }
  {
    level_t* C = &h->lev[h->nlev - 1];
    int nc = C->A.n;
    if (nc > OR_MAX_DENSE) { st = OR_ERR_AMG; goto fail; }
    h->lu = (double*)calloc((size_t)nc * nc + 1, sizeof(double));
    h->piv = (int*)malloc(sizeof(int) * (size_t)(nc + 1));
    if (!h->lu || !h->piv) { st = OR_ERR_MEM; goto fail; }
    for (int i = 0; i < nc; ++i)
      for (int e = C->A.rp[i]; e < C->A.rp[i + 1]; ++e)
        h->lu[(size_t)i * nc + C->A.ci[e]] = C->A.v[e];
    if ((st = lu_factor(nc, h->lu, h->piv)) != OR_OK) goto fail;
  }
  free(brp); free(bci); free(bv); free(sn); free(sk); free(cfp); free(cidx);
  csr_free(&Nm); csr_free(&Pk[0]); csr_free(&Pk[1]);
  *out = h;
  return OR_OK;
fail:
  free(brp); free(bci); free(bv); free(sn); free(sk); free(cfp); free(cidx);
  csr_free(&Nm); csr_free(&Ak); csr_free(&Pk[0]); csr_free(&Pk[1]);
  or_amg_free(h);
  return st;
}

/* ------------------------------------------------------------------------ */
/* V-cycle (Sec. 5.1: one V-cycle, direct coarse solve)                      */
/* ------------------------------------------------------------------------ */
static void residual(const level_t* L, const double* b, const double* x, double* r) {
  csr_mv(&L->A, x, r);
  for (int i = 0; i < L->A.n; ++i) r[i] = b[i] - r[i];
}

static void smooth_jacobi(level_t* L, const double* b, double* x, double omega) {
  residual(L, b, x, L->r);
  for (int i = 0; i < L->A.n; ++i) x[i] = x[i] + omega * (L->dinv[i] * L->r[i]);
}

/* Chebyshev semi-iteration for D^{-1} A on [lam/ratio, factor*lam], lam the
 * Gershgorin bound
 * (Saad, Iterative Methods for Sparse Linear Systems, Alg. 12.1). */
static void smooth_cheb(level_t* L, const double* b, double* x, const or_opts* o) {
  int n = L->A.n;
  double hi = o->cheb_hi_factor * L->lam_max, lo = L->lam_max / o->cheb_lo_ratio;
  double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo);
  double sigma = theta / delta, rho = 1.0 / sigma;
  double* d = L->t1;
  residual(L, b, x, L->r);
  for (int i = 0; i < n; ++i) d[i] = (L->dinv[i] * L->r[i]) / theta;
  for (int k = 1; k <= o->cheb_degree; ++k) {
    for (int i = 0; i < n; ++i) x[i] = x[i] + d[i];
    if (k == o->cheb_degree) break;
    residual(L, b, x, L->r);
    double rn = 1.0 / (2.0 * sigma - rho);
    for (int i = 0; i < n; ++i)
      d[i] = (rn * rho) * d[i] + (2.0 * rn / delta) * (L->dinv[i] * L->r[i]);
    rho = rn;
  }
}

/* symmetric Gauss-Seidel: forward then backward lexicographic sweep */
static void smooth_sgs(level_t* L, const double* b, double* x) {
  const csr_t* A = &L->A;
  for (int pass = 0; pass < 2; ++pass)
    for (int q = 0; q < A->n; ++q) {
      int i = pass == 0 ? q : A->n - 1 - q;
      double s = b[i];
      for (int e = A->rp[i]; e < A->rp[i + 1]; ++e)
        if (A->ci[e] != i) s -= A->v[e] * x[A->ci[e]];
      x[i] = s * L->dinv[i];
    }
}

/* multicolour symmetric Gauss-Seidel: the colours in order, then in reverse.
 * Points of one colour are not coupled, so each colour's updates read only
 * other colours' values and may run in any order (or all at once). */
static void smooth_mcsgs(level_t* L, const double* b, double* x) {
  const csr_t* A = &L->A;
  for (int pass = 0; pass < 2; ++pass)
    for (int k = 0; k < L->ncolour; ++k) {
      int c = pass == 0 ? k : L->ncolour - 1 - k;
      for (int q = L->cstart[c]; q < L->cstart[c + 1]; ++q) {
        int i = L->mcorder[q];
        double s = b[i];
        for (int e = A->rp[i]; e < A->rp[i + 1]; ++e)
          if (A->ci[e] != i) s -= A->v[e] * x[A->ci[e]];
        x[i] = s * L->dinv[i];
      }
    }
}

/* damped block Jacobi for the system AMG: x_i <- x_i + omega D_i^{-1} r_i
 * with D_i the 2 x 2 diagonal block of point i (unknowns 2i, 2i+1) */
static void smooth_bjac2(level_t* L, const double* b, double* x, double omega) {
  residual(L, b, x, L->r);
  for (int i = 0; i < L->A.n / 2; ++i) {
    const double* d = &L->dinv2[(size_t)4 * i];
    double r0 = L->r[2 * i], r1 = L->r[2 * i + 1];
    x[2 * i] = x[2 * i] + omega * (d[0] * r0 + d[1] * r1);
    x[2 * i + 1] = x[2 * i + 1] + omega * (d[2] * r0 + d[3] * r1);
  }
}

static void smooth(amg_t* h, level_t* L, const double* b, double* x, int nu) {
  for (int k = 0; k < nu; ++k) {
    if (h->bs == 2) smooth_bjac2(L, b, x, h->o.omega);
    else if (h->o.smoother == 1) smooth_cheb(L, b, x, &h->o);
    else if (h->o.smoother == 2) smooth_sgs(L, b, x);
    else if (h->o.smoother == 3) smooth_mcsgs(L, b, x);
    else smooth_jacobi(L, b, x, h->o.omega);
  }
}

static void vcycle(amg_t* h, int l, const double* b, double* x) {
  level_t* L = &h->lev[l];
  int n = L->A.n;
  if (l == h->nlev - 1) {
    memcpy(x, b, sizeof(double) * (size_t)n);
    lu_solve(n, h->lu, h->piv, x);
    return;
  }
  for (int i = 0; i < n; ++i) x[i] = 0.0;
  smooth(h, L, b, x, h->o.nu_pre);
  residual(L, b, x, L->r);
  level_t* C = &h->lev[l + 1];
  csr_mv(&L->R, L->r, C->b);
  vcycle(h, l + 1, C->b, C->x);
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int e = L->P.rp[i]; e < L->P.rp[i + 1]; ++e) s += L->P.v[e] * C->x[L->P.ci[e]];
    x[i] = x[i] + s;
  }
  smooth(h, L, b, x, h->o.nu_post);
}

/* ------------------------------------------------------------------------ */
/* multicolour ordering and block ILU(0) (Eq. CPTR3M3 / CPR second stage)    */
/* ------------------------------------------------------------------------ */
/* Jones-Plassmann colouring with SplitMix64 priorities (key 0xFFFF<<32 | i):
 * per synchronous round every uncoloured cell whose (priority, index) beats
 * all uncoloured neighbours takes the smallest colour unused by its coloured
 * neighbours. The block pattern must be structurally symmetric.
 * Parity: index work, compared bit-exactly; pinned by the proper-colouring
 * invariant. */
static int jp_colour(int n, const int* rp, const int* ci, uint64_t seed, int* colour,
                     int* ncol_out) {
  uint64_t* pr = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1));
  int* pick = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  if (!pr || !pick) { free(pr); free(pick); return OR_ERR_MEM; }
  for (int i = 0; i < n; ++i) {
    pr[i] = or_splitmix(seed, (0xFFFFULL << 32) | (uint64_t)(unsigned)i);
    colour[i] = -1;
  }
  int left = n, ncol = 0;
  while (left > 0) {
    for (int i = 0; i < n; ++i) {
      pick[i] = 0;
      if (colour[i] >= 0) continue;
      int best = 1;
      for (int e = rp[i]; e < rp[i + 1] && best; ++e) {
        int j = ci[e];
        if (j == i || colour[j] >= 0) continue;
        if (pr[j] > pr[i] || (pr[j] == pr[i] && j > i)) best = 0;
      }
      pick[i] = best;
    }
    for (int i = 0; i < n; ++i) {
      if (!pick[i]) continue;
      int c = 0;
      for (;;) {
        int used = 0;
        for (int e = rp[i]; e < rp[i + 1]; ++e)
          if (ci[e] != i && colour[ci[e]] == c) { used = 1; break; }
        if (!used) break;
        ++c;
      }
      pick[i] = -(c + 1);          /* stage the colour; applied below */
    }
    for (int i = 0; i < n; ++i)
      if (pick[i] < 0) {
        colour[i] = -pick[i] - 1;
        if (colour[i] + 1 > ncol) ncol = colour[i] + 1;
        --left;
      }
  }
  *ncol_out = ncol;
  free(pr); free(pick);
  return OR_OK;
}

typedef struct {
  int n, nb, nnzb, ncol;
  int* perm;    /* perm[k] = cell at position k */
  int* iperm;   /* iperm[cell] = position */
  int* colour;
  int* rp;      /* pattern of the permuted matrix, columns are positions */
  int* ci;
  int* dpos;
  double* v;    /* strictly lower blocks: L (unit diagonal implied); rest: U */
} bilu_t;

static void bilu_free(bilu_t* f) {
  if (!f) return;
  free(f->perm); free(f->iperm); free(f->colour); free(f->rp); free(f->ci); free(f->dpos);
  free(f->v);
  free(f);
}

/* First-fit strip colouring (the default strip order, a reading: the paper
 * does not fix the block ILU(0) ordering): cells are grouped into strips of
 * `strip` consecutive indices; in strip order, each strip takes the
 * smallest colour that none of its lower-index adjacent strips has (strips
 * a != b adjacent when a block couples a cell of a to a cell of b). Always a
 * proper colouring; on a structured grid's strip graph (bipartite) it needs
 * two colours. */
static int strip_colour_firstfit(int n, const int* rp, const int* ci, int strip, int* colour,
                                 int* ncol_out) {
  if (strip < 1) return OR_ERR_ARG;
  int ns = (n + strip - 1) / strip, ncol = 0;
  int* sc = (int*)malloc(sizeof(int) * (size_t)(ns > 0 ? ns : 1));
  if (!sc) return OR_ERR_MEM;
  for (int a = 0; a < ns; ++a) {
    int lo = a * strip, hi = lo + strip < n ? lo + strip : n;
    for (int c = 0;; ++c) {
      int used = 0;
      for (int i = lo; i < hi && !used; ++i)
        for (int e = rp[i]; e < rp[i + 1]; ++e) {
          int b = ci[e] / strip;
          if (b < a && sc[b] == c) { used = 1; break; }
        }
      if (!used) {
        sc[a] = c;
        if (c + 1 > ncol) ncol = c + 1;
        break;
      }
    }
  }
  for (int i = 0; i < n; ++i) colour[i] = sc[i / strip];
  *ncol_out = ncol;
  free(sc);
  return OR_OK;
}

/* Jones-Plassmann strip colouring: cells are grouped into strips of `strip`
 * consecutive indices, and the strips are coloured by Jones-Plassmann on the
 * strip graph (strips a != b adjacent when a block couples a cell of a to a cell
 * of b), with SplitMix64 priorities (key 0xFFFE<<32 | strip): per
 * synchronous round every uncoloured strip whose (priority, index) beats all
 * uncoloured adjacent strips takes the smallest colour unused by its
 * coloured adjacent strips. A cell takes its strip's colour; with the
 * colour-major order below each strip keeps its natural order. */
static int strip_colour(int n, const int* rp, const int* ci, int strip, uint64_t seed,
                        int* colour, int* ncol_out) {
  if (strip < 1) return OR_ERR_ARG;
  int ns = (n + strip - 1) / strip, ncol = 0;
  int* sc = (int*)malloc(sizeof(int) * (size_t)(ns > 0 ? ns : 1));
  int* pick = (int*)malloc(sizeof(int) * (size_t)(ns > 0 ? ns : 1));
  uint64_t* pr = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(ns > 0 ? ns : 1));
  if (!sc || !pick || !pr) return OR_ERR_MEM;
  for (int a = 0; a < ns; ++a) {
    sc[a] = -1;
    pr[a] = or_splitmix(seed, (0xFFFEULL << 32) | (uint64_t)(unsigned)a);
  }
  int left = ns;
  while (left > 0) {
    for (int a = 0; a < ns; ++a) {
      pick[a] = -1;
      if (sc[a] >= 0) continue;
      int lo = a * strip, hi = lo + strip < n ? lo + strip : n, best = 1;
      for (int i = lo; i < hi && best; ++i)
        for (int e = rp[i]; e < rp[i + 1] && best; ++e) {
          int b = ci[e] / strip;
          if (b == a || sc[b] >= 0) continue;
          if (pr[b] > pr[a] || (pr[b] == pr[a] && b > a)) best = 0;
        }
      if (!best) continue;
      for (int c = 0;; ++c) {
        int used = 0;
        for (int i = lo; i < hi && !used; ++i)
          for (int e = rp[i]; e < rp[i + 1]; ++e) {
            int b = ci[e] / strip;
            if (b != a && sc[b] == c) { used = 1; break; }
          }
        if (!used) { pick[a] = c; break; }
      }
    }
    for (int a = 0; a < ns; ++a)
      if (pick[a] >= 0) {
        sc[a] = pick[a];
        if (pick[a] + 1 > ncol) ncol = pick[a] + 1;
        --left;
      }
  }
  for (int i = 0; i < n; ++i) colour[i] = sc[i / strip];
  *ncol_out = ncol;
  free(sc); free(pick); free(pr);
  return OR_OK;
}

/* Block ILU(0) of P Abar P^T, P the ordering permutation (natural, or
 * colour-major with cells ascending within a colour), by the row-wise IKJ
 * elimination restricted to the block pattern, without pivoting.
 * Parity: pinned (exact on block-tridiagonal 1D systems in natural order,
 * L U reproduces the matrix on the pattern). */
static int bilu_factor(int n, int nb, const int* rp, const int* ci, const double* v, int order,
                       int strip, uint64_t seed, bilu_t** out) {
  int nb2 = nb * nb;
  bilu_t* f = (bilu_t*)calloc(1, sizeof(bilu_t));
  if (!f) return OR_ERR_MEM;
  f->n = n; f->nb = nb; f->nnzb = rp[n];
  f->perm = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  f->iperm = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  f->colour = (int*)calloc((size_t)(n > 0 ? n : 1), sizeof(int));
  f->rp = (int*)malloc(sizeof(int) * ((size_t)n + 1));
  f->ci = (int*)malloc(sizeof(int) * (size_t)(rp[n] > 0 ? rp[n] : 1));
  f->dpos = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  f->v = (double*)malloc(sizeof(double) * (size_t)(rp[n] > 0 ? rp[n] : 1) * nb2);
  if (!f->perm || !f->iperm || !f->colour || !f->rp || !f->ci || !f->dpos || !f->v) {
    bilu_free(f);
    return OR_ERR_MEM;
  }
  int st;
  if (order == 0) {
    if ((st = jp_colour(n, rp, ci, seed, f->colour, &f->ncol)) != OR_OK) { bilu_free(f); return st; }
  } else if (order == 2) {
    if ((st = strip_colour_firstfit(n, rp, ci, strip, f->colour, &f->ncol)) != OR_OK) { bilu_free(f); return st; }
  } else if (order == 3) {
    if ((st = strip_colour(n, rp, ci, strip, seed, f->colour, &f->ncol)) != OR_OK) { bilu_free(f); return st; }
  } else {
    f->ncol = n > 0 ? 1 : 0;
  }
  /* colour-major, ascending cell index within a colour */
  int k = 0;
  for (int c = 0; c < (order != 1 ? f->ncol : 1); ++c)
    for (int i = 0; i < n; ++i)
      if (order == 1 || f->colour[i] == c) f->perm[k++] = i;
  for (int q = 0; q < n; ++q) f->iperm[f->perm[q]] = q;
  /* permuted pattern with ascending position columns */
  f->rp[0] = 0;
  for (int q = 0; q < n; ++q) {
    int i = f->perm[q];
    int len = rp[i + 1] - rp[i], base = f->rp[q];
    for (int a = 0; a < len; ++a) {
      int e = rp[i] + a;
      int pc = f->iperm[ci[e]];
      int b = a - 1;
      while (b >= 0 && f->ci[base + b] > pc) {
        f->ci[base + b + 1] = f->ci[base + b];
        memcpy(&f->v[(size_t)(base + b + 1) * nb2], &f->v[(size_t)(base + b) * nb2],
               sizeof(double) * nb2);
        --b;
      }
      f->ci[base + b + 1] = pc;
      memcpy(&f->v[(size_t)(base + b + 1) * nb2], &v[(size_t)e * nb2], sizeof(double) * nb2);
    }
    f->rp[q + 1] = base + len;
    f->dpos[q] = -1;
    for (int e = base; e < base + len; ++e) if (f->ci[e] == q) f->dpos[q] = e;
    if (f->dpos[q] < 0) { bilu_free(f); return OR_ERR_ARG; }
  }
  /* IKJ block ILU(0) */
  double inv[32 * 32], L[32 * 32];
  for (int i = 0; i < n; ++i) {
    for (int e = f->rp[i]; e < f->rp[i + 1]; ++e) {
      int kk = f->ci[e];
      if (kk >= i) break;
      if ((st = gj_inverse_nopiv(nb, &f->v[(size_t)f->dpos[kk] * nb2], inv)) != OR_OK) {
        bilu_free(f);
        return st;
      }
      /* L_ik = W_ik U_kk^{-1} */
      const double* Wik = &f->v[(size_t)e * nb2];
      for (int r = 0; r < nb; ++r)
        for (int c = 0; c < nb; ++c) {
          double s = 0.0;
          for (int q = 0; q < nb; ++q) s += Wik[r * nb + q] * inv[q * nb + c];
          L[r * nb + c] = s;
        }
      memcpy(&f->v[(size_t)e * nb2], L, sizeof(double) * nb2);
      /* W_ij -= L_ik U_kj for j > k in row k that are in row i */
      for (int g = f->dpos[kk] + 1; g < f->rp[kk + 1]; ++g) {
        int j = f->ci[g];
        int hit = -1;
        for (int e2 = f->rp[i]; e2 < f->rp[i + 1]; ++e2) if (f->ci[e2] == j) { hit = e2; break; }
        if (hit < 0) continue;
        double* Wij = &f->v[(size_t)hit * nb2];
        const double* Ukj = &f->v[(size_t)g * nb2];
        for (int r = 0; r < nb; ++r)
          for (int c = 0; c < nb; ++c) {
            double s = 0.0;
            for (int q = 0; q < nb; ++q) s += L[r * nb + q] * Ukj[q * nb + c];
            Wij[r * nb + c] -= s;
          }
      }
    }
    if ((st = gj_inverse_nopiv(nb, &f->v[(size_t)f->dpos[i] * nb2], inv)) != OR_OK) {
      bilu_free(f);
      return st;
    }
  }
  *out = f;
  return OR_OK;
}

/* y = (L U)^{-1} u, vectors in original cell order */
static int bilu_solve(const bilu_t* f, const double* u, double* y, double* work) {
  int n = f->n, nb = f->nb, nb2 = nb * nb;
  /* forward in permuted order: w_q = u_perm[q] - sum_{k<q} L_qk w_k */
  for (int q = 0; q < n; ++q) {
    double* wq = &work[(size_t)q * nb];
    memcpy(wq, &u[(size_t)f->perm[q] * nb], sizeof(double) * nb);
    for (int e = f->rp[q]; e < f->dpos[q]; ++e) {
      const double* Lb = &f->v[(size_t)e * nb2];
      const double* wk = &work[(size_t)f->ci[e] * nb];
      for (int r = 0; r < nb; ++r) {
        double s = 0.0;
        for (int c = 0; c < nb; ++c) s += Lb[r * nb + c] * wk[c];
        wq[r] -= s;
      }
    }
  }
  /* backward: x_q = U_qq^{-1} (w_q - sum_{j>q} U_qj x_j) */
  for (int q = n - 1; q >= 0; --q) {
    double* wq = &work[(size_t)q * nb];
    for (int e = f->dpos[q] + 1; e < f->rp[q + 1]; ++e) {
      const double* Ub = &f->v[(size_t)e * nb2];
      const double* xj = &work[(size_t)f->ci[e] * nb];
      for (int r = 0; r < nb; ++r) {
        double s = 0.0;
        for (int c = 0; c < nb; ++c) s += Ub[r * nb + c] * xj[c];
        wq[r] -= s;
      }
    }
    int st = ge_solve_nopiv(nb, &f->v[(size_t)f->dpos[q] * nb2], wq);
    if (st) return st;
  }
  for (int q = 0; q < n; ++q) memcpy(&y[(size_t)f->perm[q] * nb], &work[(size_t)q * nb], sizeof(double) * nb);
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* solver: scaling, stages, Algorithms 1/2, FGMRES                           */
/* ------------------------------------------------------------------------ */
typedef struct {
  int N, nb, p, t, nnzb;
  int *rp, *ci, *dblk;
  double* A;      /* original values (copied) */
  double* Abar;   /* scaled values */
  double* W;      /* per-cell scaling matrices */
  or_opts o;
  amg_t *amgT, *amgP;
  double *luT, *luP; int *pivT, *pivP;   /* exact sub-solvers */
  bilu_t* ilu;
  double *sr, *sy;       /* scalar work vectors */
  double *z, *u, *tmp, *work;
} or_solver;

void or_free(or_solver* s) {
  if (!s) return;
  free(s->rp); free(s->ci); free(s->dblk); free(s->A); free(s->Abar); free(s->W);
  or_amg_free(s->amgT); or_amg_free(s->amgP);
  free(s->luT); free(s->luP); free(s->pivT); free(s->pivP);
  bilu_free(s->ilu);
  free(s->sr); free(s->sy); free(s->z); free(s->u); free(s->tmp); free(s->work);
  free(s);
}

static void bsr_mv(const or_solver* s, const double* vals, const double* x, double* y) {
  int nb = s->nb, nb2 = nb * nb;
  for (int i = 0; i < s->N; ++i) {
    for (int r = 0; r < nb; ++r) {
      double acc = 0.0;
      for (int e = s->rp[i]; e < s->rp[i + 1]; ++e) {
        const double* blk = &vals[(size_t)e * nb2];
        const double* xj = &x[(size_t)s->ci[e] * nb];
        for (int c = 0; c < nb; ++c) acc += blk[r * nb + c] * xj[c];
      }
      y[(size_t)i * nb + r] = acc;
    }
  }
}

static int dense_subsystem(const or_solver* s, int var, double** lu, int** piv) {
  int N = s->N, nb2 = s->nb * s->nb;
  if (N > OR_MAX_DENSE) return OR_ERR_ARG;
  *lu = (double*)calloc((size_t)N * N, sizeof(double));
  *piv = (int*)malloc(sizeof(int) * (size_t)N);
  if (!*lu || !*piv) return OR_ERR_MEM;
  for (int i = 0; i < N; ++i)
    for (int e = s->rp[i]; e < s->rp[i + 1]; ++e)
      (*lu)[(size_t)i * N + s->ci[e]] = s->Abar[(size_t)e * nb2 + var * s->nb + var];
  return lu_factor(N, *lu, *piv);
}

static int build_amg_for(or_solver* s, int var, const amg_t* frozen, amg_t** out) {
  int N = s->N, nb2 = s->nb * s->nb;
  double* v = (double*)malloc(sizeof(double) * (size_t)(s->nnzb > 0 ? s->nnzb : 1));
  if (!v) return OR_ERR_MEM;
  /* scalar subsystem: (var, var) entry of every scaled block (B_PP, C_TT) */
  for (int e = 0; e < s->nnzb; ++e) v[e] = s->Abar[(size_t)e * nb2 + var * s->nb + var];
  int st = amg_build(N, s->rp, s->ci, v, &s->o, frozen, out);
  free(v);
  return st;
}

/* Set-up: scaling (Eqs. CPR / CPTR31 / CPTR32), subsystem extraction (B_PP
 * Eq. CPR and CPTR31, C_TT Eq. CPTR32), AMG or exact sub-solvers, and the
 * last stage (block ILU(0) of the scaled matrix, Eq. CPTR3M3). */
static or_solver* setup_impl(int N, int nb, const int* rp, const int* ci, const double* vals,
                             int p, int t, const or_opts* o, const amg_t* frozT,
                             const amg_t* frozP, int* status) {
  int st = OR_OK;
  *status = OR_OK;
  if (N < 0 || nb < 2 || nb > 32 || p < 0 || p >= nb || t < 0 || t >= nb || p == t) {
    *status = OR_ERR_ARG;
    return NULL;
  }
  or_solver* s = (or_solver*)calloc(1, sizeof(or_solver));
  if (!s) { *status = OR_ERR_MEM; return NULL; }
  int nb2 = nb * nb, nnzb = rp[N];
  s->N = N; s->nb = nb; s->p = p; s->t = t; s->nnzb = nnzb; s->o = *o;
  s->rp = (int*)malloc(sizeof(int) * ((size_t)N + 1));
  s->ci = (int*)malloc(sizeof(int) * (size_t)(nnzb > 0 ? nnzb : 1));
  s->dblk = (int*)malloc(sizeof(int) * (size_t)(N > 0 ? N : 1));
  s->A = (double*)malloc(sizeof(double) * (size_t)(nnzb > 0 ? nnzb : 1) * nb2);
  s->Abar = (double*)malloc(sizeof(double) * (size_t)(nnzb > 0 ? nnzb : 1) * nb2);
  s->W = (double*)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1) * nb2);
  s->sr = (double*)calloc((size_t)(N > 0 ? N : 1), sizeof(double));
  s->sy = (double*)calloc((size_t)(N > 0 ? N : 1), sizeof(double));
  s->z = (double*)calloc((size_t)(N > 0 ? N : 1) * nb, sizeof(double));
  s->u = (double*)calloc((size_t)(N > 0 ? N : 1) * nb, sizeof(double));
  s->tmp = (double*)calloc((size_t)(N > 0 ? N : 1) * nb, sizeof(double));
  s->work = (double*)calloc((size_t)(N > 0 ? N : 1) * nb, sizeof(double));
  if (!s->rp || !s->ci || !s->dblk || !s->A || !s->Abar || !s->W || !s->sr || !s->sy || !s->z ||
      !s->u || !s->tmp || !s->work) {
    st = OR_ERR_MEM;
    goto fail;
  }
  memcpy(s->rp, rp, sizeof(int) * ((size_t)N + 1));
  memcpy(s->ci, ci, sizeof(int) * (size_t)nnzb);
  memcpy(s->A, vals, sizeof(double) * (size_t)nnzb * nb2);
  /* validate the pattern: ascending columns in range, diagonal present,
   * structurally symmetric */
  for (int i = 0; i < N; ++i) {
    s->dblk[i] = -1;
    if (rp[i + 1] < rp[i]) { st = OR_ERR_ARG; goto fail; }
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
      if (ci[e] < 0 || ci[e] >= N || (e > rp[i] && ci[e] <= ci[e - 1])) { st = OR_ERR_ARG; goto fail; }
      if (ci[e] == i) s->dblk[i] = e;
      int j = ci[e], found = 0;
      for (int f = rp[j]; f < rp[j + 1]; ++f) if (ci[f] == i) { found = 1; break; }
      if (!found) { st = OR_ERR_ARG; goto fail; }
    }
    if (s->dblk[i] < 0) { st = OR_ERR_ARG; goto fail; }
  }
  /* left scaling: W_i from the diagonal block, Abar_ij = W_i A_ij */
  for (int i = 0; i < N; ++i) {
    double* Wi = &s->W[(size_t)i * nb2];
    if ((st = build_scaling(nb, p, t, o->scheme, &vals[(size_t)s->dblk[i] * nb2], Wi)) != OR_OK)
      goto fail;
    for (int e = rp[i]; e < rp[i + 1]; ++e)
      block_left_mul(nb, Wi, &vals[(size_t)e * nb2], &s->Abar[(size_t)e * nb2]);
  }
  if (o->scheme == 3) {
    /* B_ee = Abar[e, e], e = (P, T): one 2 x 2 block per block of Abar */
    double* be = (double*)malloc(sizeof(double) * 4 * (size_t)(nnzb > 0 ? nnzb : 1));
    if (!be) { st = OR_ERR_MEM; goto fail; }
    int ev[2] = {p, t};
    for (int e = 0; e < nnzb; ++e)
      for (int k = 0; k < 2; ++k)
        for (int l = 0; l < 2; ++l)
          be[(size_t)4 * e + 2 * k + l] = s->Abar[(size_t)e * nb2 + ev[k] * nb + ev[l]];
    if (o->exact_sub) {
      /* M_ee = B_ee^{-1} by dense LU (the paper's direct sub-solver study) */
      csr_t S;
      st = bcsr2_to_scalar(N, rp, ci, be, &S);
      if (st == OR_OK && 2 * N > OR_MAX_DENSE) st = OR_ERR_ARG;
      if (st == OR_OK) {
        s->luP = (double*)calloc((size_t)4 * N * N, sizeof(double));
        s->pivP = (int*)malloc(sizeof(int) * (size_t)(2 * N > 0 ? 2 * N : 1));
        if (!s->luP || !s->pivP) st = OR_ERR_MEM;
      }
      if (st == OR_OK) {
        for (int i = 0; i < 2 * N; ++i)
          for (int e = S.rp[i]; e < S.rp[i + 1]; ++e) s->luP[(size_t)i * 2 * N + S.ci[e]] = S.v[e];
        st = lu_factor(2 * N, s->luP, s->pivP);
      }
      csr_free(&S);
    } else {
      st = amg_build_system(N, rp, ci, be, o, &s->amgP);
    }
    free(be);
    if (st != OR_OK) goto fail;
  }
  if (o->scheme == 0 || o->scheme == 1) {
    if (o->exact_sub) {
      if ((st = dense_subsystem(s, p, &s->luP, &s->pivP)) != OR_OK) goto fail;
      if (o->scheme == 0 && (st = dense_subsystem(s, t, &s->luT, &s->pivT)) != OR_OK) goto fail;
    } else {
      if ((st = build_amg_for(s, p, frozP, &s->amgP)) != OR_OK) goto fail;
      if (o->scheme == 0 && (st = build_amg_for(s, t, frozT, &s->amgT)) != OR_OK) goto fail;
    }
  }
  if (o->stage3 == 0) {
    if ((st = bilu_factor(N, nb, rp, ci, s->Abar, o->ilu_order, o->ilu_strip, o->seed, &s->ilu)) != OR_OK)
      goto fail;
  } else {
    for (int i = 0; i < N; ++i) {   /* block Jacobi: only check invertibility */
      double inv[32 * 32];
      if ((st = gj_inverse_nopiv(nb, &s->Abar[(size_t)s->dblk[i] * nb2], inv)) != OR_OK) goto fail;
    }
  }
  return s;
fail:
  *status = st;
  or_free(s);
  return NULL;
}

or_solver* or_setup(int N, int nb, const int* rp, const int* ci, const double* vals, int p,
                    int t, const or_opts* o, int* status) {
  return setup_impl(N, nb, rp, ci, vals, p, t, o, NULL, NULL, status);
}

/* The set-up for new values on the pattern of `old` (Newton-loop reuse,
 * Sec. 2.5: the grid, hence the pattern, stays fixed across Newton
 * iterations and time steps). reuse = 0: everything is recomputed, exactly
 * as or_setup does (the ordering depends on the pattern only); reuse = 1:
 * the AMG levels keep old's C/F splits. */
or_solver* or_update(const or_solver* old, const double* vals, int reuse, int* status) {
  if (!old || (reuse != 0 && reuse != 1)) {
    *status = OR_ERR_ARG;
    return NULL;
  }
  return setup_impl(old->N, old->nb, old->rp, old->ci, vals, old->p, old->t, &old->o,
                    reuse ? old->amgT : NULL, reuse ? old->amgP : NULL, status);
}

/* scalar sub-solver on unknown `var`: y_var = M_var^{-1} r_var */
static void scalar_stage(or_solver* s, int var, const double* r, double* y) {
  int N = s->N, nb = s->nb;
  for (int i = 0; i < N; ++i) s->sr[i] = r[(size_t)i * nb + var];
  if (s->o.exact_sub) {
    memcpy(s->sy, s->sr, sizeof(double) * (size_t)N);
    if (var == s->p) lu_solve(N, s->luP, s->pivP, s->sy);
    else lu_solve(N, s->luT, s->pivT, s->sy);
  } else {
    amg_t* h = var == s->p ? s->amgP : s->amgT;
    vcycle(h, 0, s->sr, s->sy);
  }
  for (int i = 0; i < N; ++i)
    for (int k = 0; k < nb; ++k) y[(size_t)i * nb + k] = k == var ? s->sy[i] : 0.0;
}

/* CPTR first stage (Eq. CPTRM1): y_e = M_ee^{-1} r_e on e = (P, T), zero
 * elsewhere; M_ee is the system AMG V-cycle (or the dense solve). */
static int system_stage(or_solver* s, const double* r, double* y) {
  int N = s->N, nb = s->nb;
  double* b2 = (double*)malloc(sizeof(double) * 2 * (size_t)(N > 0 ? N : 1));
  double* x2 = (double*)malloc(sizeof(double) * 2 * (size_t)(N > 0 ? N : 1));
  if (!b2 || !x2) { free(b2); free(x2); return OR_ERR_MEM; }
  for (int i = 0; i < N; ++i) {
    b2[2 * i] = r[(size_t)i * nb + s->p];
    b2[2 * i + 1] = r[(size_t)i * nb + s->t];
  }
  if (s->o.exact_sub) {
    memcpy(x2, b2, sizeof(double) * 2 * (size_t)N);
    lu_solve(2 * N, s->luP, s->pivP, x2);
  } else {
    vcycle(s->amgP, 0, b2, x2);
  }
  for (int i = 0; i < N; ++i)
    for (int k = 0; k < nb; ++k)
      y[(size_t)i * nb + k] = k == s->p ? x2[2 * i] : (k == s->t ? x2[2 * i + 1] : 0.0);
  free(b2); free(x2);
  return OR_OK;
}

static int last_stage(or_solver* s, const double* u, double* y) {
  int nb = s->nb, nb2 = nb * nb;
  if (s->o.stage3 == 0) return bilu_solve(s->ilu, u, y, s->work);
  for (int i = 0; i < s->N; ++i) {
    memcpy(&y[(size_t)i * nb], &u[(size_t)i * nb], sizeof(double) * nb);
    int st = ge_solve_nopiv(nb, &s->Abar[(size_t)s->dblk[i] * nb2], &y[(size_t)i * nb]);
    if (st) return st;
  }
  return OR_OK;
}

/* which: 0 = T stage (M_TT), 1 = P stage (M_PP), 2 = last stage (M_3 / M_2) */
int or_stage(or_solver* s, int which, const double* r, double* y) {
  if (which == 0) {
    if (s->o.scheme != 0) return OR_ERR_ARG;
    scalar_stage(s, s->t, r, y);
    return OR_OK;
  }
  if (which == 1) {
    if (s->o.scheme == 2) return OR_ERR_ARG;
    if (s->o.scheme == 3) return system_stage(s, r, y);
    scalar_stage(s, s->p, r, y);
    return OR_OK;
  }
  return last_stage(s, r, y);
}

/* y = M^{-1} r on the scaled system.
 * CPTR3 (Algorithm 2): x = M1 r; z = r - Abar x; v = M2 z; u = z - Abar v;
 *                      y = x + v + M3 u, with M1 = amg(C_TT) on T and
 *                      M2 = amg(B_PP) on P (swapped by stage_order = 1).
 * CPR (Algorithm 1):   x = M1 r; z = r - Abar x; y = x + M2 z, M1 = amg(B_PP).
 * CPTR (Sec. 4.2):     the same two stages with M1 = system AMG of B_ee on
 *                      (P, T) (Eq. CPTRM1) and M2 = ilu(Abar).
 * ILU only:            y = M r. */
int or_apply(or_solver* s, const double* r, double* y) {
  int n = s->N * s->nb;
  double* x = s->tmp;
  int st;
  if (s->o.scheme == 2) return last_stage(s, r, y);
  if (s->o.scheme == 1 || s->o.scheme == 3) {
    if (s->o.scheme == 1) scalar_stage(s, s->p, r, x);
    else if ((st = system_stage(s, r, x)) != OR_OK) return st;
    bsr_mv(s, s->Abar, x, s->z);
    for (int i = 0; i < n; ++i) s->z[i] = r[i] - s->z[i];
    if ((st = last_stage(s, s->z, y)) != OR_OK) return st;
    for (int i = 0; i < n; ++i) y[i] = x[i] + y[i];
    return OR_OK;
  }
  int v1 = s->o.stage_order == 0 ? s->t : s->p;
  int v2 = s->o.stage_order == 0 ? s->p : s->t;
  double* v = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  if (!v) return OR_ERR_MEM;
  scalar_stage(s, v1, r, x);                       /* x = M1 r */
  bsr_mv(s, s->Abar, x, s->z);
  for (int i = 0; i < n; ++i) s->z[i] = r[i] - s->z[i];       /* z = r - Abar x */
  scalar_stage(s, v2, s->z, v);                    /* v = M2 z */
  bsr_mv(s, s->Abar, v, s->u);
  for (int i = 0; i < n; ++i) s->u[i] = s->z[i] - s->u[i];    /* u = z - Abar v */
  st = last_stage(s, s->u, y);                     /* M3 u */
  if (st == OR_OK)
    for (int i = 0; i < n; ++i) y[i] = x[i] + v[i] + y[i];  /* y = x + v + M3 u */
  free(v);
  return st;
}

/* Right-preconditioned restarted FGMRES(m) on Abar, x0 = 0, modified
 * Gram-Schmidt, Givens rotations, stopping on the implicit residual
 * |g_{j+1}| / ||bbar|| <= tol, then checking the true residual
 * ||bbar - Abar x|| / ||bbar|| at the end of the cycle and restarting if it
 * is above tol (Sec. 5.1 uses GMRES without restart; the restart length is a
 * reading). Iterations count inner steps. Happy breakdown when
 * h_{j+1,j} <= 1e-14 ||Abar z_j||. bbar is the scaled right-hand side. */
int or_fgmres(or_solver* s, const double* bbar, double* x, double tol, int maxit, int m,
              or_result* res) {
  int n = s->N * s->nb;
  size_t nn = (size_t)(n > 0 ? n : 1);
  memset(res, 0, sizeof(*res));
  if (m < 1 || maxit < 0) return OR_ERR_ARG;
  double* V = (double*)malloc(sizeof(double) * nn * (size_t)(m + 1));
  double* Z = (double*)malloc(sizeof(double) * nn * (size_t)m);
  double* w = (double*)malloc(sizeof(double) * nn);
  double* r = (double*)malloc(sizeof(double) * nn);
  double* H = (double*)calloc((size_t)(m + 1) * m, sizeof(double));
  double* cs = (double*)calloc((size_t)m, sizeof(double));
  double* sn = (double*)calloc((size_t)m, sizeof(double));
  double* g = (double*)calloc((size_t)m + 1, sizeof(double));
  double* yv = (double*)calloc((size_t)m, sizeof(double));
  int st = OR_OK;
  if (!V || !Z || !w || !r || !H || !cs || !sn || !g || !yv) { st = OR_ERR_MEM; goto done; }
  for (int i = 0; i < n; ++i) x[i] = 0.0;
  double bnorm = nrm2(n, bbar);
  res->rel_res_true = 0.0;
  if (bnorm == 0.0) goto done;
  memcpy(r, bbar, sizeof(double) * (size_t)n);
  double beta = bnorm;
  int total = 0;
  for (;;) {
    for (int i = 0; i < n; ++i) V[i] = r[i] / beta;
    for (int i = 0; i <= m; ++i) g[i] = 0.0;
    g[0] = beta;
    int k = 0, happy = 0;
    double relres = 1.0;
    for (int j = 0; j < m; ++j) {
      if (total >= maxit) break;
      double* zj = &Z[(size_t)j * nn];
      if ((st = or_apply(s, &V[(size_t)j * nn], zj)) != OR_OK) goto done;
      bsr_mv(s, s->Abar, zj, w);
      double w0 = nrm2(n, w);
      for (int i = 0; i <= j; ++i) {
        const double* vi = &V[(size_t)i * nn];
        double h = dot(n, w, vi);
        H[(size_t)i * m + j] = h;
        for (int q = 0; q < n; ++q) w[q] -= h * vi[q];
      }
      double hn = nrm2(n, w);
      H[(size_t)(j + 1) * m + j] = hn;
      happy = (hn <= 1e-14 * w0);
      if (!happy)
        for (int q = 0; q < n; ++q) V[(size_t)(j + 1) * nn + q] = w[q] / hn;
      for (int i = 0; i < j; ++i) {
        double a = H[(size_t)i * m + j], b = H[(size_t)(i + 1) * m + j];
        H[(size_t)i * m + j] = cs[i] * a + sn[i] * b;
        H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * b;
      }
      double a = H[(size_t)j * m + j], b = H[(size_t)(j + 1) * m + j];
      double den = hypot(a, b);
      if (den == 0.0 || !isfinite(den)) { st = OR_ERR_BREAKDOWN; goto done; }
      cs[j] = a / den; sn[j] = b / den;
      H[(size_t)j * m + j] = den;
      H[(size_t)(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++total; k = j + 1;
      relres = fabs(g[j + 1]) / bnorm;
      res->rel_res_implicit = relres;
      if (relres <= tol || happy) break;
    }
    /* y = H_k^{-1} g_k; x += Z y */
    for (int i = k - 1; i >= 0; --i) {
      double sum = g[i];
      for (int q = i + 1; q < k; ++q) sum -= H[(size_t)i * m + q] * yv[q];
      yv[i] = sum / H[(size_t)i * m + i];
    }
    for (int q = 0; q < k; ++q) {
      const double* zq = &Z[(size_t)q * nn];
      for (int i = 0; i < n; ++i) x[i] += yv[q] * zq[i];
    }
    bsr_mv(s, s->Abar, x, w);
    for (int i = 0; i < n; ++i) r[i] = bbar[i] - w[i];
    beta = nrm2(n, r);
    res->rel_res_true = beta / bnorm;
    res->iters = total;
    if (!isfinite(beta)) { st = OR_ERR_BREAKDOWN; goto done; }
    if (res->rel_res_true <= tol) break;
    if (total >= maxit || k == 0) { st = OR_ERR_NOT_CONVERGED; break; }
    res->restarts++;
  }
done:
  res->status = st;
  free(V); free(Z); free(w); free(r); free(H); free(cs); free(sn); free(g); free(yv);
  return st;
}

/* ------------------------------------------------------------------------ */
/* static condensation (Sec. 3, Eqs. global and reduced)                     */
/* ------------------------------------------------------------------------ */
/* The global system [J11 J12; J21 J22] [d1; d2] = -[r1; r2] with the
 * secondary unknowns coupled only inside their cell: J12 (n1 x n2) and J22
 * (n2 x n2) are one block per cell, J11 (n1 x n1) and J21 (n2 x n1) have the
 * cell graph's block pattern (rp, ci). The reduced system A d1 = b has
 *   A = J11 - J12 J22^{-1} J21,   b = -r1 + J12 J22^{-1} r2,
 * assembled block by block: with T_i = J12_i J22_i^{-1} (cell i),
 * A_ij = J11_ij - T_i J21_ij and b_i = -r1_i + T_i r2_i. J22_i is inverted
 * without pivoting (Sec. 3 aligns the secondary equations so that its
 * diagonal is nonzero). Parity: pinned against a dense solve of the global
 * system and the dense Schur complement. */
int or_condense(int N, const int* rp, const int* ci, int n1, int n2, const double* j11,
                const double* j21, const double* j12, const double* j22, const double* r1,
                const double* r2, double* a, double* b) {
  if (N < 0 || n1 < 1 || n1 > 32 || n2 < 0 || n2 > 32) return OR_ERR_ARG;
  double inv[32 * 32], T[32 * 32];
  for (int i = 0; i < N; ++i) {
    if (n2 > 0) {
      int st = gj_inverse_nopiv(n2, &j22[(size_t)i * n2 * n2], inv);
      if (st != OR_OK) return st;
    }
    const double* J12 = &j12[(size_t)i * n1 * n2];
    for (int r = 0; r < n1; ++r)
      for (int c = 0; c < n2; ++c) {
        double s = 0.0;
        for (int k = 0; k < n2; ++k) s += J12[r * n2 + k] * inv[k * n2 + c];
        T[r * n2 + c] = s;
      }
    for (int r = 0; r < n1; ++r) {
      double s = 0.0;
      for (int k = 0; k < n2; ++k) s += T[r * n2 + k] * r2[(size_t)i * n2 + k];
      b[(size_t)i * n1 + r] = -r1[(size_t)i * n1 + r] + s;
    }
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
      const double* J11 = &j11[(size_t)e * n1 * n1];
      const double* J21 = &j21[(size_t)e * n2 * n1];
      double* A = &a[(size_t)e * n1 * n1];
      for (int r = 0; r < n1; ++r)
        for (int c = 0; c < n1; ++c) {
          double s = 0.0;
          for (int k = 0; k < n2; ++k) s += T[r * n2 + k] * J21[k * n1 + c];
          A[r * n1 + c] = J11[r * n1 + c] - s;
        }
    }
  }
  return OR_OK;
}

/* Secondary unknowns from the primary ones (the second block row of Eq.
 * global): J22_i d2_i = -r2_i - sum_j J21_ij d1_j, solved per cell by
 * Gaussian elimination without pivoting. */
int or_recover(int N, const int* rp, const int* ci, int n1, int n2, const double* j21,
               const double* j22, const double* r2, const double* d1, double* d2) {
  if (N < 0 || n1 < 1 || n1 > 32 || n2 < 0 || n2 > 32) return OR_ERR_ARG;
  for (int i = 0; i < N; ++i) {
    double* w = &d2[(size_t)i * n2];
    for (int k = 0; k < n2; ++k) {
      double s = 0.0;
      for (int e = rp[i]; e < rp[i + 1]; ++e) {
        const double* J21 = &j21[(size_t)e * n2 * n1];
        const double* x = &d1[(size_t)ci[e] * n1];
        for (int c = 0; c < n1; ++c) s += J21[k * n1 + c] * x[c];
      }
      w[k] = -r2[(size_t)i * n2 + k] - s;
    }
    if (n2 > 0) {
      int st = ge_solve_nopiv(n2, &j22[(size_t)i * n2 * n2], w);
      if (st != OR_OK) return st;
    }
  }
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* accessors for the tests                                                  */
/* ------------------------------------------------------------------------ */
void or_get_scaled(const or_solver* s, double* abar, double* W) {
  size_t nb2 = (size_t)s->nb * s->nb;
  if (abar) memcpy(abar, s->Abar, sizeof(double) * (size_t)s->nnzb * nb2);
  if (W) memcpy(W, s->W, sizeof(double) * (size_t)s->N * nb2);
}

void or_scale_rhs(const or_solver* s, const double* b, double* bbar) {
  int nb = s->nb;
  for (int i = 0; i < s->N; ++i)
    block_vec_left_mul(nb, &s->W[(size_t)i * nb * nb], &b[(size_t)i * nb], &bbar[(size_t)i * nb]);
}

void or_spmv(const or_solver* s, const double* x, double* y) { bsr_mv(s, s->Abar, x, y); }

static amg_t* pick_amg(const or_solver* s, int which) { return which == 0 ? s->amgT : s->amgP; }

int or_amg_nlevels(const or_solver* s, int which) {
  amg_t* h = pick_amg(s, which);
  return h ? h->nlev : 0;
}

/* sizes: out[0] = n, out[1] = nnz(A), out[2] = nnz(P) (0 on the coarsest) */
int or_amg_level_sizes(const or_solver* s, int which, int l, int* out) {
  amg_t* h = pick_amg(s, which);
  if (!h || l < 0 || l >= h->nlev) return OR_ERR_ARG;
  out[0] = h->lev[l].A.n; out[1] = h->lev[l].A.nnz;
  out[2] = l < h->nlev - 1 ? h->lev[l].P.nnz : 0;
  return OR_OK;
}

int or_amg_level_get(const or_solver* s, int which, int l, int* arp, int* aci, double* av,
                     int* cf, int* prp, int* pci, double* pv, double* lam_max) {
  amg_t* h = pick_amg(s, which);
  if (!h || l < 0 || l >= h->nlev) return OR_ERR_ARG;
  const level_t* L = &h->lev[l];
  memcpy(arp, L->A.rp, sizeof(int) * ((size_t)L->A.n + 1));
  memcpy(aci, L->A.ci, sizeof(int) * (size_t)L->A.nnz);
  memcpy(av, L->A.v, sizeof(double) * (size_t)L->A.nnz);
  if (lam_max) *lam_max = L->lam_max;
  if (l < h->nlev - 1) {
    memcpy(cf, L->cf, sizeof(int) * (size_t)L->A.n);
    memcpy(prp, L->P.rp, sizeof(int) * ((size_t)L->A.n + 1));
    memcpy(pci, L->P.ci, sizeof(int) * (size_t)L->P.nnz);
    memcpy(pv, L->P.v, sizeof(double) * (size_t)L->P.nnz);
  }
  return OR_OK;
}

int or_bilu_ncolours(const or_solver* s) { return s->ilu ? s->ilu->ncol : 0; }

int or_bilu_get(const or_solver* s, int* colour, int* perm, int* frp, int* fci, double* fv) {
  const bilu_t* f = s->ilu;
  if (!f) return OR_ERR_ARG;
  size_t nb2 = (size_t)f->nb * f->nb;
  if (colour) memcpy(colour, f->colour, sizeof(int) * (size_t)f->n);
  if (perm) memcpy(perm, f->perm, sizeof(int) * (size_t)f->n);
  if (frp) memcpy(frp, f->rp, sizeof(int) * ((size_t)f->n + 1));
  if (fci) memcpy(fci, f->ci, sizeof(int) * (size_t)f->nnzb);
  if (fv) memcpy(fv, f->v, sizeof(double) * (size_t)f->nnzb * nb2);
  return OR_OK;
}

/* Stand-alone AMG on a scalar CSR matrix (Poisson pins). */
amg_t* or_amg_create(int n, const int* rp, const int* ci, const double* v, const or_opts* o,
                     int* status) {
  amg_t* h = NULL;
  *status = amg_build(n, rp, ci, v, o, NULL, &h);
  return h;
}

/* Stand-alone system AMG on np points of 2 x 2 blocks (bv: 4 per block,
 * row-major); levels are read back in the scalar interleaved form. */
amg_t* or_amg_create_system(int np, const int* rp, const int* ci, const double* bv,
                            const or_opts* o, int* status) {
  amg_t* h = NULL;
  *status = amg_build_system(np, rp, ci, bv, o, &h);
  return *status == OR_OK ? h : NULL;
}

int or_amg_nlev(const amg_t* h) { return h->nlev; }

int or_amg_sizes(const amg_t* h, int l, int* out) {
  if (l < 0 || l >= h->nlev) return OR_ERR_ARG;
  out[0] = h->lev[l].A.n; out[1] = h->lev[l].A.nnz;
  out[2] = l < h->nlev - 1 ? h->lev[l].P.nnz : 0;
  return OR_OK;
}

int or_amg_get(const amg_t* h, int l, int* arp, int* aci, double* av, int* cf, int* prp,
               int* pci, double* pv) {
  if (l < 0 || l >= h->nlev) return OR_ERR_ARG;
  const level_t* L = &h->lev[l];
  memcpy(arp, L->A.rp, sizeof(int) * ((size_t)L->A.n + 1));
  memcpy(aci, L->A.ci, sizeof(int) * (size_t)L->A.nnz);
  memcpy(av, L->A.v, sizeof(double) * (size_t)L->A.nnz);
  if (l < h->nlev - 1) {
    memcpy(cf, L->cf, sizeof(int) * (size_t)L->A.n);
    memcpy(prp, L->P.rp, sizeof(int) * ((size_t)L->A.n + 1));
    memcpy(pci, L->P.ci, sizeof(int) * (size_t)L->P.nnz);
    memcpy(pv, L->P.v, sizeof(double) * (size_t)L->P.nnz);
  }
  return OR_OK;
}

void or_amg_vcycle(amg_t* h, const double* b, double* x) { vcycle(h, 0, b, x); }

/* nu applications of the configured smoother on level l, starting from the
 * caller's x (tests pin the smoothers against their error polynomials). */
int or_amg_smooth(amg_t* h, int l, const double* b, double* x, int nu) {
  if (l < 0 || l >= h->nlev || nu < 0) return OR_ERR_ARG;
  smooth(h, &h->lev[l], b, x, nu);
  return OR_OK;
}

/* Strength, PMIS and interpolation on a scalar CSR matrix with an optional
 * forced C/F split (cf_in != NULL). Fills cf_out and the P arrays (caller
 * sizes pci/pv with nnz(A) entries). Returns nnz(P) or a negative status. */
int or_interp_only(int n, const int* rp, const int* ci, const double* v, double theta,
                   int maxel, uint64_t seed, const int* cf_in, int* cf_out, int* strong_out,
                   int* prp, int* pci, double* pv) {
  csr_t A = {n, n, rp[n], (int*)rp, (int*)ci, (double*)v};
  unsigned char* strong = (unsigned char*)malloc((size_t)(rp[n] > 0 ? rp[n] : 1));
  int* cidx = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  if (!strong || !cidx) return OR_ERR_MEM;
  amg_strength(&A, theta, strong);
  if (cf_in) memcpy(cf_out, cf_in, sizeof(int) * (size_t)n);
  else {
    int st = amg_pmis(&A, strong, seed, 0, cf_out, NULL, NULL);
    if (st) return st;
  }
  int nc = 0;
  for (int i = 0; i < n; ++i) cidx[i] = cf_out[i] ? nc++ : -1;
  csr_t P;
  int st = amg_interp(&A, strong, cf_out, cidx, nc, maxel, &P);
  if (st) return st;
  for (int e = 0; e < rp[n]; ++e) strong_out[e] = strong[e];
  memcpy(prp, P.rp, sizeof(int) * ((size_t)n + 1));
  memcpy(pci, P.ci, sizeof(int) * (size_t)P.nnz);
  memcpy(pv, P.v, sizeof(double) * (size_t)P.nnz);
  int nnz = P.nnz;
  csr_free(&P);
  free(strong); free(cidx);
  return nnz;
}

/* Strength and PMIS on a scalar CSR matrix for level `level`, with the
 * rounds exposed (tests): strong_out per nonzero, pre (split before the
 * F-to-C fix-up), rnd (round of each decision), cf_out (final split). */
int or_pmis_rounds(int n, const int* rp, const int* ci, const double* v, double theta,
                   uint64_t seed, int level, int* strong_out, int* pre, int* rnd, int* cf_out) {
  csr_t A = {n, n, rp[n], (int*)rp, (int*)ci, (double*)v};
  unsigned char* strong = (unsigned char*)malloc((size_t)(rp[n] > 0 ? rp[n] : 1));
  if (!strong) return OR_ERR_MEM;
  amg_strength(&A, theta, strong);
  int st = amg_pmis(&A, strong, seed, level, cf_out, pre, rnd);
  for (int e = 0; e < rp[n]; ++e) strong_out[e] = strong[e];
  free(strong);
  return st;
}

/* Jones-Plassmann colouring on a block pattern (exported for the tests). */
int or_colour(int n, const int* rp, const int* ci, uint64_t seed, int* colour) {
  int ncol = 0;
  int st = jp_colour(n, rp, ci, seed, colour, &ncol);
  return st ? st : ncol;
}

uint64_t or_hash(uint64_t seed, uint64_t key) { return or_splitmix(seed, key); }
