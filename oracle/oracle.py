"""ctypes binding of the FP64 CPU oracle (``mss_oracle.c``).

TEST INFRASTRUCTURE: imported only by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline / reference leg of ``bench.py``. The product path never
imports it. It shares no code with the CUDA library.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np

from .build import build_oracle

OK, ERR_ARG, ERR_SINGULAR, ERR_NOT_CONVERGED, ERR_BREAKDOWN, ERR_MEM, ERR_AMG = 0, -1, -2, -3, -4, -5, -6

SCHEME = {"cptr3": 0, "cpr": 1, "ilu0": 2, "cptr": 3}
SMOOTHER = {"jacobi": 0, "chebyshev": 1, "sgs": 2, "mcsgs": 3}


class OrOpts(C.Structure):
    _fields_ = [("scheme", C.c_int), ("stage_order", C.c_int), ("exact_sub", C.c_int),
                ("stage3", C.c_int), ("ilu_order", C.c_int), ("smoother", C.c_int),
                ("nu_pre", C.c_int), ("nu_post", C.c_int), ("cheb_degree", C.c_int),
                ("max_coarse", C.c_int), ("max_levels", C.c_int), ("interp_max", C.c_int),
                ("restart", C.c_int), ("ilu_strip", C.c_int),
                ("theta", C.c_double), ("omega", C.c_double), ("cheb_lo_ratio", C.c_double),
                ("cheb_hi_factor", C.c_double), ("seed", C.c_uint64)]


class OrResult(C.Structure):
    _fields_ = [("iters", C.c_int), ("restarts", C.c_int), ("status", C.c_int),
                ("pad_", C.c_int), ("rel_res_implicit", C.c_double),
                ("rel_res_true", C.c_double)]


_lib = None

_P = C.c_void_p


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(str(build_oracle()))
        L.or_opts_default.argtypes = [C.POINTER(OrOpts)]
        L.or_setup.restype = _P
        L.or_setup.argtypes = [C.c_int, C.c_int, _P, _P, _P, C.c_int, C.c_int,
                               C.POINTER(OrOpts), C.POINTER(C.c_int)]
        L.or_free.argtypes = [_P]
        L.or_update.restype = _P
        L.or_update.argtypes = [_P, _P, C.c_int, C.POINTER(C.c_int)]
        L.or_get_scaled.argtypes = [_P, _P, _P]
        L.or_scale_rhs.argtypes = [_P, _P, _P]
        L.or_spmv.argtypes = [_P, _P, _P]
        L.or_apply.argtypes = [_P, _P, _P]
        L.or_stage.argtypes = [_P, C.c_int, _P, _P]
        L.or_fgmres.argtypes = [_P, _P, _P, C.c_double, C.c_int, C.c_int, C.POINTER(OrResult)]
        L.or_amg_nlevels.argtypes = [_P, C.c_int]
        L.or_amg_level_sizes.argtypes = [_P, C.c_int, C.c_int, _P]
        L.or_amg_level_get.argtypes = [_P, C.c_int, C.c_int, _P, _P, _P, _P, _P, _P, _P, _P]
        L.or_bilu_ncolours.argtypes = [_P]
        L.or_bilu_get.argtypes = [_P, _P, _P, _P, _P, _P]
        L.or_amg_create.restype = _P
        L.or_amg_create.argtypes = [C.c_int, _P, _P, _P, C.POINTER(OrOpts), C.POINTER(C.c_int)]
        L.or_amg_free.argtypes = [_P]
        L.or_amg_create_system.restype = _P
        L.or_amg_create_system.argtypes = [C.c_int, _P, _P, _P, C.POINTER(OrOpts),
                                           C.POINTER(C.c_int)]
        L.or_amg_nlev.argtypes = [_P]
        L.or_amg_sizes.argtypes = [_P, C.c_int, _P]
        L.or_amg_get.argtypes = [_P, C.c_int, _P, _P, _P, _P, _P, _P, _P]
        L.or_amg_vcycle.argtypes = [_P, _P, _P]
        L.or_amg_smooth.argtypes = [_P, C.c_int, _P, _P, C.c_int]
        L.or_interp_only.argtypes = [C.c_int, _P, _P, _P, C.c_double, C.c_int, C.c_uint64,
                                     _P, _P, _P, _P, _P, _P]
        L.or_colour.argtypes = [C.c_int, _P, _P, C.c_uint64, _P]
        L.or_condense.argtypes = [C.c_int, _P, _P, C.c_int, C.c_int, _P, _P, _P, _P, _P, _P,
                                  _P, _P]
        L.or_recover.argtypes = [C.c_int, _P, _P, C.c_int, C.c_int, _P, _P, _P, _P, _P]
        L.or_pmis_rounds.argtypes = [C.c_int, _P, _P, _P, C.c_double, C.c_uint64, C.c_int,
                                     _P, _P, _P, _P]
        L.or_hash.restype = C.c_uint64
        L.or_hash.argtypes = [C.c_uint64, C.c_uint64]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def options(**kw) -> OrOpts:
    """Default options (Sec. 5.1 settings and the stated readings), with
    keyword overrides; ``scheme`` and ``smoother`` accept names."""
    o = OrOpts()
    lib().or_opts_default(C.byref(o))
    for k, v in kw.items():
        if k == "scheme" and isinstance(v, str):
            v = SCHEME[v]
        if k == "smoother" and isinstance(v, str):
            v = SMOOTHER[v]
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


class OracleError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: oracle status {status}")
        self.status = status


@dataclass
class Level:
    A: tuple          # (row_ptr, col_idx, vals)
    cf: np.ndarray | None
    P: tuple | None
    lam_max: float = 0.0


class OracleSolver:
    """Set-up of the scaled system, the stage operators and the last stage."""

    def __init__(self, row_ptr, col_idx, vals, nb: int, p_idx: int = 0, t_idx: int = 1,
                 opts: OrOpts | None = None, **kw):
        self._keep = (_i32(row_ptr), _i32(col_idx), _f64(vals))
        self.N = self._keep[0].shape[0] - 1
        self.nb = nb
        self.nnzb = self._keep[1].shape[0]
        self.opts = opts if opts is not None else options(**kw)
        st = C.c_int(0)
        self._h = lib().or_setup(self.N, nb, _ptr(self._keep[0]), _ptr(self._keep[1]),
                                 _ptr(self._keep[2]), p_idx, t_idx, C.byref(self.opts),
                                 C.byref(st))
        if not self._h:
            raise OracleError(st.value, "or_setup")

    @classmethod
    def from_system(cls, sysm, **kw):
        return cls(sysm.row_ptr, sysm.col_idx, sysm.vals, sysm.nb, sysm.p_idx, sysm.t_idx, **kw)

    def updated(self, vals, reuse: int = 0) -> "OracleSolver":
        """A new solver for new block values on this solver's pattern
        (or_update): reuse = 0 recomputes everything, reuse = 1 keeps every
        AMG level's C/F split."""
        new = object.__new__(OracleSolver)
        new._keep = (self._keep[0], self._keep[1], _f64(vals))
        new.N, new.nb, new.nnzb, new.opts = self.N, self.nb, self.nnzb, self.opts
        st = C.c_int(0)
        new._h = lib().or_update(self._h, _ptr(new._keep[2]), int(reuse), C.byref(st))
        if not new._h:
            raise OracleError(st.value, "or_update")
        return new

    def __del__(self):
        if getattr(self, "_h", None):
            lib().or_free(self._h)
            self._h = None

    # -- scaling ----------------------------------------------------------
    def scaled(self):
        nb2 = self.nb * self.nb
        abar = np.empty((self.nnzb, self.nb, self.nb))
        W = np.empty((self.N, self.nb, self.nb))
        lib().or_get_scaled(self._h, _ptr(abar), _ptr(W))
        return abar, W

    def scale_rhs(self, b):
        b = _f64(b)
        out = np.empty_like(b)
        lib().or_scale_rhs(self._h, _ptr(b), _ptr(out))
        return out

    def spmv(self, x):
        x = _f64(x)
        y = np.empty_like(x)
        lib().or_spmv(self._h, _ptr(x), _ptr(y))
        return y

    # -- preconditioner -----------------------------------------------------
    def apply(self, r):
        r = _f64(r)
        y = np.empty_like(r)
        st = lib().or_apply(self._h, _ptr(r), _ptr(y))
        if st:
            raise OracleError(st, "or_apply")
        return y

    def stage(self, which: int, r):
        r = _f64(r)
        y = np.empty_like(r)
        st = lib().or_stage(self._h, which, _ptr(r), _ptr(y))
        if st:
            raise OracleError(st, "or_stage")
        return y

    def fgmres(self, bbar, tol=1e-6, maxit=500, restart=None):
        bbar = _f64(bbar)
        x = np.zeros_like(bbar)
        res = OrResult()
        m = self.opts.restart if restart is None else restart
        lib().or_fgmres(self._h, _ptr(bbar), _ptr(x), tol, maxit, m, C.byref(res))
        info = dict(iters=res.iters, restarts=res.restarts, status=res.status,
                    rel_res_implicit=res.rel_res_implicit, rel_res_true=res.rel_res_true)
        return x, info

    # -- hierarchy ----------------------------------------------------------
    def amg_levels(self, which: int):
        """which: 0 = temperature (C_TT), 1 = pressure (B_PP)."""
        L = lib()
        out = []
        nlev = L.or_amg_nlevels(self._h, which)
        for l in range(nlev):
            sz = np.zeros(3, np.int32)
            L.or_amg_level_sizes(self._h, which, l, _ptr(sz))
            n, nnz, nnzp = (int(v) for v in sz)
            arp = np.empty(n + 1, np.int32); aci = np.empty(max(nnz, 1), np.int32)
            av = np.empty(max(nnz, 1)); cf = np.empty(max(n, 1), np.int32)
            prp = np.empty(n + 1, np.int32); pci = np.empty(max(nnzp, 1), np.int32)
            pv = np.empty(max(nnzp, 1)); lam = C.c_double(0.0)
            L.or_amg_level_get(self._h, which, l, _ptr(arp), _ptr(aci), _ptr(av), _ptr(cf),
                               _ptr(prp), _ptr(pci), _ptr(pv), C.byref(lam))
            last = l == nlev - 1
            out.append(Level(A=(arp, aci[:nnz], av[:nnz]),
                             cf=None if last else cf[:n],
                             P=None if last else (prp, pci[:nnzp], pv[:nnzp]),
                             lam_max=lam.value))
        return out

    def bilu(self):
        L = lib()
        ncol = L.or_bilu_ncolours(self._h)
        colour = np.empty(self.N, np.int32); perm = np.empty(self.N, np.int32)
        frp = np.empty(self.N + 1, np.int32); fci = np.empty(self.nnzb, np.int32)
        fv = np.empty((self.nnzb, self.nb, self.nb))
        st = L.or_bilu_get(self._h, _ptr(colour), _ptr(perm), _ptr(frp), _ptr(fci), _ptr(fv))
        if st:
            raise OracleError(st, "or_bilu_get")
        return dict(ncolours=ncol, colour=colour, perm=perm, row_ptr=frp, col_idx=fci, vals=fv)


class OracleAMG:
    """Stand-alone hierarchy on a scalar CSR matrix."""

    def __init__(self, row_ptr, col_idx, vals, opts: OrOpts | None = None, **kw):
        self._keep = (_i32(row_ptr), _i32(col_idx), _f64(vals))
        self.n = self._keep[0].shape[0] - 1
        self.opts = opts if opts is not None else options(**kw)
        st = C.c_int(0)
        self._h = lib().or_amg_create(self.n, _ptr(self._keep[0]), _ptr(self._keep[1]),
                                      _ptr(self._keep[2]), C.byref(self.opts), C.byref(st))
        if not self._h:
            raise OracleError(st.value, "or_amg_create")

    @classmethod
    def system(cls, row_ptr, col_idx, blocks, opts: OrOpts | None = None, **kw):
        """System AMG (the CPTR first stage) on 2 x 2 blocks [nnzb, 2, 2];
        levels and vectors are in the scalar form with the two unknowns of a
        point interleaved."""
        new = object.__new__(cls)
        new._keep = (_i32(row_ptr), _i32(col_idx), _f64(blocks))
        new.n = 2 * (new._keep[0].shape[0] - 1)
        new.opts = opts if opts is not None else options(**kw)
        st = C.c_int(0)
        new._h = lib().or_amg_create_system(new.n // 2, _ptr(new._keep[0]), _ptr(new._keep[1]),
                                            _ptr(new._keep[2]), C.byref(new.opts), C.byref(st))
        if not new._h:
            raise OracleError(st.value, "or_amg_create_system")
        return new

    def __del__(self):
        if getattr(self, "_h", None):
            lib().or_amg_free(self._h)
            self._h = None

    def nlev(self):
        return lib().or_amg_nlev(self._h)

    def levels(self):
        L = lib()
        out = []
        for l in range(self.nlev()):
            sz = np.zeros(3, np.int32)
            L.or_amg_sizes(self._h, l, _ptr(sz))
            n, nnz, nnzp = (int(v) for v in sz)
            arp = np.empty(n + 1, np.int32); aci = np.empty(max(nnz, 1), np.int32)
            av = np.empty(max(nnz, 1)); cf = np.empty(max(n, 1), np.int32)
            prp = np.empty(n + 1, np.int32); pci = np.empty(max(nnzp, 1), np.int32)
            pv = np.empty(max(nnzp, 1))
            L.or_amg_get(self._h, l, _ptr(arp), _ptr(aci), _ptr(av), _ptr(cf), _ptr(prp),
                         _ptr(pci), _ptr(pv))
            last = l == self.nlev() - 1
            out.append(Level(A=(arp, aci[:nnz], av[:nnz]), cf=None if last else cf[:n],
                             P=None if last else (prp, pci[:nnzp], pv[:nnzp])))
        return out

    def vcycle(self, b):
        b = _f64(b)
        x = np.zeros_like(b)
        lib().or_amg_vcycle(self._h, _ptr(b), _ptr(x))
        return x

    def smooth(self, b, x0, nu=1, level=0):
        """nu applications of the configured smoother on one level from x0."""
        b = _f64(b)
        x = _f64(x0).copy()
        st = lib().or_amg_smooth(self._h, level, _ptr(b), _ptr(x), nu)
        if st != 0:
            raise OracleError(st, "or_amg_smooth")
        return x


def interp_only(row_ptr, col_idx, vals, theta=0.25, maxel=4, seed=0x5eed, cf=None):
    """Strength + (PMIS or the given C/F split) + interpolation on one level.
    Returns (cf, strong mask, P=(rp, ci, v))."""
    rp, ci, v = _i32(row_ptr), _i32(col_idx), _f64(vals)
    n = rp.shape[0] - 1
    nnz = ci.shape[0]
    cf_out = np.empty(n, np.int32)
    strong = np.empty(nnz, np.int32)
    prp = np.empty(n + 1, np.int32)
    pci = np.empty(max(nnz, 1), np.int32)
    pv = np.empty(max(nnz, 1))
    cf_in = None if cf is None else _i32(cf)
    st = lib().or_interp_only(n, _ptr(rp), _ptr(ci), _ptr(v), theta, maxel, seed,
                              None if cf_in is None else _ptr(cf_in), _ptr(cf_out),
                              _ptr(strong), _ptr(prp), _ptr(pci), _ptr(pv))
    if st < 0:
        raise OracleError(st, "or_interp_only")
    return cf_out, strong.astype(bool), (prp, pci[:st], pv[:st])


def pmis_rounds(row_ptr, col_idx, vals, theta=0.25, seed=0x5eed, level=0):
    """Strength and PMIS with the rounds exposed: (strong mask, split before
    the F-to-C fix-up, round of each decision, final split)."""
    rp, ci, v = _i32(row_ptr), _i32(col_idx), _f64(vals)
    n = rp.shape[0] - 1
    strong = np.empty(max(ci.shape[0], 1), np.int32)
    pre, rnd, cf = (np.empty(max(n, 1), np.int32) for _ in range(3))
    st = lib().or_pmis_rounds(n, _ptr(rp), _ptr(ci), _ptr(v), theta, seed, level, _ptr(strong),
                              _ptr(pre), _ptr(rnd), _ptr(cf))
    if st:
        raise OracleError(st, "or_pmis_rounds")
    return strong[:ci.shape[0]].astype(bool), pre[:n], rnd[:n], cf[:n]


def condense(full):
    """Static condensation (Sec. 3, Eq. reduced) of a synthetic.FullSystem:
    (A blocks [nnzb, n1, n1], b [N * n1])."""
    rp, ci = _i32(full.row_ptr), _i32(full.col_idx)
    j11, j21, j12, j22 = (_f64(x) for x in (full.j11, full.j21, full.j12, full.j22))
    r1, r2 = _f64(full.r1), _f64(full.r2)
    a = np.empty((full.nnzb, full.n1, full.n1))
    b = np.empty(full.n_cells * full.n1)
    st = lib().or_condense(full.n_cells, _ptr(rp), _ptr(ci), full.n1, full.n2, _ptr(j11),
                           _ptr(j21), _ptr(j12), _ptr(j22), _ptr(r1), _ptr(r2), _ptr(a), _ptr(b))
    if st:
        raise OracleError(st, "or_condense")
    return a, b


def recover(full, d1):
    """The secondary unknowns d2 from the primary ones d1 (Eq. global)."""
    rp, ci = _i32(full.row_ptr), _i32(full.col_idx)
    j21, j22, r2, x1 = (_f64(x) for x in (full.j21, full.j22, full.r2, d1))
    d2 = np.empty(full.n_cells * full.n2)
    st = lib().or_recover(full.n_cells, _ptr(rp), _ptr(ci), full.n1, full.n2, _ptr(j21),
                          _ptr(j22), _ptr(r2), _ptr(x1), _ptr(d2))
    if st:
        raise OracleError(st, "or_recover")
    return d2


def colour(row_ptr, col_idx, seed=0x5eed):
    rp, ci = _i32(row_ptr), _i32(col_idx)
    n = rp.shape[0] - 1
    out = np.empty(n, np.int32)
    nc = lib().or_colour(n, _ptr(rp), _ptr(ci), seed, _ptr(out))
    if nc < 0:
        raise OracleError(nc, "or_colour")
    return out, nc


def splitmix(seed: int, key: int) -> int:
    return int(lib().or_hash(seed, key))
