"""Thin ctypes binding of libmss.so (the C-ABI in include/mss.h).

Argument marshalling only: every step of the set-up and the solve runs in the
CUDA library. PyTorch provides device memory (its caching allocator, through
the allocation hooks) and the stream. A missing library raises; there is no
CPU or PyTorch fallback.
"""
from __future__ import annotations

import ctypes as C
import sys
from pathlib import Path

import numpy as np

LIB_PATH = Path(__file__).resolve().parent / "libmss.so"

OK = 0
ERR_INVALID_ARG, ERR_SINGULAR_BLOCK, ERR_NOT_CONVERGED, ERR_BREAKDOWN = -1, -2, -3, -4
ERR_CUDA, ERR_OOM, ERR_AMG, ERR_NOT_SETUP = -5, -6, -7, -8

SCHEMES = {"cptr3": 0, "cpr": 1, "ilu0": 2, "cptr": 3}
SMOOTHERS = {"jacobi": 0, "chebyshev": 1, "mcsgs": 3}
PRECISIONS = {"fp64": 0, "mixed": 1}
DRIVERS = {"host": 0, "graph": 1}
FACTOR_FORMS = {"auto": 0, "warp": 1, "lanes": 2}

# every exported symbol declared in include/mss.h
EXPORTS = ["mss_options_default", "mss_create", "mss_destroy", "mss_setup", "mss_update_values", "mss_scale_rhs",
           "mss_spmv", "mss_apply", "mss_stage_apply", "mss_fgmres_solve", "mss_solve_host",
           "mss_residual_norm", "mss_residual_norm_noalloc", "mss_condense", "mss_recover", "mss_get_scaled", "mss_amg_num_levels", "mss_amg_level_sizes", "mss_amg_level_copy",
           "mss_bilu_num_colours", "mss_bilu_ordering", "mss_bilu_factors", "mss_probe_wait_limit", "mss_kernel_launches",
           "mss_trace_enable", "mss_trace_read", "mss_status_string", "mss_last_error",
           "mss_batch_create", "mss_batch_destroy", "mss_batch_set_schedule", "mss_batch_solve",
           "mss_batch_tuned",
           "mss_batch_last_error", "mss_gnn_num_params", "mss_gnn_create", "mss_gnn_destroy",
           "mss_gnn_info", "mss_gnn_set_vectors", "mss_gnn_weights", "mss_gnn_loss_grad",
           "mss_gnn_adam", "mss_gnn_last_error"]

TRACE_KINDS = {"spmv": 0, "bilu_fwd": 1, "bilu_bwd": 2, "vcycle": 3, "ortho": 4,
               "setup_scale": 5, "setup_amg": 6, "setup_bilu": 7, "apply": 8,
               "condense": 9, "recover": 10}


class Options(C.Structure):
    _fields_ = [("scheme", C.c_int32), ("stage_order", C.c_int32), ("stage3", C.c_int32),
                ("ilu_order", C.c_int32), ("smoother", C.c_int32), ("nu_pre", C.c_int32),
                ("nu_post", C.c_int32), ("cheb_degree", C.c_int32),
                ("amg_max_coarse", C.c_int32), ("amg_max_levels", C.c_int32),
                ("interp_max_elems", C.c_int32), ("restart", C.c_int32),
                ("precision", C.c_int32), ("ilu_strip", C.c_int32),
                ("orthog", C.c_int32), ("driver", C.c_int32), ("factor_form", C.c_int32),
                ("amg_theta", C.c_double), ("jacobi_omega", C.c_double),
                ("cheb_lo_ratio", C.c_double), ("cheb_hi_factor", C.c_double),
                ("seed", C.c_uint64), ("learned_interp", C.c_void_p)]


class Result(C.Structure):
    _fields_ = [("iters", C.c_int32), ("restarts", C.c_int32), ("status", C.c_int32),
                ("pad_", C.c_int32), ("rel_res_implicit", C.c_double),
                ("rel_res_true", C.c_double), ("setup_ms", C.c_double),
                ("solve_ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad_"}


class Bsr(C.Structure):
    _fields_ = [("n_rows", C.c_int32), ("nnzb", C.c_int32), ("row_ptr", C.c_void_p),
                ("col_idx", C.c_void_p), ("vals", C.c_void_p)]


class Full(C.Structure):
    _fields_ = [("n_rows", C.c_int32), ("nnzb", C.c_int32), ("row_ptr", C.c_void_p),
                ("col_idx", C.c_void_p), ("n1", C.c_int32), ("n2", C.c_int32),
                ("j11", C.c_void_p), ("j21", C.c_void_p), ("j12", C.c_void_p),
                ("j22", C.c_void_p)]


class Layout(C.Structure):
    _fields_ = [("p_idx", C.c_int32), ("t_idx", C.c_int32), ("col_major_blocks", C.c_int32)]


class System(C.Structure):
    _fields_ = [("J", Bsr), ("nb", C.c_int32), ("layout", Layout), ("b", C.c_void_p),
                ("x", C.c_void_p)]


class BatchInfo(C.Structure):
    _fields_ = [("bucket", C.c_int32), ("threads", C.c_int32), ("driver", C.c_int32),
                ("lane", C.c_int32), ("latency_ms", C.c_double), ("finish_ms", C.c_double),
                ("schedule", C.c_int32), ("group", C.c_int32), ("tile_blocks", C.c_int32),
                ("per_sm", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)

_lib = None


def load(path: Path | str | None = None):
    """Load libmss.so (raises if it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = Path(path) if path else LIB_PATH
    if not p.exists():
        raise RuntimeError(f"{p} is missing: build it with paper_1912_04385_gb300.build.build()")
    L = C.CDLL(str(p))
    P = C.c_void_p
    L.mss_options_default.argtypes = [C.POINTER(Options)]
    L.mss_create.argtypes = [C.POINTER(P), P, ALLOC_FN, FREE_FN, P]
    L.mss_destroy.argtypes = [P]
    L.mss_destroy.restype = None
    L.mss_setup.argtypes = [P, C.POINTER(Bsr), C.c_int, Layout, C.POINTER(Options)]
    L.mss_update_values.argtypes = [P, C.POINTER(Bsr), C.c_int]
    L.mss_scale_rhs.argtypes = [P, P, P]
    L.mss_spmv.argtypes = [P, P, P]
    L.mss_apply.argtypes = [P, P, P]
    L.mss_stage_apply.argtypes = [P, C.c_int, P, P]
    L.mss_fgmres_solve.argtypes = [P, C.POINTER(Bsr), P, P, C.c_double, C.c_int,
                                   C.POINTER(Result)]
    L.mss_solve_host.argtypes = [P, C.POINTER(Bsr), C.c_int, Layout, C.POINTER(Options), P, P,
                                 C.c_double, C.c_int, C.POINTER(Result)]
    L.mss_residual_norm.argtypes = [P, C.POINTER(Bsr), C.c_int, P, P, P]
    L.mss_condense.argtypes = [P, C.POINTER(Full), P, P, P, P]
    L.mss_recover.argtypes = [P, C.POINTER(Full), P, P, P]
    L.mss_residual_norm_noalloc.argtypes = [P, C.POINTER(Bsr), C.c_int, P, P, P]
    L.mss_get_scaled.argtypes = [P, P]
    L.mss_amg_num_levels.argtypes = [P, C.c_int]
    L.mss_amg_level_sizes.argtypes = [P, C.c_int, C.c_int, P]
    L.mss_amg_level_copy.argtypes = [P, C.c_int, C.c_int, P, P, P, P, P, P, P]
    L.mss_bilu_num_colours.argtypes = [P, P]
    L.mss_bilu_ordering.argtypes = [P, P, P]
    L.mss_bilu_factors.argtypes = [P, P, P]
    L.mss_probe_wait_limit.argtypes = [C.c_void_p, C.POINTER(C.c_int32)]
    L.mss_kernel_launches.restype = C.c_longlong
    L.mss_kernel_launches.argtypes = [C.c_int]
    L.mss_trace_enable.argtypes = [P, C.c_int]
    L.mss_trace_read.argtypes = [P, C.c_int, P, P, C.c_int]
    L.mss_status_string.restype = C.c_char_p
    L.mss_status_string.argtypes = [C.c_int]
    L.mss_last_error.restype = C.c_char_p
    L.mss_last_error.argtypes = [P]
    L.mss_batch_create.argtypes = [C.POINTER(P), C.c_int, C.c_int]
    L.mss_batch_destroy.argtypes = [P]
    L.mss_batch_destroy.restype = None
    L.mss_batch_solve.argtypes = [P, C.c_int, C.POINTER(System), C.POINTER(Options), C.c_double,
                                  C.c_int, C.POINTER(Result), C.POINTER(BatchInfo)]
    L.mss_batch_set_schedule.argtypes = [P, C.c_int]
    L.mss_batch_tuned.argtypes = [P, C.c_int, P]
    L.mss_batch_last_error.restype = C.c_char_p
    L.mss_batch_last_error.argtypes = [P]
    L.mss_gnn_num_params.argtypes = []
    L.mss_gnn_create.argtypes = [P, C.POINTER(P)]
    L.mss_gnn_destroy.argtypes = [P]
    L.mss_gnn_destroy.restype = None
    L.mss_gnn_info.argtypes = [P, P, P, P]
    L.mss_gnn_set_vectors.argtypes = [P, C.c_int, P, C.c_int, C.c_double, C.c_int]
    L.mss_gnn_weights.argtypes = [P, P, P]
    L.mss_gnn_loss_grad.argtypes = [P, P, P, P]
    L.mss_gnn_adam.argtypes = [P, P, P, P, P, C.c_int, C.c_float, C.c_float, C.c_float,
                               C.c_float]
    L.mss_gnn_last_error.restype = C.c_char_p
    L.mss_gnn_last_error.argtypes = [P]
    if path is None:
        _lib = L
    return L


class MssError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(msg)
        self.status = status


def options(**kw) -> Options:
    """Library defaults with keyword overrides (scheme, smoother, precision and
    driver accept names)."""
    o = Options()
    load().mss_options_default(C.byref(o))
    for k, v in kw.items():
        if k == "scheme" and isinstance(v, str):
            v = SCHEMES[v]
        if k == "smoother" and isinstance(v, str):
            v = SMOOTHERS[v]
        if k == "precision" and isinstance(v, str):
            v = PRECISIONS[v]
        if k == "driver" and isinstance(v, str):
            v = DRIVERS[v]
        if k == "factor_form" and isinstance(v, str):
            v = FACTOR_FORMS[v]
        if k == "learned_interp" and v is not None and not isinstance(v, int):
            # a float32 CUDA tensor of mss_gnn_num_params() parameters
            if v.dtype.is_floating_point is False or v.element_size() != 4 or not v.is_cuda:
                raise ValueError("learned_interp must be a float32 CUDA tensor")
            v = v.data_ptr()
        if not hasattr(o, k) or k == "pad_":
            raise KeyError(k)
        setattr(o, k, v)
    return o


def _ptr(t) -> int:
    return t.data_ptr()


class Solver:
    """One library handle on the current device and torch stream."""

    def __init__(self, stream=None, torch_allocator: bool = True):
        import torch
        self._torch = torch
        self.lib = load()
        self.device = torch.cuda.current_device()
        s = stream if stream is not None else torch.cuda.current_stream()
        self.stream = s
        self._keep = []
        if torch_allocator:
            dev = self.device

            def _alloc(nbytes, ctx):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), dev, s)
                except Exception:   # the library reports MSS_ERR_OOM
                    return None

            def _free(ptr, ctx):
                torch.cuda.caching_allocator_delete(ptr)

            a, f = ALLOC_FN(_alloc), FREE_FN(_free)
        else:
            a, f = ALLOC_FN(), FREE_FN()
        self._keep += [a, f]
        h = C.c_void_p()
        self._check(self.lib.mss_create(C.byref(h), C.c_void_p(s.cuda_stream), a, f, None),
                    "mss_create", handle=False)
        self.h = h
        self.N = self.nb = self.nnzb = 0
        self._J = None

    def close(self):
        if getattr(self, "h", None):
            self.lib.mss_destroy(self.h)
            self.h = None

    def __del__(self):
        if sys.is_finalizing():   # the hooks would call into a half torn-down torch
            return
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what, handle=True):
        if st != OK:
            msg = self.lib.mss_status_string(st).decode()
            if handle and getattr(self, "h", None):
                msg += ": " + self.lib.mss_last_error(self.h).decode()
            raise MssError(st, f"{what} -> {msg}")
        return st

    # ---- set-up ---------------------------------------------------------
    def setup(self, row_ptr, col_idx, vals, nb: int, p_idx: int = 0, t_idx: int = 1,
              col_major: bool = False, opts: Options | None = None, **kw):
        """row_ptr/col_idx: int32 CUDA tensors, vals: float64 CUDA tensor of
        nnzb*nb*nb entries. The tensors are kept alive by the solver."""
        torch = self._torch
        for t in (row_ptr, col_idx, vals):
            if not t.is_cuda or not t.is_contiguous():
                raise ValueError("matrix arrays must be contiguous CUDA tensors")
        if row_ptr.dtype != torch.int32 or col_idx.dtype != torch.int32 or vals.dtype != torch.float64:
            raise ValueError("row_ptr/col_idx must be int32 and vals float64")
        o = opts if opts is not None else options(**kw)
        self.N, self.nb, self.nnzb = row_ptr.numel() - 1, nb, col_idx.numel()
        self._J = Bsr(self.N, self.nnzb, _ptr(row_ptr), _ptr(col_idx), _ptr(vals))
        self._Jt = (row_ptr, col_idx, vals)
        self.opts = o
        self._check(self.lib.mss_setup(self.h, C.byref(self._J), nb,
                                       Layout(p_idx, t_idx, int(col_major)), C.byref(o)),
                    "mss_setup")
        return self

    def update_values(self, vals, row_ptr=None, col_idx=None, reuse: str = "pattern"):
        """New block values on the set-up's pattern (mss_update_values);
        reuse "pattern" (same result as a new set-up) or "coarsening" (the
        AMG levels keep their C/F splits). The pattern tensors default to the
        set-up's."""
        torch = self._torch
        rp0, ci0, _ = self._Jt
        rp = rp0 if row_ptr is None else row_ptr
        ci = ci0 if col_idx is None else col_idx
        if not vals.is_cuda or not vals.is_contiguous() or vals.dtype != torch.float64:
            raise ValueError("vals must be a contiguous float64 CUDA tensor")
        J = Bsr(rp.numel() - 1, ci.numel(), _ptr(rp), _ptr(ci), _ptr(vals))
        self._check(self.lib.mss_update_values(self.h, C.byref(J),
                                               {"pattern": 0, "coarsening": 1}[reuse]),
                    "mss_update_values")
        self._J = J
        self._Jt = (rp, ci, vals)
        return self

    def setup_system(self, sysm, **kw):
        torch = self._torch
        rp = torch.from_numpy(np.ascontiguousarray(sysm.row_ptr, np.int32)).cuda()
        ci = torch.from_numpy(np.ascontiguousarray(sysm.col_idx, np.int32)).cuda()
        v = torch.from_numpy(np.ascontiguousarray(sysm.vals, np.float64)).cuda()
        return self.setup(rp, ci, v, sysm.nb, sysm.p_idx, sysm.t_idx, **kw)

    # ---- operators ------------------------------------------------------
    def _vec(self, x):
        torch = self._torch
        if not (x.is_cuda and x.dtype == torch.float64 and x.is_contiguous()
                and x.numel() == self.N * self.nb):
            raise ValueError("expected a contiguous float64 CUDA vector of length N*nb")
        return x

    def _out(self):
        return self._torch.empty(self.N * self.nb, dtype=self._torch.float64, device="cuda")

    def scale_rhs(self, b):
        out = self._out()
        self._check(self.lib.mss_scale_rhs(self.h, _ptr(self._vec(b)), _ptr(out)), "mss_scale_rhs")
        return out

    def spmv(self, x):
        out = self._out()
        self._check(self.lib.mss_spmv(self.h, _ptr(self._vec(x)), _ptr(out)), "mss_spmv")
        return out

    def apply(self, r):
        out = self._out()
        self._check(self.lib.mss_apply(self.h, _ptr(self._vec(r)), _ptr(out)), "mss_apply")
        return out

    def stage(self, which: int, r):
        out = self._out()
        self._check(self.lib.mss_stage_apply(self.h, which, _ptr(self._vec(r)), _ptr(out)),
                    "mss_stage_apply")
        return out

    def solve(self, b, tol: float = 1e-6, maxit: int = 1000, x=None, raise_on_fail=False):
        """Returns (x, info); info['status'] is the library status."""
        x = self._out() if x is None else self._vec(x)
        res = Result()
        st = self.lib.mss_fgmres_solve(self.h, C.byref(self._J), _ptr(self._vec(b)), _ptr(x),
                                       tol, maxit, C.byref(res))
        if st not in (OK, ERR_NOT_CONVERGED) or (raise_on_fail and st != OK):
            self._check(st, "mss_fgmres_solve")
        return x, res.as_dict()

    def solve_host(self, sysm, b=None, tol=1e-6, maxit=1000, opts: Options | None = None,
                   x_out=None, **kw):
        """End-to-end solve from host (numpy) arrays through mss_solve_host.
        Arrays that already are contiguous (e.g. views of pinned memory) are
        passed without a copy; x_out receives the solution when given."""
        o = opts if opts is not None else options(**kw)
        rp = np.ascontiguousarray(sysm.row_ptr, np.int32)
        ci = np.ascontiguousarray(sysm.col_idx, np.int32)
        v = np.ascontiguousarray(sysm.vals, np.float64)
        bb = np.ascontiguousarray(sysm.b if b is None else b, np.float64)
        x = np.empty_like(bb) if x_out is None else x_out
        J = Bsr(rp.shape[0] - 1, ci.shape[0], rp.ctypes.data, ci.ctypes.data, v.ctypes.data)
        res = Result()
        st = self.lib.mss_solve_host(self.h, C.byref(J), sysm.nb,
                                     Layout(sysm.p_idx, sysm.t_idx, 0), C.byref(o),
                                     bb.ctypes.data, x.ctypes.data, tol, maxit, C.byref(res))
        if st not in (OK, ERR_NOT_CONVERGED):
            self._check(st, "mss_solve_host")
        return x, res.as_dict()

    def probe_wait_limit(self) -> bool:
        """Runs one grid-barrier wait that cannot complete; True when it gave
        up at its limit and the kernel returned."""
        t = C.c_int32(0)
        self._check(self.lib.mss_probe_wait_limit(self.h, C.byref(t)), "mss_probe_wait_limit")
        return bool(t.value)

    # ---- measurement ------------------------------------------------------
    def trace(self, enable: bool = True):
        self._check(self.lib.mss_trace_enable(self.h, int(enable)), "mss_trace_enable")

    def trace_read(self, reset: bool = True):
        """{kind: (regions, total ms)} for every traced kind."""
        out = {}
        for name, k in TRACE_KINDS.items():
            n = C.c_int64(0)
            ms = C.c_double(0.0)
            self._check(self.lib.mss_trace_read(self.h, k, C.byref(n), C.byref(ms), int(reset)),
                        "mss_trace_read")
            out[name] = (n.value, ms.value)
        return out

    def residual_norm(self, row_ptr, col_idx, vals, nb, b, x):
        """(||b - J x||, ||b||) for device tensors through mss_residual_norm."""
        torch = self._torch
        J = Bsr(row_ptr.numel() - 1, col_idx.numel(), _ptr(row_ptr), _ptr(col_idx), _ptr(vals))
        out = torch.empty(2, dtype=torch.float64, device="cuda")
        self._check(self.lib.mss_residual_norm(self.h, C.byref(J), nb, _ptr(b), _ptr(x),
                                               _ptr(out)), "mss_residual_norm")
        r = out.cpu()
        return float(r[0]), float(r[1])

    # ---- static condensation (Sec. 3) --------------------------------------
    @staticmethod
    def _full(f):
        """An mss_full over CUDA tensors (row_ptr, col_idx, j11, j21, j12, j22
        in a dict, n1, n2); the tensors must stay alive during the call."""
        t = f["tensors"]
        z = lambda k: _ptr(t[k]) if t.get(k) is not None and t[k].numel() else None
        return Full(t["row_ptr"].numel() - 1, t["col_idx"].numel(), _ptr(t["row_ptr"]),
                    _ptr(t["col_idx"]), f["n1"], f["n2"], _ptr(t["j11"]), z("j21"), z("j12"),
                    z("j22"))

    def condense(self, f, r1, r2):
        """(A blocks, b) of Eq. reduced for the full system f (see _full)."""
        torch = self._torch
        t = f["tensors"]
        a = torch.empty_like(t["j11"])
        b = torch.empty(r1.numel(), dtype=torch.float64, device="cuda")
        J = self._full(f)
        self._check(self.lib.mss_condense(self.h, C.byref(J), _ptr(r1),
                                          _ptr(r2) if r2 is not None and r2.numel() else None,
                                          _ptr(a), _ptr(b)), "mss_condense")
        return a, b

    def recover(self, f, r2, d1):
        torch = self._torch
        d2 = torch.empty(max(r2.numel(), 1), dtype=torch.float64, device="cuda")
        J = self._full(f)
        self._check(self.lib.mss_recover(self.h, C.byref(J), _ptr(r2), _ptr(d1), _ptr(d2)),
                    "mss_recover")
        return d2[:r2.numel()]

    # ---- introspection ----------------------------------------------------
    def scaled(self):
        torch = self._torch
        out = torch.empty(self.nnzb * self.nb * self.nb, dtype=torch.float64, device="cuda")
        self._check(self.lib.mss_get_scaled(self.h, _ptr(out)), "mss_get_scaled")
        return out.view(self.nnzb, self.nb, self.nb)

    def amg_levels(self, which: int):
        torch = self._torch
        out = []
        nlev = self.lib.mss_amg_num_levels(self.h, which)
        for l in range(nlev):
            sz = np.zeros(3, np.int32)
            self._check(self.lib.mss_amg_level_sizes(self.h, which, l, sz.ctypes.data),
                        "mss_amg_level_sizes")
            n, nnz, nnzp = (int(v) for v in sz)
            last = l == nlev - 1
            i32 = dict(dtype=torch.int32, device="cuda")
            f64 = dict(dtype=torch.float64, device="cuda")
            arp, aci, av = torch.empty(n + 1, **i32), torch.empty(max(nnz, 1), **i32), \
                torch.empty(max(nnz, 1), **f64)
            cf, prp = torch.empty(max(n, 1), **i32), torch.empty(n + 1, **i32)
            pci, pv = torch.empty(max(nnzp, 1), **i32), torch.empty(max(nnzp, 1), **f64)
            self._check(self.lib.mss_amg_level_copy(
                self.h, which, l, _ptr(arp), _ptr(aci), _ptr(av),
                None if last else _ptr(cf), None if last else _ptr(prp),
                None if last else _ptr(pci), None if last else _ptr(pv)), "mss_amg_level_copy")
            out.append(dict(A=(arp, aci[:nnz], av[:nnz]), cf=None if last else cf[:n],
                            P=None if last else (prp, pci[:nnzp], pv[:nnzp])))
        return out

    def bilu_ordering(self):
        torch = self._torch
        nc = C.c_int32(0)
        self._check(self.lib.mss_bilu_num_colours(self.h, C.byref(nc)), "mss_bilu_num_colours")
        colour = torch.empty(self.N, dtype=torch.int32, device="cuda")
        perm = torch.empty(self.N, dtype=torch.int32, device="cuda")
        self._check(self.lib.mss_bilu_ordering(self.h, _ptr(colour), _ptr(perm)),
                    "mss_bilu_ordering")
        return nc.value, colour, perm

    def bilu_factors(self):
        """(fv, fdinv): the block ILU(0) factors in colour-major positions,
        shapes (nnzb, nb, nb) and (N, nb, nb) (see mss_bilu_factors)."""
        torch = self._torch
        fv = torch.empty(self.nnzb * self.nb * self.nb, dtype=torch.float64, device="cuda")
        fd = torch.empty(self.N * self.nb * self.nb, dtype=torch.float64, device="cuda")
        self._check(self.lib.mss_bilu_factors(self.h, _ptr(fv), _ptr(fd)), "mss_bilu_factors")
        return fv.view(self.nnzb, self.nb, self.nb), fd.view(self.N, self.nb, self.nb)


SCHEDULES = {"lanes": 0, "fused": 1}


class Batch:
    """Batched set-up and solve of independent systems (mss_batch_*): `lanes`
    worker threads, each with its own handle and stream; the autotuner picks
    threads per CTA and the solve driver per size bucket. schedule="fused"
    solves the systems of each block size in lock step through multi-system
    launches (one graph per group; the autotuner picks their tile shape)."""

    def __init__(self, lanes: int = 8, autotune: bool = True, schedule: str = "lanes"):
        import torch
        self._torch = torch
        self.lib = load()
        self.b = C.c_void_p()
        st = self.lib.mss_batch_create(C.byref(self.b), int(lanes), int(autotune))
        if st != OK:
            raise MssError(st, "mss_batch_create -> " + self.lib.mss_status_string(st).decode())
        self.set_schedule(schedule)

    def set_schedule(self, schedule: str):
        st = self.lib.mss_batch_set_schedule(self.b, SCHEDULES[schedule])
        if st != OK:
            raise MssError(st, "mss_batch_set_schedule -> " + self.lib.mss_status_string(st).decode())

    def __del__(self):
        if sys.is_finalizing():
            return
        if getattr(self, "b", None) and self.b.value:
            self.lib.mss_batch_destroy(self.b)
            self.b = None

    def solve(self, systems, tol: float = 1e-6, maxit: int = 1000, opts: Options | None = None,
              **kw):
        """systems: sequence of dicts with CUDA tensors row_ptr, col_idx (int32),
        vals, b (float64) and ints nb, p_idx, t_idx; an optional float64 tensor
        x receives the solution. Returns (xs, results, infos) as lists."""
        torch = self._torch
        o = opts if opts is not None else options(**kw)
        n = len(systems)
        arr = (System * n)()
        xs, keep = [], []
        for i, sd in enumerate(systems):
            rp, ci, v, b = sd["row_ptr"], sd["col_idx"], sd["vals"], sd["b"]
            for t in (rp, ci, v, b):
                if not t.is_cuda or not t.is_contiguous():
                    raise ValueError("system arrays must be contiguous CUDA tensors")
            x = sd.get("x")
            if x is None:
                x = torch.empty_like(b)
            xs.append(x)
            keep.append((rp, ci, v, b, x))
            arr[i].J = Bsr(rp.numel() - 1, ci.numel(), _ptr(rp), _ptr(ci), _ptr(v))
            arr[i].nb = int(sd["nb"])
            arr[i].layout = Layout(int(sd.get("p_idx", 0)), int(sd.get("t_idx", 1)), 0)
            arr[i].b = _ptr(b)
            arr[i].x = _ptr(x)
        res = (Result * max(n, 1))()
        inf = (BatchInfo * max(n, 1))()
        st = self.lib.mss_batch_solve(self.b, n, arr, C.byref(o), tol, maxit, res, inf)
        if st != OK and all(res[i].status == OK for i in range(n)):
            # the call failed before any system ran (per-system failures are
            # reported in the results)
            raise MssError(st, "mss_batch_solve -> " + self.lib.mss_batch_last_error(self.b).decode())
        del keep
        return xs, [res[i].as_dict() for i in range(n)], [inf[i].as_dict() for i in range(n)]

    def tuned(self):
        """[(bucket, nb, threads, driver)] chosen by the autotuner so far."""
        k = self.lib.mss_batch_tuned(self.b, 0, None)
        buf = (C.c_int32 * (4 * max(k, 1)))()
        k = self.lib.mss_batch_tuned(self.b, k, buf)
        return [tuple(buf[4 * i:4 * i + 4]) for i in range(k)]


class Gnn:
    """Training graph of the learned temperature interpolation (mss_gnn_*),
    copied from a Solver's current CPTR3 set-up (independent of the Solver
    afterwards). Parameters are float32 CUDA tensors of num_params() entries."""

    def __init__(self, solver: "Solver"):
        self.lib = solver.lib
        self._torch = solver._torch
        self.g = C.c_void_p()
        solver._check(self.lib.mss_gnn_create(solver.h, C.byref(self.g)), "mss_gnn_create")
        n, m, t = C.c_int32(), C.c_int32(), C.c_int32()
        self.lib.mss_gnn_info(self.g, C.byref(n), C.byref(m), C.byref(t))
        self.n, self.m, self.t = n.value, m.value, t.value

    @staticmethod
    def num_params() -> int:
        return int(load().mss_gnn_num_params())

    def __del__(self):
        if sys.is_finalizing():
            return
        if getattr(self, "g", None) and self.g.value:
            self.lib.mss_gnn_destroy(self.g)
            self.g = None

    def _check(self, st, what):
        if st != OK:
            raise MssError(st, f"{what} -> {self.lib.mss_status_string(st).decode()}: "
                               f"{self.lib.mss_gnn_last_error(self.g).decode()}")

    def set_vectors(self, starts, nu: int = 10, omega: float = 2.0 / 3.0, norm: str = "A"):
        """starts: float64 CUDA tensor (n, K); norm "A" (residual) or "D"
        (diagonal-weighted interpolation error)."""
        torch = self._torch
        starts = starts.contiguous()
        if not starts.is_cuda or starts.dtype != torch.float64 or starts.shape[0] != self.n:
            raise ValueError("starts must be a float64 CUDA tensor of shape (n, K)")
        self._check(self.lib.mss_gnn_set_vectors(self.g, starts.shape[1], _ptr(starts), nu,
                                                 omega, {"A": 0, "D": 1}[norm]),
                    "mss_gnn_set_vectors")

    def weights(self, params):
        w = self._torch.empty(max(self.t, 1), dtype=self._torch.float64, device="cuda")
        self._check(self.lib.mss_gnn_weights(self.g, _ptr(params), _ptr(w)), "mss_gnn_weights")
        return w[:self.t]

    def loss_grad(self, params, grad=None):
        """(loss, grad): grad is filled when given (float32 CUDA tensor)."""
        L = C.c_double(0.0)
        self._check(self.lib.mss_gnn_loss_grad(self.g, _ptr(params), C.byref(L),
                                               _ptr(grad) if grad is not None else None),
                    "mss_gnn_loss_grad")
        return L.value, grad

    def adam(self, params, m1, m2, grad, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self._check(self.lib.mss_gnn_adam(self.g, _ptr(params), _ptr(m1), _ptr(m2), _ptr(grad),
                                          int(step), lr, beta1, beta2, eps), "mss_gnn_adam")
