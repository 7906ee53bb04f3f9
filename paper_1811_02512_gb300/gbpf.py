"""Thin ctypes binding of libgbpf (include/gbpf.h), same names as the C ABI.

Only argument marshalling lives here: every step of the power flow runs in
the CUDA library.  PyTorch supplies device memory (``Tensor.data_ptr()``) and
streams.  If the shared library is missing the import of any entry point
raises; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

from . import gridgen

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libgbpf.so")
HEADER = os.path.join(os.path.dirname(PKG), "include", "gbpf.h")

PF_OK, PF_ERR_ARG, PF_ERR_ISLAND, PF_ERR_SINGULAR, PF_ERR_NONFINITE = 0, 1, 2, 3, 4
PF_ERR_NOT_CONVERGED, PF_ERR_TIMEOUT, PF_ERR_CUDA, PF_ERR_OOM, PF_ERR_STATE = 5, 6, 7, 8, 9
STATUS_NAMES = {0: "PF_OK", 1: "PF_ERR_ARG", 2: "PF_ERR_ISLAND", 3: "PF_ERR_SINGULAR",
                4: "PF_ERR_NONFINITE", 5: "PF_ERR_NOT_CONVERGED", 6: "PF_ERR_TIMEOUT",
                7: "PF_ERR_CUDA", 8: "PF_ERR_OOM", 9: "PF_ERR_STATE"}
PF_BUS_PQ, PF_BUS_PV, PF_BUS_SLACK = 1, 2, 3
PF_MAT_BP, PF_MAT_BPP = 0, 1
PF_FDPF, PF_NR = 1, 2
PF_FP64, PF_FP32 = 0, 1


class pf_bus(C.Structure):
    _fields_ = [("id", C.c_int32), ("type", C.c_int32), ("pd", C.c_double), ("qd", C.c_double),
                ("gs", C.c_double), ("bs", C.c_double), ("pg", C.c_double), ("vset", C.c_double),
                ("va", C.c_double)]


class pf_branch(C.Structure):
    _fields_ = [("from_", C.c_int32), ("to", C.c_int32), ("r", C.c_double), ("x", C.c_double),
                ("b", C.c_double), ("tap", C.c_double), ("status", C.c_int32)]


class pf_symbolic_info(C.Structure):
    _fields_ = [("n", C.c_int32 * 2), ("nnz_l", C.c_int64 * 2), ("nlevels", C.c_int32 * 2),
                ("max_col", C.c_int32 * 2), ("nupdates", C.c_int64 * 2), ("nnz_ybus", C.c_int32),
                ("analyze_ms", C.c_double)]


class pf_run_opts(C.Structure):
    _fields_ = [("method", C.c_int32), ("precision", C.c_int32), ("tol", C.c_double),
                ("max_iter", C.c_int32), ("ir_max", C.c_int32), ("ir_tol", C.c_double),
                ("ir_abs", C.c_double), ("flat_start", C.c_int32), ("spin_limit", C.c_int32),
                ("engine", C.c_int32), ("fallback", C.c_int32)]


class pf_case_result(C.Structure):
    _fields_ = [("status", C.c_int32), ("iters", C.c_int32), ("ir_steps", C.c_int32),
                ("method", C.c_int32), ("max_mismatch", C.c_double)]


assert C.sizeof(pf_bus) == gridgen.BUS_DTYPE.itemsize
assert C.sizeof(pf_branch) == gridgen.BRANCH_DTYPE.itemsize
CASE_RESULT_DTYPE = np.dtype([("status", "<i4"), ("iters", "<i4"), ("ir_steps", "<i4"),
                              ("method", "<i4"), ("max_mismatch", "<f8")], align=True)

_lib = None
_P = C.c_void_p


def load():
    """Loads libgbpf.so (built by paper_1811_02512_gb300.build); raises if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run __graft_entry__.build() "
                              "(the CUDA library is required; there is no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        S = C.c_int
        L.pf_create.argtypes = [_P, C.c_int32, _P, C.c_int32, C.POINTER(_P)]
        L.pf_analyze.argtypes = [_P, C.POINTER(pf_symbolic_info)]
        L.pf_get_symbolic.argtypes = [_P, C.c_int32, _P, _P, _P, _P, _P]
        L.pf_set_cases.argtypes = [_P, C.c_int32, _P, _P]
        L.pf_factor.argtypes = [_P, C.c_int32, C.c_int32, _P]
        L.pf_get_factor.argtypes = [_P, C.c_int32, C.c_int32, C.c_int32, _P, _P, _P]
        L.pf_solve.argtypes = [_P, C.c_int32, C.c_int32, C.c_int32, _P, C.c_int32, _P]
        L.pf_mismatch.argtypes = [_P, _P, _P, _P, _P, _P, C.c_int32, _P]
        L.pf_run_to_tol.argtypes = [_P, C.POINTER(pf_run_opts), _P, _P, _P, _P]
        L.pf_get_ybus.argtypes = [_P, _P, _P, _P, _P]
        L.pf_set_profiling.argtypes = [_P, C.c_int32]
        L.pf_set_graphs.argtypes = [_P, C.c_int32]
        L.pf_set_graphs.restype = S
        L.pf_get_profile.argtypes = [_P, C.c_int32, _P, _P, C.c_int32]
        L.pf_set_injections.argtypes = [_P, _P, _P, _P]
        L.pf_adjoint.argtypes = [_P, C.c_int32, _P, _P, _P, _P, _P, _P, _P, _P]
        L.pf_objective.argtypes = [_P, _P, _P, _P, _P, _P, _P]
        for nm in ("pf_set_injections", "pf_adjoint", "pf_objective"):
            getattr(L, nm).restype = S
        L.pf_mismatch_static.argtypes = [C.c_int32] + [_P] * 13
        L.pf_mismatch_static.restype = S
        L.pf_last_error.argtypes = [_P]
        L.pf_last_error.restype = C.c_char_p
        L.pf_destroy.argtypes = [_P]
        L.pf_destroy.restype = None
        L.pf_etree_levels_device.argtypes = [C.c_int32, _P, _P, _P, _P, _P, _P, _P]
        L.pf_etree_levels_device.restype = S
        L.pf_branch_flows.argtypes = [_P, _P, _P, C.c_int32, _P, _P, _P]
        L.pf_branch_flows.restype = S
        L.pf_autotune.argtypes = [_P, C.POINTER(pf_run_opts), _P, _P, C.c_int32, _P, _P]
        L.pf_get_tuning.argtypes = [_P, _P]
        L.pf_set_tuning.argtypes = [_P, _P]
        for nm in ("pf_autotune", "pf_get_tuning", "pf_set_tuning"):
            getattr(L, nm).restype = S
        L.pf_pack_create.argtypes = [_P, C.c_int32, C.POINTER(_P)]
        L.pf_pack_create.restype = S
        L.pf_pack_run.argtypes = [_P, C.POINTER(pf_run_opts), _P, _P, _P, _P]
        L.pf_pack_run.restype = S
        L.pf_pack_last_error.argtypes = [_P]
        L.pf_pack_last_error.restype = C.c_char_p
        L.pf_pack_destroy.argtypes = [_P]
        L.pf_pack_destroy.restype = None
        for name in ("pf_create", "pf_analyze", "pf_get_symbolic", "pf_set_cases", "pf_factor",
                     "pf_get_factor", "pf_solve", "pf_mismatch", "pf_run_to_tol", "pf_get_ybus",
                     "pf_set_profiling", "pf_get_profile"):
            getattr(L, name).restype = S
        _lib = L
    return _lib


def header_functions():
    """Names of every function the public header declares."""
    with open(HEADER) as fh:
        text = fh.read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ ]*?\**\s*\**(pf_\w+)\s*\(",
                                 text, flags=re.M)))


class PFError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return a.ctypes.data_as(C.c_void_p)


def _stream(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


# ----------------------------------------------------------------- C ABI names

def pf_create(bus_table: np.ndarray, branch_table: np.ndarray):
    L = load()
    bus_table = np.ascontiguousarray(bus_table, dtype=gridgen.BUS_DTYPE)
    branch_table = np.ascontiguousarray(branch_table, dtype=gridgen.BRANCH_DTYPE)
    out = C.c_void_p()
    st = L.pf_create(_ptr(bus_table), len(bus_table), _ptr(branch_table), len(branch_table),
                     C.byref(out))
    if st != PF_OK:
        raise PFError(st, "pf_create rejected the tables")
    return out


def _check(ctx, st, what):
    if st != PF_OK:
        raise PFError(st, f"{what}: {load().pf_last_error(ctx).decode()}")


def pf_analyze(ctx):
    info = pf_symbolic_info()
    _check(ctx, load().pf_analyze(ctx, C.byref(info)), "pf_analyze")
    return info


def pf_get_symbolic(ctx, which, info):
    n, nz = info.n[which], info.nnz_l[which]
    perm = np.zeros(n, np.int32)
    parent = np.zeros(n, np.int32)
    level = np.zeros(n, np.int32)
    Lp = np.zeros(n + 1, np.int64)
    Li = np.zeros(max(nz, 1), np.int32)
    _check(ctx, load().pf_get_symbolic(ctx, which, _ptr(perm), _ptr(parent), _ptr(level), _ptr(Lp),
                                       _ptr(Li)), "pf_get_symbolic")
    return dict(perm=perm, parent=parent, level=level, Lp=Lp, Li=Li[:nz])


def pf_set_cases(ctx, ncase, load_scale=None, outage=None):
    ls = None if load_scale is None else np.ascontiguousarray(load_scale, dtype=np.float64)
    out = None if outage is None else np.ascontiguousarray(outage, dtype=np.int32)
    _check(ctx, load().pf_set_cases(ctx, int(ncase), _ptr(ls), _ptr(out)), "pf_set_cases")


def pf_factor(ctx, which, precision=PF_FP64, stream=None):
    _check(ctx, load().pf_factor(ctx, which, precision, _stream(stream)), "pf_factor")


def pf_get_factor(ctx, which, precision, case, info):
    n, nz = info.n[which], info.nnz_l[which]
    D = np.zeros(n)
    Lx = np.zeros(max(nz, 1))
    st = C.c_int32(0)
    _check(ctx, load().pf_get_factor(ctx, which, precision, case, _ptr(D), _ptr(Lx), C.byref(st)),
           "pf_get_factor")
    return D, Lx[:nz], st.value


def pf_solve(ctx, which, precision, rhs_dev, ncase, transpose=0, stream=None):
    _check(ctx, load().pf_solve(ctx, which, precision, transpose, _ptr(rhs_dev), int(ncase),
                                _stream(stream)), "pf_solve")


def pf_mismatch(ctx, vm_dev, va_dev, dp_dev, dq_dev, maxmis_dev, ncase, stream=None):
    _check(ctx, load().pf_mismatch(ctx, _ptr(vm_dev), _ptr(va_dev), _ptr(dp_dev), _ptr(dq_dev),
                                   _ptr(maxmis_dev), int(ncase), _stream(stream)), "pf_mismatch")


PF_ENGINE_AUTO, PF_ENGINE_BLOCK, PF_ENGINE_LANES, PF_ENGINE_CLUSTER = 0, 1, 2, 3


def run_opts(method=PF_FDPF, precision=PF_FP64, tol=1e-8, max_iter=None, ir_max=5, ir_tol=1e-10,
             ir_abs=0.0, flat_start=1, spin_limit=0, engine=PF_ENGINE_AUTO, fallback=0):
    if max_iter is None:
        max_iter = 200 if method == PF_FDPF else 20
    return pf_run_opts(method, precision, tol, max_iter, ir_max, ir_tol, ir_abs, flat_start,
                       spin_limit, engine, fallback)


def pf_run_to_tol(ctx, opts, vm_dev, va_dev, ncase, stream=None, check=True):
    res = np.zeros(ncase, dtype=CASE_RESULT_DTYPE)
    st = load().pf_run_to_tol(ctx, C.byref(opts), _ptr(vm_dev), _ptr(va_dev), _ptr(res),
                              _stream(stream))
    if check and st not in (PF_OK, PF_ERR_NOT_CONVERGED, PF_ERR_SINGULAR, PF_ERR_NONFINITE):
        _check(ctx, st, "pf_run_to_tol")
    return st, res


def pf_get_ybus(ctx, nbus, nnz):
    rowptr = np.zeros(nbus + 1, np.int32)
    col = np.zeros(nnz, np.int32)
    G = np.zeros(nnz)
    B = np.zeros(nnz)
    _check(ctx, load().pf_get_ybus(ctx, _ptr(rowptr), _ptr(col), _ptr(G), _ptr(B)), "pf_get_ybus")
    return rowptr, col, G, B


PF_K_YBUS, PF_K_SPEC, PF_K_ASSEMBLE, PF_K_FACTOR, PF_K_SOLVE, PF_K_MISMATCH, PF_K_RUN = range(7)
KERNEL_KINDS = ["ybus", "spec", "assemble", "factor", "solve", "mismatch", "run"]


def pf_set_profiling(ctx, on):
    _check(ctx, load().pf_set_profiling(ctx, 1 if on else 0), "pf_set_profiling")


def pf_get_profile(ctx, kind, reset=False):
    n = C.c_int64(0)
    ms = C.c_double(0.0)
    _check(ctx, load().pf_get_profile(ctx, kind, C.byref(n), C.byref(ms), 1 if reset else 0),
           "pf_get_profile")
    return n.value, ms.value


def pf_set_injections(ctx, psp_dev, qsp_dev, stream=None):
    _check(ctx, load().pf_set_injections(ctx, _ptr(psp_dev), _ptr(qsp_dev), _stream(stream)),
           "pf_set_injections")


def pf_adjoint(ctx, precision, vm_dev, va_dev, gva_dev, gvm_dev, dJdP_dev, dJdQ_dev, ncase,
               stream=None):
    res = np.zeros(ncase, dtype=CASE_RESULT_DTYPE)
    _check(ctx, load().pf_adjoint(ctx, precision, _ptr(vm_dev), _ptr(va_dev), _ptr(gva_dev),
                                  _ptr(gvm_dev), _ptr(dJdP_dev), _ptr(dJdQ_dev), _ptr(res),
                                  _stream(stream)), "pf_adjoint")
    return res


def pf_objective(ctx, vm_dev, va_dev, J_dev, gva_dev, gvm_dev, stream=None):
    _check(ctx, load().pf_objective(ctx, _ptr(vm_dev), _ptr(va_dev), _ptr(J_dev), _ptr(gva_dev),
                                    _ptr(gvm_dev), _stream(stream)), "pf_objective")


PF_STATIC_MAX_BUS = 131072


def pf_mismatch_static(nbus, rowptr_dev, col_dev, G_dev, B_dev, btype_dev, psp_dev, qsp_dev,
                       vm_dev, va_dev, dp_dev, dq_dev, maxmis_dev, stream=None):
    """Allocation-free single-case mismatch; returns the pf_status code."""
    return load().pf_mismatch_static(int(nbus), _ptr(rowptr_dev), _ptr(col_dev), _ptr(G_dev),
                                     _ptr(B_dev), _ptr(btype_dev), _ptr(psp_dev), _ptr(qsp_dev),
                                     _ptr(vm_dev), _ptr(va_dev), _ptr(dp_dev), _ptr(dq_dev),
                                     _ptr(maxmis_dev), _stream(stream))


def pf_last_error(ctx):
    return load().pf_last_error(ctx).decode()


def pf_destroy(ctx):
    if ctx:
        load().pf_destroy(ctx)


# ----------------------------------------------------------------- convenience

def pf_etree_levels_device(n, Lp_dev, Li_dev, parent_dev, level_dev, nlev_dev, scratch_dev,
                           stream=None):
    st = load().pf_etree_levels_device(int(n), _ptr(Lp_dev), _ptr(Li_dev), _ptr(parent_dev),
                                       _ptr(level_dev), _ptr(nlev_dev), _ptr(scratch_dev),
                                       _stream(stream))
    if st != PF_OK:
        raise PFError(st, "pf_etree_levels_device")


def pf_branch_flows(ctx, vm_dev, va_dev, ncase, flows_dev, loss_dev, stream=None):
    """flows_dev [ncase, nbranch, 4] (P_f, Q_f, P_t, Q_t), loss_dev [ncase]."""
    _check(ctx, load().pf_branch_flows(ctx, _ptr(vm_dev), _ptr(va_dev), int(ncase), _ptr(flows_dev),
                                       _ptr(loss_dev), _stream(stream)), "pf_branch_flows")


class pf_tuning(C.Structure):
    _fields_ = [("engine", C.c_int32), ("cluster", C.c_int32), ("factor", C.c_int32),
                ("tail", C.c_int32), ("outage", C.c_int32), ("threads", C.c_int32), ("ms", C.c_double)]


def pf_autotune(ctx, opts, vm_dev, va_dev, reps=3, stream=None):
    """Times the applicable kernel mappings on this context's problem and keeps
    the fastest converging one; returns it as a dict."""
    t = pf_tuning()
    _check(ctx, load().pf_autotune(ctx, C.byref(opts), _ptr(vm_dev), _ptr(va_dev), int(reps),
                                   C.byref(t), _stream(stream)), "pf_autotune")
    return {k: getattr(t, k) for k, _ in pf_tuning._fields_}


def pf_get_tuning(ctx):
    t = pf_tuning()
    _check(ctx, load().pf_get_tuning(ctx, C.byref(t)), "pf_get_tuning")
    return {k: getattr(t, k) for k, _ in pf_tuning._fields_}


def pf_set_graphs(ctx, on):
    """CUDA-graph replay of repeated runs on (default) or off."""
    _check(ctx, load().pf_set_graphs(ctx, int(bool(on))), "pf_set_graphs")


def pf_set_tuning(ctx, engine=0, cluster=0, factor=0, tail=0, outage=0, threads=0):
    t = pf_tuning(engine, cluster, factor, tail, outage, threads, 0.0)
    _check(ctx, load().pf_set_tuning(ctx, C.byref(t)), "pf_set_tuning")


class Pack:
    """An uneven multi-grid batch over analysed ``Grid`` objects (which it
    does not own): ``run`` solves every grid in one persistent launch."""

    def __init__(self, grids):
        self.grids = list(grids)
        arr = (_P * len(self.grids))(*[g.ctx for g in self.grids])
        h = _P()
        st = load().pf_pack_create(arr, len(self.grids), C.byref(h))
        if st != PF_OK:
            raise PFError(st, "pf_pack_create")
        self.h = h
        self.nbus = [g.nbus for g in self.grids]
        self.offset = np.concatenate([[0], np.cumsum(self.nbus)]).astype(np.int64)

    def run(self, opts, vm_dev, va_dev, stream=None, check=True):
        """vm_dev/va_dev: device float64 vectors of sum(nbus), grids in pack order."""
        res = np.zeros(len(self.grids), dtype=CASE_RESULT_DTYPE)
        st = load().pf_pack_run(self.h, C.byref(opts), _ptr(vm_dev), _ptr(va_dev), _ptr(res),
                                _stream(stream))
        if check and st not in (PF_OK, PF_ERR_NOT_CONVERGED, PF_ERR_SINGULAR, PF_ERR_NONFINITE):
            raise PFError(st, "pf_pack_run: " + load().pf_pack_last_error(self.h).decode())
        return st, res

    def last_error(self):
        return load().pf_pack_last_error(self.h).decode()

    def close(self):
        if getattr(self, "h", None):
            load().pf_pack_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Grid:
    """A context for one grid: ``Grid(case)`` runs pf_create and pf_analyze."""

    def __init__(self, case):
        self.case = case
        self.ctx = pf_create(case.bus_table(), case.branch_table())
        self.info = pf_analyze(self.ctx)
        self.ncase = 0

    @property
    def nbus(self):
        return self.case.n

    def symbolic(self, which):
        return pf_get_symbolic(self.ctx, which, self.info)

    def set_cases(self, ncase=1, load_scale=None, outage=None):
        pf_set_cases(self.ctx, ncase, load_scale, outage)
        self.ncase = ncase

    def close(self):
        if self.ctx:
            pf_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------- autograd

def _torch():
    import torch
    return torch


class PowerFlowFn:
    """torch.autograd.Function: (Psp, Qsp) [ncase, nbus] -> (vm, va) by
    Newton-Raphson in libgbpf; backward by the adjoint kernel (transposed
    solve with the forward factors, FP64-refined)."""

    _fn = None

    @classmethod
    def apply(cls, grid, psp, qsp, precision=PF_FP64, tol=1e-10, max_iter=30):
        if cls._fn is None:
            torch = _torch()

            class _PF(torch.autograd.Function):
                @staticmethod
                def forward(ctx_, psp_, qsp_, g, prec, tol_, mi):
                    psp_c = psp_.detach().contiguous()
                    qsp_c = qsp_.detach().contiguous()
                    ncase = psp_c.shape[0]
                    pf_set_injections(g.ctx, psp_c, qsp_c)
                    vm = torch.zeros_like(psp_c)
                    va = torch.zeros_like(psp_c)
                    st, res = pf_run_to_tol(g.ctx, run_opts(PF_NR, prec, tol=tol_, max_iter=mi), vm,
                                            va, ncase)
                    if st != PF_OK:
                        raise PFError(st, pf_last_error(g.ctx))
                    ctx_.save_for_backward(vm, va)
                    ctx_.g, ctx_.prec = g, prec
                    ctx_.mark_non_differentiable()
                    return vm, va

                @staticmethod
                def backward(ctx_, gvm, gva):
                    vm, va = ctx_.saved_tensors
                    g = ctx_.g
                    gvm = torch.zeros_like(vm) if gvm is None else gvm.contiguous()
                    gva = torch.zeros_like(va) if gva is None else gva.contiguous()
                    dP = torch.empty_like(vm)
                    dQ = torch.empty_like(vm)
                    pf_adjoint(g.ctx, ctx_.prec, vm, va, gva, gvm, dP, dQ, vm.shape[0])
                    return dP, dQ, None, None, None, None

            cls._fn = _PF
        return cls._fn.apply(psp, qsp, grid, precision, tol, max_iter)


class ObjectiveFn:
    """torch.autograd.Function: (vm, va) -> J = sum (V - 1)^2 + total losses
    per case, value and gradient from the objective kernel."""

    _fn = None

    @classmethod
    def apply(cls, grid, vm, va):
        if cls._fn is None:
            torch = _torch()

            class _Obj(torch.autograd.Function):
                @staticmethod
                def forward(ctx_, vm_, va_, g):
                    vm_c, va_c = vm_.detach().contiguous(), va_.detach().contiguous()
                    J = torch.empty(vm_c.shape[0], dtype=torch.float64, device=vm_c.device)
                    gva = torch.empty_like(vm_c)
                    gvm = torch.empty_like(vm_c)
                    pf_objective(g.ctx, vm_c, va_c, J, gva, gvm)
                    ctx_.save_for_backward(gvm, gva)
                    return J

                @staticmethod
                def backward(ctx_, gJ):
                    gvm, gva = ctx_.saved_tensors
                    return gJ[:, None] * gvm, gJ[:, None] * gva, None

            cls._fn = _Obj
        return cls._fn.apply(vm, va, grid)
