"""Python face of the FP64 CPU oracle (``oracle_pf.c``).

TEST INFRASTRUCTURE.  Only the test-suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this module.  The CUDA
library never does, and nothing here imports the library.

The C file does the arithmetic; this module only marshals numpy arrays and
composes the C routines in the order the paper uses them:
ordering -> FormFilledGraph / etree symbolic (Section II.B.1) ->
FormEliminationTree (Section II.B.2) -> FormHierarchicalPartition
(Section II.B, Table I) -> factor (Section III.B) -> substitutions
(Section III.C) -> power-flow iterations (Section III).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle_pf.c")
LIB = os.path.join(HERE, "liboracle_pf.so")

OK, ERR_ARG, ERR_ISLAND, ERR_SINGULAR, ERR_NONFINITE, ERR_NOT_CONVERGED = 0, 1, 2, 3, 4, 5
PQ, PV, SLACK = 1, 2, 3
FDPF, NR = 1, 2

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library next to its source."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = C.CDLL(LIB)
        _declare(_lib)
    return _lib


_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i8p = np.ctypeslib.ndpointer(dtype=np.int8, flags="C_CONTIGUOUS")


def _declare(L):
    I, LL, D = C.c_int, C.c_longlong, C.c_double
    L.or_ybus_pattern.argtypes = [I, I, _i32p, _i32p, _i32p, _i32p]
    L.or_ybus_pattern.restype = I
    L.or_ybus_values.argtypes = [I, I, _i32p, _i32p, _f64p, _f64p, _f64p, _f64p, _i32p, _f64p,
                                 _f64p, _i32p, _i32p, _f64p, _f64p]
    L.or_ybus_values.restype = I
    L.or_bprime_values.argtypes = [I, I, _i32p, _i32p, _f64p, _i32p, _i32p, _i32p, _f64p]
    L.or_bprime_values.restype = I
    L.or_injections.argtypes = [I, _i32p, _i32p, _f64p, _f64p, _f64p, _f64p, _f64p, _f64p]
    L.or_injections.restype = None
    L.or_mismatch.argtypes = [I, _i32p, _f64p, _f64p, _f64p, _f64p, _f64p, _f64p]
    L.or_mismatch.restype = D
    L.or_min_degree.argtypes = [I, _i32p, _i32p, _i32p]
    L.or_min_degree.restype = I
    L.or_filled_graph.argtypes = [I, _i32p, _i32p, _i64p, _i32p, LL]
    L.or_filled_graph.restype = LL
    L.or_symbolic_etree.argtypes = [I, _i32p, _i32p, _i64p, _i32p, LL]
    L.or_symbolic_etree.restype = LL
    L.or_etree.argtypes = [I, _i64p, _i32p, _i32p]
    L.or_etree.restype = None
    L.or_levels.argtypes = [I, _i32p, _i32p]
    L.or_levels.restype = I
    L.or_lu.argtypes = [I, _i32p, _i32p, _f64p, _i64p, _i32p, _f64p, _f64p, _f64p,
                        C.POINTER(C.c_int)]
    L.or_lu.restype = I
    L.or_lu_solve.argtypes = [I, _i64p, _i32p, _f64p, _f64p, _f64p, _f64p, _f64p, I]
    L.or_lu_solve.restype = I
    L.or_power_flow.argtypes = [I, I, I, _i32p, _f64p, _f64p, _f64p, _f64p, _f64p, _f64p, _f64p,
                                _i32p, _i32p, _f64p, _f64p, _f64p, _f64p, _i32p, D, I, I,
                                _f64p, _f64p, C.POINTER(C.c_int), C.POINTER(C.c_double)]
    L.or_power_flow.restype = I
    L.or_adjoint.argtypes = [I, I, _i32p, _f64p, _f64p, _i32p, _i32p, _f64p, _f64p, _f64p, _f64p,
                             _i32p, _f64p, _f64p, _f64p, _f64p, C.POINTER(C.c_double)]
    L.or_adjoint.restype = I
    L.or_jacobian_dense.argtypes = [I, I, _i32p, _f64p, _f64p, _i32p, _i32p, _f64p, _f64p, _f64p,
                                    _f64p, _i32p, _f64p, _f64p, _f64p]
    L.or_jacobian_dense.restype = I


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _tap(case):
    return _f64(case.tap)


# ------------------------------------------------------------------ network

def ybus(case):
    """Section III.A FormMatrixA: (rowptr, col, G, B) of the bus admittance matrix."""
    L = lib()
    n, m = case.n, case.m
    rowptr = np.zeros(n + 1, np.int32)
    col = np.zeros(n + 2 * m + 1, np.int32)
    nnz = L.or_ybus_pattern(n, m, _i32(case.f), _i32(case.t), rowptr, col)
    if nnz < 0:
        raise ValueError("bad branch table")
    col = col[:nnz].copy()
    G = np.zeros(nnz)
    B = np.zeros(nnz)
    rc = L.or_ybus_values(n, m, _i32(case.f), _i32(case.t), _f64(case.r), _f64(case.x),
                          _f64(case.b), _tap(case), _i32(case.status), _f64(case.gs),
                          _f64(case.bs), rowptr, col, G, B)
    if rc:
        raise ValueError(f"ybus values rc={rc}")
    return rowptr, col, G, B


def bprime(case, rowptr, col):
    """XB fast-decoupled B' on the Ybus pattern."""
    Bp = np.zeros(col.shape[0])
    rc = lib().or_bprime_values(case.n, case.m, _i32(case.f), _i32(case.t), _f64(case.x),
                                _i32(case.status), rowptr, col, Bp)
    if rc:
        raise ValueError(f"bprime rc={rc}")
    return Bp


def injections(rowptr, col, G, B, vm, va):
    """Section II.A: P + jQ = V conj(Y V) at every bus."""
    n = rowptr.shape[0] - 1
    P = np.zeros(n)
    Q = np.zeros(n)
    lib().or_injections(n, rowptr, col, G, B, _f64(vm), _f64(va), P, Q)
    return P, Q


def specified(case):
    return case.pg - case.pd, -case.qd


def mismatch(case, rowptr, col, G, B, vm, va):
    """Section II.A: (dP, dQ, max |mismatch|)."""
    P, Q = injections(rowptr, col, G, B, vm, va)
    Psp, Qsp = specified(case)
    dP = np.zeros(case.n)
    dQ = np.zeros(case.n)
    mx = lib().or_mismatch(case.n, _i32(case.btype), _f64(Psp), _f64(Qsp), P, Q, dP, dQ)
    return dP, dQ, mx


# ------------------------------------------------------------------ symbolic

def min_degree(n, adjp, adji):
    perm = np.zeros(max(n, 1), np.int32)
    rc = lib().or_min_degree(n, _i32(adjp), _i32(adji), perm)
    if rc:
        raise RuntimeError(f"min_degree rc={rc}")
    return perm[:n]


def _symbolic(fn, n, adjp, adji):
    cap = max(16, 8 * (len(adji) + n))
    while True:
        Lp = np.zeros(n + 1, np.int64)
        Li = np.zeros(cap, np.int32)
        nz = fn(n, _i32(adjp), _i32(adji), Lp, Li, cap)
        if nz == -2:
            cap *= 4
            continue
        if nz < 0:
            raise MemoryError
        return Lp, Li[:nz].copy()


def filled_graph(n, adjp, adji):
    """Section II.B.1 FormFilledGraph, literal: strict-lower pattern of L by column."""
    return _symbolic(lib().or_filled_graph, n, adjp, adji)


def symbolic_etree(n, adjp, adji):
    """Etree-merge symbolic factorisation: same output as filled_graph."""
    return _symbolic(lib().or_symbolic_etree, n, adjp, adji)


def etree(n, Lp, Li):
    """Section II.B.2 FormEliminationTree."""
    parent = np.zeros(max(n, 1), np.int32)
    lib().or_etree(n, _i64(Lp), _i32(Li), parent)
    return parent[:n]


def _i64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


def levels(parent):
    """Section II.B FormHierarchicalPartition: level of every node (leaves = 1)."""
    n = len(parent)
    lev = np.zeros(max(n, 1), np.int32)
    nl = lib().or_levels(n, _i32(parent), lev)
    if nl < 0:
        raise ValueError("parent array is not a forest")
    return lev[:n], nl


def matrix_buses(case, which):
    """Buses in a matrix, ascending: 'bp' (B', NR) = non-slack, 'bpp' (B'') = PQ."""
    if which in ("bp", "nr"):
        return np.nonzero(case.btype != SLACK)[0].astype(np.int32)
    if which == "bpp":
        return np.nonzero(case.btype == PQ)[0].astype(np.int32)
    raise ValueError(which)


def local_graph(case, which, rowptr=None, col=None):
    """Induced bus graph of a matrix in local (ascending bus) numbering, CSR, no diagonal."""
    if rowptr is None:
        rowptr, col, _, _ = ybus(case)
    buses = matrix_buses(case, which)
    loc = np.full(case.n, -1, np.int64)
    loc[buses] = np.arange(buses.shape[0])
    gp = [0]
    gi = []
    for i in buses:
        nb = [int(loc[j]) for j in col[rowptr[i]:rowptr[i + 1]] if j != i and loc[j] >= 0]
        gi.extend(nb)
        gp.append(len(gi))
    return buses, np.array(gp, np.int32), np.array(gi, np.int32)


def permute_graph(n, gp, gi, perm):
    """Graph of P A P^T: vertex k of the result is vertex perm[k] of the input."""
    iperm = np.empty(n, np.int64)
    iperm[perm] = np.arange(n)
    pp = [0]
    pi = []
    for k in range(n):
        a = perm[k]
        nb = sorted(int(iperm[j]) for j in gi[gp[a]:gp[a + 1]])
        pi.extend(nb)
        pp.append(len(pi))
    return np.array(pp, np.int32), np.array(pi, np.int32)


def analyze(case, which, literal=False):
    """Ordering, filled pattern, elimination tree and levels of one matrix.

    Returns dict(buses, perm, Lp, Li, parent, level, nlevels); ``perm[k]`` is
    the local index eliminated at step k, L is in permuted numbering."""
    rowptr, col, _, _ = ybus(case)
    buses, gp, gi = local_graph(case, which, rowptr, col)
    n = buses.shape[0]
    perm = min_degree(n, gp, gi)
    pp, pi = permute_graph(n, gp, gi, perm)
    Lp, Li = (filled_graph if literal else symbolic_etree)(n, pp, pi)
    parent = etree(n, Lp, Li)
    level, nl = levels(parent)
    return dict(buses=buses, perm=perm, Lp=Lp, Li=Li, parent=parent, level=level, nlevels=nl)


# ------------------------------------------------------------------ numeric

def lu(n, Ap, Ai, Ax, Lp, Li):
    """Section III.B: LU without pivoting on the filled pattern.  Returns (Lx, Ux, d)."""
    nz = len(Li)
    Lx = np.zeros(max(nz, 1))
    Ux = np.zeros(max(nz, 1))
    d = np.zeros(max(n, 1))
    bad = C.c_int(-1)
    rc = lib().or_lu(n, _i32(Ap), _i32(Ai), _f64(Ax), _i64(Lp), _i32(Li), Lx, Ux, d,
                     C.byref(bad))
    return rc, Lx[:nz], Ux[:nz], d[:n], bad.value


def lu_solve(n, Lp, Li, Lx, Ux, d, rhs, transpose=False):
    """Section III.C forward substitution, normalisation (Eq. 4), back substitution."""
    x = np.zeros(max(n, 1))
    nz = len(Li)
    Lx1 = np.zeros(max(nz, 1)); Lx1[:nz] = Lx
    Ux1 = np.zeros(max(nz, 1)); Ux1[:nz] = Ux
    rhs1 = np.zeros(max(n, 1)); rhs1[:n] = rhs
    d1 = np.ones(max(n, 1)); d1[:n] = d
    lib().or_lu_solve(n, _i64(Lp), _i32(Li), Lx1, Ux1, d1, rhs1, x, 1 if transpose else 0)
    return x[:n]


def bmatrix_values(case, which, rowptr=None, col=None, G=None, B=None):
    """Values of B' ('bp') or B'' ('bpp') on the Ybus pattern."""
    if rowptr is None:
        rowptr, col, G, B = ybus(case)
    if which == "bp":
        return bprime(case, rowptr, col)
    if which == "bpp":
        return -B
    raise ValueError(which)


def permuted_csc(case, which, an, vals, rowptr, col):
    """CSC of P A P^T for a symmetric B-type matrix given its values on the Ybus pattern."""
    buses, perm = an["buses"], an["perm"]
    n = buses.shape[0]
    loc = np.full(case.n, -1, np.int64)
    loc[buses] = np.arange(n)
    iperm = np.empty(n, np.int64)
    iperm[perm] = np.arange(n)
    Ap = [0]
    Ai = []
    Ax = []
    for c in range(n):
        i = buses[perm[c]]
        for p in range(rowptr[i], rowptr[i + 1]):
            j = col[p]
            if loc[j] >= 0:
                Ai.append(int(iperm[loc[j]]))
                Ax.append(float(vals[p]))
        Ap.append(len(Ai))
    return np.array(Ap, np.int32), np.array(Ai, np.int32), np.array(Ax)


def factor_bmatrix(case, which):
    """LDL^T of B' or B'' in the minimum-degree order: (analysis, L values, D)."""
    rowptr, col, G, B = ybus(case)
    an = analyze(case, which)
    vals = bmatrix_values(case, which, rowptr, col, G, B)
    Ap, Ai, Ax = permuted_csc(case, which, an, vals, rowptr, col)
    n = an["buses"].shape[0]
    rc, Lx, Ux, d, bad = lu(n, Ap, Ai, Ax, an["Lp"], an["Li"])
    if rc:
        raise RuntimeError(f"factor rc={rc} at {bad}")
    return an, Lx, d, (Ap, Ai, Ax)


# ------------------------------------------------------------------ power flow

def power_flow(case, method=FDPF, tol=1e-8, max_iter=None, vm0=None, va0=None):
    """Section III power flow.  Returns (status, vm, va, iters, maxmis)."""
    if max_iter is None:
        max_iter = 200 if method == FDPF else 20
    n = case.n
    vm = np.zeros(n) if vm0 is None else _f64(vm0).copy()
    va = np.zeros(n) if va0 is None else _f64(va0).copy()
    it = C.c_int(0)
    mx = C.c_double(0.0)
    rc = lib().or_power_flow(method, n, case.m, _i32(case.btype), _f64(case.pd), _f64(case.qd),
                             _f64(case.gs), _f64(case.bs), _f64(case.pg), _f64(case.vset),
                             _f64(case.va), _i32(case.f), _i32(case.t), _f64(case.r),
                             _f64(case.x), _f64(case.b), _tap(case), _i32(case.status),
                             float(tol), int(max_iter), 0 if vm0 is None else 1, vm, va,
                             C.byref(it), C.byref(mx))
    return rc, vm, va, it.value, mx.value


def adjoint(case, vm, va):
    """Gradient of J = sum (V-1)^2 + sum P_i w.r.t. specified P and Q (fresh factor at x*)."""
    n = case.n
    dP = np.zeros(n)
    dQ = np.zeros(n)
    J = C.c_double(0.0)
    rc = lib().or_adjoint(n, case.m, _i32(case.btype), _f64(case.gs), _f64(case.bs),
                          _i32(case.f), _i32(case.t), _f64(case.r), _f64(case.x),
                          _f64(case.b), _tap(case), _i32(case.status), _f64(vm), _f64(va), dP,
                          dQ, C.byref(J))
    if rc:
        raise RuntimeError(f"adjoint rc={rc}")
    return dP, dQ, J.value


def branch_flows(case, vm, va):
    """Flows of every branch at the state (vm, va): the complex power entering
    the branch at its from end, S_f = V_f conj(I_f), and at its to end, S_t =
    V_t conj(I_t), with the pi model of the admittance matrix (Section III.A:
    series y = 1/(r + jx), charging jb/2 at each end, the tap t on the from
    side): I_f = (y + jb/2)/t^2 V_f - y/t V_t, I_t = -y/t V_f + (y + jb/2) V_t.
    Out-of-service branches carry nothing.  Returns (Pf, Qf, Pt, Qt, loss)
    with loss = sum of Pf + Pt over branches plus the shunt consumption
    sum gs V^2 (the total active loss)."""
    V = vm * np.exp(1j * va)
    m = case.m
    Pf = np.zeros(m); Qf = np.zeros(m); Pt = np.zeros(m); Qt = np.zeros(m)
    for k in range(m):
        if not case.status[k]:
            continue
        y = 1.0 / complex(case.r[k], case.x[k])
        t = case.tap[k] if case.tap[k] != 0 else 1.0
        ysh = 0.5j * case.b[k]
        vf, vt = V[case.f[k]], V[case.t[k]]
        i_f = (y + ysh) / (t * t) * vf - y / t * vt
        i_t = -y / t * vf + (y + ysh) * vt
        sf = vf * np.conj(i_f)
        st = vt * np.conj(i_t)
        Pf[k], Qf[k], Pt[k], Qt[k] = sf.real, sf.imag, st.real, st.imag
    loss = float(np.sum(Pf + Pt) + np.sum(case.gs * vm ** 2))
    return Pf, Qf, Pt, Qt, loss


def objective(case, vm, va):
    rowptr, col, G, B = ybus(case)
    P, _ = injections(rowptr, col, G, B, vm, va)
    return float(np.sum((vm - 1.0) ** 2) + np.sum(P))


def jacobian_dense(case, vm, va):
    """NR Jacobian at (vm, va), natural non-slack bus order, (theta, V) per bus."""
    nb = int(np.sum(case.btype != SLACK))
    Jd = np.zeros((2 * nb) * (2 * nb))
    rc = lib().or_jacobian_dense(case.n, case.m, _i32(case.btype), _f64(case.gs), _f64(case.bs),
                                 _i32(case.f), _i32(case.t), _f64(case.r), _f64(case.x),
                                 _f64(case.b), _tap(case), _i32(case.status), _f64(vm), _f64(va),
                                 Jd)
    if rc:
        raise RuntimeError(f"jacobian rc={rc}")
    return Jd.reshape(2 * nb, 2 * nb)
