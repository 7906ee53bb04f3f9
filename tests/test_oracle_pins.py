"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Every check here is independent of the oracle's own arithmetic: closed forms
derived from Ohm's and Kirchhoff's laws, energy conservation, hand-worked
orderings, the paper's Table I, dense library factorisations, brute-force
boolean elimination and finite differences.  No GPU is needed.
"""
import math
import os

import numpy as np
import pytest

from paper_1811_02512_gb300 import gridgen
from paper_1811_02512_gb300.gridgen import Case

GOLD = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------- helpers

def two_bus(kind, P, Q_or_V, r, x, b, tap=1.0, v1=1.0, reverse=False):
    """Slack bus 0 and one PQ (kind 'pq', load P + jQ) or PV (kind 'pv', generation
    P at |V| = Q_or_V) bus, joined by one pi-model branch."""
    btype = np.array([gridgen.SLACK, gridgen.PQ if kind == "pq" else gridgen.PV], np.int32)
    pd = np.array([0.0, P if kind == "pq" else 0.0])
    qd = np.array([0.0, Q_or_V if kind == "pq" else 0.0])
    pg = np.array([0.0, P if kind == "pv" else 0.0])
    vset = np.array([v1, Q_or_V if kind == "pv" else 1.0])
    f, t = (np.array([1], np.int32), np.array([0], np.int32)) if reverse else \
        (np.array([0], np.int32), np.array([1], np.int32))
    return Case(name="2bus", btype=btype, pd=pd, qd=qd, gs=np.zeros(2), bs=np.zeros(2), pg=pg,
                vset=vset, va=np.zeros(2), f=f, t=t, r=np.array([r]), x=np.array([x]),
                b=np.array([b]), tap=np.array([tap]), status=np.ones(1, np.int32))


def closed_form_pq(v1, P, Q, R, X, b):
    """Load bus fed from a slack bus through R + jX with charging b/2 at each end.

    Kirchhoff: V1 = V2 + z (I_load + j b/2 V2), I_load = conj(S_L / V2).
    Multiplying by conj(V2):  V1 conj(V2) = (a w + c) + j (e + f w), w = |V2|^2,
    a = 1 - X b/2, c = R P + X Q, e = X P - R Q, f = R b/2, and taking modulus
    squared: v1^2 w = (a w + c)^2 + (e + f w)^2 (take the larger root)."""
    a, c, e, f = 1.0 - X * b / 2.0, R * P + X * Q, X * P - R * Q, R * b / 2.0
    A2, A1, A0 = a * a + f * f, 2 * a * c + 2 * e * f - v1 * v1, c * c + e * e
    disc = A1 * A1 - 4 * A2 * A0
    assert disc > 0
    w = (-A1 + math.sqrt(disc)) / (2 * A2)
    theta2 = -math.atan2(e + f * w, a * w + c)
    return math.sqrt(w), theta2


def closed_form_pv(v1, Pg, Vs, R, X):
    """Generator bus at |V| = Vs exporting Pg to a slack bus through R + jX.

    Real power injected at bus 2 (charging is lossless):
    P2 = g Vs^2 - Vs v1 (g cos th + bs sin th) with y = 1/z = g + j bs;
    solve alpha cos th + beta sin th = gamma, root nearest 0."""
    y = 1.0 / complex(R, X)
    g, bs = y.real, y.imag
    alpha, beta, gamma = g * Vs * v1, bs * Vs * v1, g * Vs * Vs - Pg
    Rr = math.hypot(alpha, beta)
    delta = math.atan2(beta, alpha)
    cands = [delta + math.acos(gamma / Rr), delta - math.acos(gamma / Rr)]
    cands = [math.atan2(math.sin(c), math.cos(c)) for c in cands]
    return min(cands, key=abs)


def branch_losses(case, vm, va):
    """Active and reactive power consumed by branches and shunts, from the
    physical model: series current I_s = (V_f / t - V_t) / (r + jx) through
    the ideal tap on the from side, charging b/2 at each end of the series
    element, shunt gs + j bs at the bus."""
    V = vm * np.exp(1j * va)
    pl = 0.0
    ql = 0.0
    for k in range(case.m):
        if not case.status[k]:
            continue
        t = case.tap[k] if case.tap[k] != 0 else 1.0
        vf = V[case.f[k]] / t
        vt = V[case.t[k]]
        i_s = (vf - vt) / complex(case.r[k], case.x[k])
        pl += case.r[k] * abs(i_s) ** 2
        ql += case.x[k] * abs(i_s) ** 2 - case.b[k] / 2 * (abs(vf) ** 2 + abs(vt) ** 2)
    pl += float(np.sum(case.gs * vm ** 2))
    ql -= float(np.sum(case.bs * vm ** 2))
    return pl, ql


def random_grid(n, seed, taps=True, shunts=True):
    c = gridgen.small_raw(n, seed)
    rng = np.random.default_rng(seed + 7)
    if taps:
        k = rng.integers(0, c.m)
        c.tap[k] = rng.uniform(0.9, 1.1)
        c.b[k] = 0.0
    if shunts:
        c.gs = rng.uniform(0, 0.02, n)
        c.bs = rng.uniform(-0.05, 0.05, n)
    return c


# --------------------------------------------------------------------- network

@pytest.mark.parametrize("P,Q,R,X,b", [(0.5, 0.2, 0.02, 0.1, 0.04), (1.2, 0.6, 0.01, 0.08, 0.0),
                                      (0.3, -0.1, 0.05, 0.2, 0.1)])
@pytest.mark.parametrize("method", [1, 2])
def test_two_bus_pq_closed_form(oracle, P, Q, R, X, b, method):
    v1 = 1.02
    case = two_bus("pq", P, Q, R, X, b, v1=v1)
    rc, vm, va, it, mx = oracle.power_flow(case, method, tol=1e-12, max_iter=200)
    assert rc == oracle.OK
    v2, th2 = closed_form_pq(v1, P, Q, R, X, b)
    assert abs(vm[1] - v2) < 1e-10
    assert abs(va[1] - th2) < 1e-10


@pytest.mark.parametrize("reverse", [False, True])
def test_two_bus_transformer_tap_on_from_side(oracle, reverse):
    """Ideal t:1 transformer on the from side, no charging.  Forward: slack is the
    from bus, so the series element sees v1/t.  Reverse: the load bus is the from
    bus; the load sees the series element through the ideal ratio, so the
    internal node W = V2/t carries the load and |V2| = t |W|."""
    P, Q, R, X, t, v1 = 0.8, 0.3, 0.01, 0.12, 1.04, 1.0
    case = two_bus("pq", P, Q, R, X, 0.0, tap=t, v1=v1, reverse=reverse)
    rc, vm, va, it, mx = oracle.power_flow(case, 2, tol=1e-12)
    assert rc == oracle.OK
    if not reverse:
        v2, th2 = closed_form_pq(v1 / t, P, Q, R, X, 0.0)
    else:
        w, th2 = closed_form_pq(v1, P, Q, R, X, 0.0)
        v2 = t * w
    assert abs(vm[1] - v2) < 1e-10
    assert abs(va[1] - th2) < 1e-10


@pytest.mark.parametrize("Pg,Vs,R,X", [(0.7, 1.03, 0.02, 0.15), (1.5, 1.0, 0.01, 0.05)])
@pytest.mark.parametrize("method", [1, 2])
def test_two_bus_pv_closed_form(oracle, Pg, Vs, R, X, method):
    case = two_bus("pv", Pg, Vs, R, X, 0.03, v1=1.0)
    rc, vm, va, it, mx = oracle.power_flow(case, method, tol=1e-12, max_iter=200)
    assert rc == oracle.OK
    assert vm[1] == Vs
    assert abs(va[1] - closed_form_pv(1.0, Pg, Vs, R, X)) < 1e-10


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_energy_conservation_any_voltage(oracle, seed):
    """Sum of injections equals branch + shunt consumption for ANY voltage
    vector (Tellegen), so it pins the admittance bookkeeping, not convergence."""
    case = random_grid(15, seed)
    rng = np.random.default_rng(seed)
    vm = rng.uniform(0.9, 1.1, case.n)
    va = rng.uniform(-0.3, 0.3, case.n)
    rowptr, col, G, B = oracle.ybus(case)
    P, Q = oracle.injections(rowptr, col, G, B, vm, va)
    pl, ql = branch_losses(case, vm, va)
    assert abs(P.sum() - pl) < 1e-12 * max(1.0, abs(pl)) * case.n
    assert abs(Q.sum() - ql) < 1e-12 * max(1.0, abs(ql)) * case.n


@pytest.mark.parametrize("seed", [4, 5])
def test_branch_flows_kirchhoff_and_losses(oracle, seed):
    """Branch flows at an arbitrary state: at every bus the injection from the
    admittance matrix equals the flows entering its branches plus its shunt
    consumption (Kirchhoff's current law, per bus: pins every branch's value,
    not only a sum), and the total loss equals the physical-model consumption
    of the series elements, charging and shunts."""
    case = random_grid(15, seed)
    case.status[2] = 0
    rng = np.random.default_rng(seed)
    vm = rng.uniform(0.9, 1.1, case.n)
    va = rng.uniform(-0.3, 0.3, case.n)
    rowptr, col, G, B = oracle.ybus(case)
    P, Q = oracle.injections(rowptr, col, G, B, vm, va)
    Pf, Qf, Pt, Qt, loss = oracle.branch_flows(case, vm, va)
    assert Pf[2] == Qf[2] == Pt[2] == Qt[2] == 0.0
    Pb = case.gs * vm ** 2
    Qb = -case.bs * vm ** 2
    np.add.at(Pb, case.f, Pf); np.add.at(Pb, case.t, Pt)
    np.add.at(Qb, case.f, Qf); np.add.at(Qb, case.t, Qt)
    assert np.max(np.abs(Pb - P)) < 1e-12 and np.max(np.abs(Qb - Q)) < 1e-12
    pl, _ = branch_losses(case, vm, va)
    assert abs(loss - pl) < 1e-12 * max(1.0, abs(pl))


def test_out_of_service_branch_keeps_slot(oracle):
    case = random_grid(10, 4, taps=False, shunts=False)
    rowptr, col, G, B = oracle.ybus(case)
    case2 = case.copy()
    case2.status[0] = 0
    rowptr2, col2, G2, B2 = oracle.ybus(case2)
    assert np.array_equal(rowptr, rowptr2) and np.array_equal(col, col2)
    f, t = case.f[0], case.t[0]
    p = rowptr[f] + np.searchsorted(col[rowptr[f]:rowptr[f + 1]], t)
    assert G2[p] == 0.0 and B2[p] == 0.0 and G[p] != 0.0


def test_bprime_is_xb_laplacian(oracle):
    """B' of the XB scheme: a weighted Laplacian with weights 1/x (rows sum to 0)."""
    case = random_grid(12, 5)
    rowptr, col, G, B = oracle.ybus(case)
    Bp = oracle.bprime(case, rowptr, col)
    rs = np.add.reduceat(Bp, rowptr[:-1])
    assert np.max(np.abs(rs)) < 1e-12
    k = 3
    p = rowptr[case.f[k]] + np.searchsorted(col[rowptr[case.f[k]]:rowptr[case.f[k] + 1]], case.t[k])
    assert abs(Bp[p] + 1.0 / case.x[k]) < 1e-14


# --------------------------------------------------------------------- ordering

def _golden_md():
    rows = []
    with open(os.path.join(GOLD, "md_orderings.txt")) as fh:
        for line in fh:
            if not line.strip() or line.startswith("#"):
                continue
            name, n, edges, order = [s.strip() for s in line.split("|")]
            e = [tuple(int(v) for v in s.split("-")) for s in edges.split()]
            rows.append((name, int(n), e, [int(v) for v in order.split()]))
    return rows


def _csr(n, edges):
    adj = [set() for _ in range(n)]
    for a, b in edges:
        adj[a].add(b)
        adj[b].add(a)
    p = [0]
    idx = []
    for i in range(n):
        idx.extend(sorted(adj[i]))
        p.append(len(idx))
    return np.array(p, np.int32), np.array(idx, np.int32)


@pytest.mark.parametrize("name,n,edges,order", _golden_md(), ids=[r[0] for r in _golden_md()])
def test_min_degree_hand_worked(oracle, name, n, edges, order):
    p, i = _csr(n, edges)
    assert oracle.min_degree(n, p, i).tolist() == order


@pytest.mark.parametrize("seed", range(5))
def test_min_degree_rule_replay(oracle, seed):
    """Each chosen vertex had the minimum current degree (ties: smallest index)."""
    rng = np.random.default_rng(seed)
    n = 40
    edges = set()
    while len(edges) < 70:
        a, b = rng.integers(0, n, 2)
        if a != b:
            edges.add((min(a, b), max(a, b)))
    p, idx = _csr(n, sorted(edges))
    perm = oracle.min_degree(n, p, idx)
    adj = {v: set(idx[p[v]:p[v + 1]].tolist()) for v in range(n)}
    for v in perm:
        best = min(adj, key=lambda u: (len(adj[u]), u))
        assert v == best
        nb = adj.pop(v)
        for u in nb:
            adj[u].discard(v)
            adj[u].update(nb - {u})
    assert sorted(perm.tolist()) == list(range(n))


# --------------------------------------------------------------------- symbolic

def _dense_fill(n, p, idx):
    M = np.zeros((n, n), bool)
    for i in range(n):
        M[i, idx[p[i]:p[i + 1]]] = True
    for k in range(n):
        nb = np.nonzero(M[k + 1:, k])[0] + k + 1
        for a in nb:
            M[a, nb] = True
    np.fill_diagonal(M, False)
    return M


@pytest.mark.parametrize("seed", range(4))
def test_filled_graph_vs_dense_elimination(oracle, seed):
    rng = np.random.default_rng(100 + seed)
    n = 14
    edges = set()
    while len(edges) < 22:
        a, b = rng.integers(0, n, 2)
        if a != b:
            edges.add((min(a, b), max(a, b)))
    p, idx = _csr(n, sorted(edges))
    M = _dense_fill(n, p, idx)
    for fn in (oracle.filled_graph, oracle.symbolic_etree):
        Lp, Li = fn(n, p, idx)
        for j in range(n):
            assert Li[Lp[j]:Lp[j + 1]].tolist() == np.nonzero(M[j + 1:, j])[0].__add__(j + 1).tolist()
    # elimination tree: parent[i] = min{ j > i : L_ji != 0 }
    Lp, Li = oracle.filled_graph(n, p, idx)
    parent = oracle.etree(n, Lp, Li)
    for i in range(n):
        below = np.nonzero(M[i + 1:, i])[0]
        assert parent[i] == (i + 1 + below[0] if below.size else -1)


@pytest.mark.parametrize("cfg", [0, 1])
@pytest.mark.parametrize("which", ["bp", "bpp"])
def test_two_symbolic_algorithms_agree(oracle, cfg, which):
    case = gridgen.config_raw(cfg)
    a = oracle.analyze(case, which, literal=False)
    b = oracle.analyze(case, which, literal=True)
    assert np.array_equal(a["Lp"], b["Lp"]) and np.array_equal(a["Li"], b["Li"])
    n = a["buses"].shape[0]
    parent, Lp, Li, level = a["parent"], a["Lp"], a["Li"], a["level"]
    cols = [set(Li[Lp[j]:Lp[j + 1]].tolist()) for j in range(n)]
    for j in range(n):
        if parent[j] >= 0:
            assert parent[j] > j
            assert cols[j] - {parent[j]} <= cols[parent[j]]
            assert level[parent[j]] > level[j]
    # level = 1 for leaves, 1 + max over children otherwise
    kids = [[] for _ in range(n)]
    for j in range(n):
        if parent[j] >= 0:
            kids[parent[j]].append(j)
    for j in range(n):
        assert level[j] == (1 + max(level[c] for c in kids[j]) if kids[j] else 1)


def test_table_one_levels(oracle):
    """Section II.B, Table I: leaf peeling of the 10-node elimination tree."""
    with open(os.path.join(GOLD, "table1_levels.txt")) as fh:
        lines = [ln.strip() for ln in fh if ln.strip() and not ln.startswith("#")]
    par1 = [int(v) for v in lines[0].split()[1:]]
    parent = np.array([p - 1 for p in par1], np.int32)  # 1-based -> 0-based, 0 -> -1
    expect = {}
    for ln in lines[1:]:
        lv, nodes = ln.split(":")
        for v in nodes.split():
            expect[int(v) - 1] = int(lv)
    level, nl = oracle.levels(parent)
    assert nl == 6
    assert {i: int(level[i]) for i in range(10)} == expect


# --------------------------------------------------------------------- numeric

def _dense_from_csc(n, Ap, Ai, Ax):
    A = np.zeros((n, n))
    for j in range(n):
        for p in range(Ap[j], Ap[j + 1]):
            A[Ai[p], j] += Ax[p]
    return A


@pytest.mark.parametrize("which", ["bp", "bpp"])
def test_ldlt_matches_dense_cholesky(oracle, which):
    """For SPD B' and B'', the unique LDL^T equals numpy's Cholesky rescaled."""
    case = gridgen.config_raw(0).scaled(0.0625)
    an, Lx, d, (Ap, Ai, Ax) = oracle.factor_bmatrix(case, which)
    n = an["buses"].shape[0]
    A = _dense_from_csc(n, Ap, Ai, Ax)
    Lc = np.linalg.cholesky(A)
    D_ref = np.diag(Lc) ** 2
    L_ref = Lc / np.diag(Lc)[None, :]
    assert np.max(np.abs(d - D_ref) / D_ref) < 1e-12
    Lp, Li = an["Lp"], an["Li"]
    for j in range(n):
        rows = Li[Lp[j]:Lp[j + 1]]
        assert np.allclose(Lx[Lp[j]:Lp[j + 1]], L_ref[rows, j], rtol=0, atol=1e-12)
        mask = np.ones(n, bool)
        mask[rows] = False
        mask[:j + 1] = False
        assert np.all(np.abs(L_ref[mask, j]) < 1e-12)  # outside the pattern: zero


def test_lu_and_solves_on_jacobian(oracle):
    """Unsymmetric LU without pivoting on the NR Jacobian: reconstruction and
    both solves against numpy's dense solver."""
    case = gridgen.config_raw(0).scaled(0.0625)
    rng = np.random.default_rng(0)
    vm = rng.uniform(0.95, 1.05, case.n)
    va = rng.uniform(-0.1, 0.1, case.n)
    Jd = oracle.jacobian_dense(case, vm, va)
    N = Jd.shape[0]
    # factor the dense matrix through the sparse routine with a full pattern
    Ap = np.arange(0, N * N + 1, N, dtype=np.int32)
    Ai = np.tile(np.arange(N, dtype=np.int32), N)
    Ax = Jd.T.reshape(-1).copy()
    Lp = np.array([sum(N - 1 - k for k in range(j)) for j in range(N + 1)], np.int64)
    Li = np.concatenate([np.arange(j + 1, N, dtype=np.int32) for j in range(N)])
    rc, Lx, Ux, d, bad = oracle.lu(N, Ap, Ai, Ax, Lp, Li)
    assert rc == 0
    L = np.eye(N)
    U = np.diag(d)
    for j in range(N):
        for p in range(Lp[j], Lp[j + 1]):
            L[Li[p], j] = Lx[p]
            U[j, Li[p]] = Ux[p]
    assert np.max(np.abs(L @ U - Jd)) < 1e-12 * np.max(np.abs(Jd))
    b = rng.standard_normal(N)
    for tr in (False, True):
        x = oracle.lu_solve(N, Lp, Li, Lx, Ux, d, b, transpose=tr)
        ref = np.linalg.solve(Jd.T if tr else Jd, b)
        assert np.max(np.abs(x - ref)) < 1e-10 * max(1, np.max(np.abs(ref)))


def test_jacobian_matches_finite_differences(oracle):
    """Analytic polar Jacobian vs central differences of the injections,
    including the identity rows/columns of PV voltage unknowns."""
    case = random_grid(10, 11)
    rng = np.random.default_rng(3)
    vm = rng.uniform(0.95, 1.05, case.n)
    va = rng.uniform(-0.2, 0.2, case.n)
    Jd = oracle.jacobian_dense(case, vm, va)
    rowptr, col, G, B = oracle.ybus(case)
    buses = np.nonzero(case.btype != gridgen.SLACK)[0]
    h = 1e-6
    for a, k in enumerate(buses):
        for s in (0, 1):
            if s == 1 and case.btype[k] == gridgen.PV:
                colref = np.zeros(2 * len(buses))
                colref[2 * a + 1] = 1.0
            else:
                vp, ap_ = vm.copy(), va.copy()
                vn, an_ = vm.copy(), va.copy()
                if s == 0:
                    ap_[k] += h; an_[k] -= h
                else:
                    vp[k] += h; vn[k] -= h
                Pp, Qp = oracle.injections(rowptr, col, G, B, vp, ap_)
                Pn, Qn = oracle.injections(rowptr, col, G, B, vn, an_)
                dPc, dQc = (Pp - Pn) / (2 * h), (Qp - Qn) / (2 * h)
                colref = np.zeros(2 * len(buses))
                colref[0::2] = dPc[buses]
                colref[1::2] = np.where(case.btype[buses] == gridgen.PV, 0.0, dQc[buses])
            assert np.max(np.abs(Jd[:, 2 * a + s] - colref)) < 1e-7


# --------------------------------------------------------------------- power flow

def _residual_fn(oracle, case):
    rowptr, col, G, B = oracle.ybus(case)
    nons = np.nonzero(case.btype != gridgen.SLACK)[0]
    pq = np.nonzero(case.btype == gridgen.PQ)[0]
    Psp, Qsp = case.pg - case.pd, -case.qd

    def state(z):
        vm = np.where(case.btype == gridgen.PQ, 1.0, case.vset).astype(float)
        va = case.va.astype(float).copy()
        va[nons] = z[:len(nons)]
        vm[pq] = z[len(nons):]
        return vm, va

    def F(z):
        vm, va = state(z)
        P, Q = oracle.injections(rowptr, col, G, B, vm, va)
        return np.concatenate([(Psp - P)[nons], (Qsp - Q)[pq]])

    return F, state, len(nons), len(pq)


@pytest.mark.parametrize("n,seed", [(6, 1), (9, 2), (12, 3)])
def test_power_flow_vs_generic_root_finder(oracle, n, seed):
    """Brute force: MINPACK's hybrid root finder on the same equations."""
    from scipy.optimize import root
    case = random_grid(n, seed).scaled(0.25)
    F, state, n1, n2 = _residual_fn(oracle, case)
    sol = root(F, np.concatenate([np.zeros(n1), np.ones(n2)]), tol=1e-14, method="hybr")
    assert np.max(np.abs(F(sol.x))) < 1e-10  # MINPACK may flag xtol; the residual decides
    vm_ref, va_ref = state(sol.x)
    for method in (oracle.NR, oracle.FDPF):
        rc, vm, va, it, mx = oracle.power_flow(case, method, tol=1e-12, max_iter=500)
        assert rc == oracle.OK
        assert np.max(np.abs(vm - vm_ref)) < 1e-9
        assert np.max(np.abs(va - va_ref)) < 1e-9


def test_nr_and_fdpf_same_fixed_point_and_balance(oracle):
    case = gridgen.config_raw(0).scaled(0.0625)
    rc1, vm1, va1, it1, _ = oracle.power_flow(case, oracle.NR, tol=1e-11)
    rc2, vm2, va2, it2, _ = oracle.power_flow(case, oracle.FDPF, tol=1e-11, max_iter=500)
    assert rc1 == rc2 == oracle.OK
    assert it1 <= 6  # quadratic convergence with the exact Jacobian
    assert np.max(np.abs(vm1 - vm2)) < 1e-10 and np.max(np.abs(va1 - va2)) < 1e-10
    # balance at convergence: slack output + specified injections = losses
    rowptr, col, G, B = oracle.ybus(case)
    P, Q = oracle.injections(rowptr, col, G, B, vm1, va1)
    pl, _ = branch_losses(case, vm1, va1)
    Psp = case.pg - case.pd
    nons = case.btype != gridgen.SLACK
    assert abs(P[~nons].sum() + Psp[nons].sum() - pl) < case.n * 1e-11


def test_not_converged_and_diverged_status(oracle):
    case = gridgen.config_raw(0)  # unscaled: no solution
    rc, *_ = oracle.power_flow(case, oracle.NR, tol=1e-8, max_iter=20)
    assert rc in (oracle.ERR_NOT_CONVERGED, oracle.ERR_NONFINITE)
    ok = gridgen.config_raw(0).scaled(0.0625)
    rc, *_ = oracle.power_flow(ok, oracle.NR, tol=1e-8, max_iter=1)
    assert rc == oracle.ERR_NOT_CONVERGED


# --------------------------------------------------------------------- adjoint

def test_adjoint_vs_central_differences(oracle):
    """dJ/dPsp and dJ/dQsp from the transposed solve vs central differences
    (h = 1e-6) of J at re-solved power flows, plus a dense brute-force adjoint."""
    case = gridgen.config_raw(0).scaled(0.0625)
    rc, vm, va, _, _ = oracle.power_flow(case, oracle.NR, tol=1e-13, max_iter=30)
    assert rc == oracle.OK
    dJdP, dJdQ, J0 = oracle.adjoint(case, vm, va)
    assert abs(J0 - oracle.objective(case, vm, va)) < 1e-12
    h = 1e-6
    rng = np.random.default_rng(5)
    nons = np.nonzero(case.btype != gridgen.SLACK)[0]
    pq = np.nonzero(case.btype == gridgen.PQ)[0]
    picks = [("P", i) for i in rng.choice(nons, 6, replace=False)] + \
            [("Q", i) for i in rng.choice(pq, 6, replace=False)]
    fd_all = []
    for kind, i in picks:
        vals = []
        for sgn in (1, -1):
            c = case.copy()
            if kind == "P":
                c.pd[i] -= sgn * h  # +h net injection
            else:
                c.qd[i] -= sgn * h
            rc2, vm2, va2, _, _ = oracle.power_flow(c, oracle.NR, tol=1e-13, max_iter=30,
                                                    vm0=vm, va0=va)
            assert rc2 == oracle.OK
            vals.append(oracle.objective(c, vm2, va2))
        fd_all.append((vals[0] - vals[1]) / (2 * h))
    fd_all = np.array(fd_all)
    scale = 1e-3 * np.max(np.abs(fd_all))
    for (kind, i), fd in zip(picks, fd_all):
        g = dJdP[i] if kind == "P" else dJdQ[i]
        assert abs(g - fd) <= 1e-6 * max(abs(fd), scale) + 1e-9, (kind, i, g, fd)
    pv = case.btype == gridgen.PV
    assert np.all(dJdQ[pv] == 0.0)
    # dense brute force: lambda = J^{-T} grad_x J with grad by differences
    Jd = oracle.jacobian_dense(case, vm, va)
    gx = np.zeros(Jd.shape[0])
    for a, k in enumerate(nons):
        for s in (0, 1):
            if s == 1 and case.btype[k] != gridgen.PQ:
                continue
            vp, ap_, vn, an_ = vm.copy(), va.copy(), vm.copy(), va.copy()
            if s == 0:
                ap_[k] += 1e-6; an_[k] -= 1e-6
            else:
                vp[k] += 1e-6; vn[k] -= 1e-6
            gx[2 * a + s] = (oracle.objective(case, vp, ap_) - oracle.objective(case, vn, an_)) / 2e-6
    lam = np.linalg.solve(Jd.T, gx)
    assert np.max(np.abs(lam[0::2] - dJdP[nons])) < 1e-6 * max(1.0, np.max(np.abs(lam)))
    assert np.max(np.abs(lam[1::2][case.btype[nons] == gridgen.PQ] - dJdQ[pq])) < \
        1e-6 * max(1.0, np.max(np.abs(lam)))
