"""Seeded synthetic power-grid generator (input synthesis only).

This module builds the bus and branch tables that both the CUDA library and
the CPU oracle consume.  It contains none of the power-flow arithmetic (no
admittance matrix, no mismatch, no factorisation): it only draws topologies,
impedances, loads and scenarios from seeded distributions, so that tests and
benchmarks feed identical inputs to both sides.

Grids follow the shape of the practical systems of the paper's case study
(Section IV: roughly 1.2-1.35 branches per bus, about 15 % generator buses):

* ``config0``: 120 buses placed uniformly in the unit square, a random
  spanning tree (each bus, in seeded random order, attaches to its nearest
  already placed bus) plus 60 extra nearest-neighbour branches.
* ``delaunay_grid(n, seed)``: buses placed uniformly in the unit square, the
  Delaunay triangulation pruned to a uniform-random-weight spanning tree plus
  uniformly drawn further Delaunay edges until ``m = round(1.35 n)``;
  12 % PV buses and 2 % transformer branches (tap on the from side,
  ``tap ~ U(0.95, 1.05)``, no charging).

Electrical data (all per unit): ``r ~ U(0.005, 0.05)``, ``x = r * U(3, 10)``,
line charging ``b ~ U(0, 0.05)``; bus 0 is the slack at 1.0 p.u. / 0 rad;
PV buses have ``P ~ U(0.5, 2.0)`` and ``V ~ U(1.0, 1.05)``; PQ buses carry a
load ``P ~ U(0.1, 1.0)`` at a lagging power factor ``pf ~ U(0.9, 0.98)``
(``Q = P tan(acos pf)``).  PV generation is rescaled so that total generation
equals total load, and every injection is then multiplied by the grid's
loading factor ``lam`` (the largest ``2^-k`` at which a flat-start
Newton-Raphson converges within 10 iterations, halved), which is looked up
from ``data/loading_factors.json``.
"""
from __future__ import annotations

import json
import math
import os
from dataclasses import dataclass, field

import numpy as np

PQ, PV, SLACK = 1, 2, 3
SEED_BASE = 1811025120

_HERE = os.path.dirname(os.path.abspath(__file__))
LOADING_FACTOR_FILE = os.path.join(_HERE, "data", "loading_factors.json")

# numpy structured dtypes laid out exactly like the C-ABI structs pf_bus /
# pf_branch (natural C alignment).
BUS_DTYPE = np.dtype(
    [("id", "<i4"), ("type", "<i4"), ("pd", "<f8"), ("qd", "<f8"), ("gs", "<f8"),
     ("bs", "<f8"), ("pg", "<f8"), ("vset", "<f8"), ("va", "<f8")], align=True)
BRANCH_DTYPE = np.dtype(
    [("from", "<i4"), ("to", "<i4"), ("r", "<f8"), ("x", "<f8"), ("b", "<f8"),
     ("tap", "<f8"), ("status", "<i4")], align=True)


@dataclass
class Case:
    """One grid: bus and branch tables in per unit plus provenance."""
    name: str
    btype: np.ndarray      # int32 [n]  1 PQ, 2 PV, 3 slack
    pd: np.ndarray         # float64 [n] load P
    qd: np.ndarray         # float64 [n] load Q
    gs: np.ndarray         # float64 [n] shunt conductance
    bs: np.ndarray         # float64 [n] shunt susceptance
    pg: np.ndarray         # float64 [n] generation P (PV and slack)
    vset: np.ndarray       # float64 [n] voltage set-point (PV, slack); 1.0 elsewhere
    va: np.ndarray         # float64 [n] slack angle (0 elsewhere)
    f: np.ndarray          # int32 [m] from bus
    t: np.ndarray          # int32 [m] to bus
    r: np.ndarray          # float64 [m]
    x: np.ndarray          # float64 [m]
    b: np.ndarray          # float64 [m] total line charging
    tap: np.ndarray        # float64 [m] off-nominal ratio on the from side (1 = none)
    status: np.ndarray     # int32 [m] 1 in service
    lam: float = 1.0
    seed: int = 0
    xy: np.ndarray | None = field(default=None, repr=False)

    @property
    def n(self) -> int:
        return int(self.btype.shape[0])

    @property
    def m(self) -> int:
        return int(self.f.shape[0])

    def bus_table(self) -> np.ndarray:
        a = np.zeros(self.n, dtype=BUS_DTYPE)
        a["id"] = np.arange(self.n, dtype=np.int32)
        a["type"], a["pd"], a["qd"] = self.btype, self.pd, self.qd
        a["gs"], a["bs"], a["pg"] = self.gs, self.bs, self.pg
        a["vset"], a["va"] = self.vset, self.va
        return a

    def branch_table(self) -> np.ndarray:
        a = np.zeros(self.m, dtype=BRANCH_DTYPE)
        a["from"], a["to"] = self.f, self.t
        a["r"], a["x"], a["b"], a["tap"] = self.r, self.x, self.b, self.tap
        a["status"] = self.status
        return a

    def copy(self) -> "Case":
        kw = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in self.__dict__.items()}
        return Case(**kw)

    def scaled(self, lam: float) -> "Case":
        """Same grid with every P and Q injection multiplied by ``lam``."""
        c = self.copy()
        c.pd = c.pd * lam
        c.qd = c.qd * lam
        c.pg = c.pg * lam
        c.lam = self.lam * lam
        return c

    def scaled_network(self, lam: float) -> "Case":
        """``scaled`` plus the other sources of flow at a flat start scaled
        towards the flat profile: line charging b -> lam b, off-nominal taps
        t -> 1 + lam (t - 1), PV and slack set-points v -> 1 + lam (v - 1)."""
        c = self.scaled(lam)
        c.b = c.b * lam
        c.tap = np.where(c.tap != 0.0, 1.0 + lam * (c.tap - 1.0), c.tap)
        gen = c.btype != PQ
        c.vset = np.where(gen, 1.0 + lam * (c.vset - 1.0), c.vset)
        return c


# --------------------------------------------------------------------------- topology

def _nearest_tree_plus_nn(rng, xy, n_extra):
    """Random spanning tree by nearest attachment plus ``n_extra`` NN branches."""
    n = xy.shape[0]
    order = rng.permutation(n)
    placed = [int(order[0])]
    edges = set()
    for v in order[1:]:
        v = int(v)
        d = np.sum((xy[placed] - xy[v]) ** 2, axis=1)
        u = placed[int(np.argmin(d))]
        edges.add((min(u, v), max(u, v)))
        placed.append(v)
    extra_src = rng.permutation(n)[:n_extra]
    for v in extra_src:
        v = int(v)
        d = np.sum((xy - xy[v]) ** 2, axis=1)
        d[v] = np.inf
        for u in np.argsort(d, kind="stable"):
            u = int(u)
            e = (min(u, v), max(u, v))
            if e not in edges:
                edges.add(e)
                break
    return sorted(edges)


def _delaunay_edges(xy):
    from scipy.spatial import Delaunay
    tri = Delaunay(xy)
    s = tri.simplices
    e = np.concatenate([s[:, [0, 1]], s[:, [1, 2]], s[:, [0, 2]]], axis=0)
    e = np.sort(e, axis=1)
    e = np.unique(e, axis=0)
    return e.astype(np.int64)


class _DSU:
    def __init__(self, n):
        self.p = np.arange(n)

    def find(self, a):
        p = self.p
        root = a
        while p[root] != root:
            root = p[root]
        while p[a] != root:
            p[a], a = root, p[a]
        return root

    def union(self, a, b):
        ra, rb = self.find(a), self.find(b)
        if ra == rb:
            return False
        self.p[ra] = rb
        return True


def _pruned_delaunay(rng, xy, m_target):
    """Uniform-random-weight spanning tree of the Delaunay graph plus random extra edges."""
    n = xy.shape[0]
    e = _delaunay_edges(xy)
    w = rng.random(e.shape[0])
    order = np.argsort(w, kind="stable")
    dsu = _DSU(n)
    in_tree = np.zeros(e.shape[0], dtype=bool)
    for k in order:
        if dsu.union(int(e[k, 0]), int(e[k, 1])):
            in_tree[k] = True
    rest = np.nonzero(~in_tree)[0]
    rest = rest[rng.permutation(rest.shape[0])]
    n_extra = max(0, min(m_target - (n - 1), rest.shape[0]))
    keep = np.concatenate([np.nonzero(in_tree)[0], rest[:n_extra]])
    keep.sort()
    return [(int(a), int(b)) for a, b in e[keep]]


def bridges(n, f, t, status=None):
    """Indices of bridge branches (iterative Tarjan low-link), input selection only."""
    m = len(f)
    if status is None:
        status = np.ones(m, dtype=np.int32)
    adj = [[] for _ in range(n)]
    for k in range(m):
        if status[k]:
            adj[int(f[k])].append((int(t[k]), k))
            adj[int(t[k])].append((int(f[k]), k))
    disc = [-1] * n
    low = [0] * n
    out = []
    timer = 0
    for root in range(n):
        if disc[root] >= 0:
            continue
        disc[root] = low[root] = timer
        timer += 1
        stack = [(root, -1, iter(adj[root]))]
        while stack:
            v, pe, it = stack[-1]
            advanced = False
            for (u, k) in it:
                if k == pe:
                    continue
                if disc[u] < 0:
                    disc[u] = low[u] = timer
                    timer += 1
                    stack.append((u, k, iter(adj[u])))
                    advanced = True
                    break
                low[v] = min(low[v], disc[u])
            if not advanced:
                stack.pop()
                if stack:
                    p = stack[-1][0]
                    low[p] = min(low[p], low[v])
                    if low[v] > disc[p]:
                        out.append(pe)
    return sorted(out)


# --------------------------------------------------------------------------- electrical data

def _electrical(rng, name, seed, xy, edges, n_pv, transformer_frac):
    n = xy.shape[0]
    m = len(edges)
    f = np.array([a for a, _ in edges], dtype=np.int32)
    t = np.array([b for _, b in edges], dtype=np.int32)
    r = rng.uniform(0.005, 0.05, m)
    x = r * rng.uniform(3.0, 10.0, m)
    b = rng.uniform(0.0, 0.05, m)
    tap = np.ones(m)
    n_tr = int(round(transformer_frac * m))
    if n_tr:
        tr = np.sort(rng.permutation(m)[:n_tr])
        tap[tr] = rng.uniform(0.95, 1.05, n_tr)
        b[tr] = 0.0
    btype = np.full(n, PQ, dtype=np.int32)
    btype[0] = SLACK
    pv = np.sort(1 + rng.permutation(n - 1)[:n_pv])
    btype[pv] = PV
    pd = np.zeros(n)
    qd = np.zeros(n)
    pg = np.zeros(n)
    vset = np.ones(n)
    pq = np.nonzero(btype == PQ)[0]
    pd[pq] = rng.uniform(0.1, 1.0, pq.shape[0])
    pf = rng.uniform(0.9, 0.98, pq.shape[0])
    qd[pq] = pd[pq] * np.tan(np.arccos(pf))
    pg[pv] = rng.uniform(0.5, 2.0, pv.shape[0])
    vset[pv] = rng.uniform(1.0, 1.05, pv.shape[0])
    # generation balanced against load: the slack then supplies only the losses
    pg[pv] *= pd.sum() / pg[pv].sum()
    c = Case(name=name, btype=btype, pd=pd, qd=qd, gs=np.zeros(n), bs=np.zeros(n), pg=pg,
             vset=vset, va=np.zeros(n), f=f, t=t, r=r, x=x, b=b, tap=tap,
             status=np.ones(m, dtype=np.int32), lam=1.0, seed=seed, xy=xy)
    return c


def config0_raw(seed=SEED_BASE + 0):
    """120-bus grid: nearest-attachment spanning tree + 60 NN branches, 20 PV, 99 PQ."""
    rng = np.random.default_rng(seed)
    xy = rng.random((120, 2))
    edges = _nearest_tree_plus_nn(rng, xy, 60)
    return _electrical(rng, "grid120", seed, xy, edges, n_pv=20, transformer_frac=0.0)


def delaunay_raw(n, seed, name=None):
    """n-bus pruned-Delaunay grid, average degree 2.7, 12 % PV, 2 % transformers."""
    rng = np.random.default_rng(seed)
    xy = rng.random((n, 2))
    edges = _pruned_delaunay(rng, xy, int(round(1.35 * n)))
    n_pv = int(round(0.12 * n))
    return _electrical(rng, name or f"delaunay{n}", seed, xy, edges, n_pv=n_pv,
                       transformer_frac=0.02)


def small_raw(n, seed, extra=None):
    """Tiny test grid (n >= 3) of the config-0 family for brute-force checks."""
    rng = np.random.default_rng(seed)
    xy = rng.random((n, 2))
    edges = _nearest_tree_plus_nn(rng, xy, extra if extra is not None else max(1, n // 3))
    return _electrical(rng, f"small{n}_{seed}", seed, xy, edges, n_pv=max(1, n // 5),
                       transformer_frac=0.0)


# --------------------------------------------------------------------------- loading factor

def load_loading_factors():
    if not os.path.exists(LOADING_FACTOR_FILE):
        return {}
    with open(LOADING_FACTOR_FILE) as fh:
        return json.load(fh)


def loading_key(case: Case) -> str:
    return f"{case.name}:{case.seed}:{case.n}:{case.m}"


def network_scaled(name: str) -> bool:
    """Grids of the uneven multi-grid batch take their loading factor on the
    whole network (Case.scaled_network); the others on the injections only."""
    return name.startswith("multigrid")


def with_loading_factor(raw: Case, table=None) -> Case:
    table = load_loading_factors() if table is None else table
    key = loading_key(raw)
    if key not in table:
        raise KeyError(f"no stored loading factor for {key}; run oracle/find_loading_factors.py")
    lam = float(table[key])
    return raw.scaled_network(lam) if network_scaled(raw.name) else raw.scaled(lam)


# --------------------------------------------------------------------------- named workloads

CONFIG4_NGRID = 256


def config_raw(k: int):
    """Raw (unscaled) grid(s) of workload k."""
    if k == 0:
        return config0_raw()
    if k in (1, 2):
        return delaunay_raw(10000, SEED_BASE + 1, name="delaunay10k")
    if k == 3:
        return delaunay_raw(20000, SEED_BASE + 3, name="delaunay20k")
    if k == 4:
        return [delaunay_raw(nk, sk, name=f"multigrid{g}") for g, (nk, sk) in enumerate(config4_sizes())]
    raise ValueError(k)


def config4_sizes():
    rng = np.random.default_rng(SEED_BASE + 4)
    u = rng.uniform(math.log(2000.0), math.log(80000.0), CONFIG4_NGRID)
    sizes = np.rint(np.exp(u)).astype(np.int64)
    seeds = [int(SEED_BASE + 4) * 1000 + g for g in range(CONFIG4_NGRID)]
    return list(zip([int(s) for s in sizes], seeds))


def config(k: int):
    """Workload k with its stored loading factor applied."""
    raw = config_raw(k)
    table = load_loading_factors()
    if isinstance(raw, list):
        return [with_loading_factor(r, table) for r in raw]
    return with_loading_factor(raw, table)


@dataclass
class Scenarios:
    """Per-case modifications of one base grid (batched contingency / load study)."""
    load_scale: np.ndarray   # float64 [ncase, n] multiplier of pd/qd at PQ buses
    outage: np.ndarray       # int32 [ncase]  branch index taken out, -1 = none

    @property
    def ncase(self):
        return int(self.outage.shape[0])


def scenarios(base: Case, n_load=512, n_outage=512, seed=SEED_BASE + 2) -> Scenarios:
    """``n_load`` load cases (per-bus PQ scale ~ N(1, 0.08)) then ``n_outage``
    single-branch outages of distinct non-bridge branches."""
    rng = np.random.default_rng(seed)
    n = base.n
    ls = np.ones((n_load + n_outage, n))
    pq = base.btype == PQ
    draw = rng.normal(1.0, 0.08, (n_load, n))
    ls[:n_load][:, pq] = draw[:, pq]
    br = set(bridges(n, base.f, base.t, base.status))
    cand = np.array([k for k in range(base.m) if k not in br and base.status[k]], dtype=np.int64)
    pick = cand[rng.permutation(cand.shape[0])[:n_outage]]
    out = np.full(n_load + n_outage, -1, dtype=np.int32)
    out[n_load:] = pick.astype(np.int32)
    return Scenarios(load_scale=ls, outage=out)


def apply_scenario(base: Case, sc: Scenarios, c: int) -> Case:
    """Case c of a scenario set as a stand-alone grid (used by the CPU side)."""
    g = base.copy()
    g.pd = g.pd * sc.load_scale[c]
    g.qd = g.qd * sc.load_scale[c]
    if sc.outage[c] >= 0:
        g.status = g.status.copy()
        g.status[sc.outage[c]] = 0
    return g
