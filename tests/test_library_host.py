"""Host-side checks of libgbpf that need no GPU: the library loads and exports
every entry point of include/gbpf.h, input validation, and the symbolic
analysis (ordering, fill, elimination tree, levels) bit-exact against the
oracle's independent implementation."""
import ctypes as C

import numpy as np
import pytest

from paper_1811_02512_gb300 import gbpf, gridgen


@pytest.fixture(scope="module")
def lib():
    from paper_1811_02512_gb300 import build
    build.build()
    return gbpf.load()


def test_exports_every_header_symbol(lib):
    names = gbpf.header_functions()
    assert len(names) >= 12
    for nm in names:
        assert hasattr(lib, nm), nm
        assert C.cast(getattr(lib, nm), C.c_void_p).value


def _tables(case):
    return case.bus_table(), case.branch_table()


def test_create_rejects_bad_tables(lib):
    case = gridgen.config_raw(0)
    bus, br = _tables(case)
    bad = br.copy(); bad["to"][3] = case.n + 5
    with pytest.raises(gbpf.PFError) as e:
        gbpf.pf_create(bus, bad)
    assert e.value.status == gbpf.PF_ERR_ARG
    bad = br.copy(); bad["x"][0] = np.nan
    with pytest.raises(gbpf.PFError) as e:
        gbpf.pf_create(bus, bad)
    assert e.value.status == gbpf.PF_ERR_ARG
    b2 = bus.copy(); b2["type"][5] = gridgen.SLACK
    with pytest.raises(gbpf.PFError) as e:
        gbpf.pf_create(b2, br)
    assert e.value.status == gbpf.PF_ERR_ARG
    # island: take every branch of one leaf bus out of service
    deg = np.bincount(np.concatenate([case.f, case.t]), minlength=case.n)
    leaf = int(np.nonzero(deg == 1)[0][0])
    bad = br.copy(); bad["status"][(case.f == leaf) | (case.t == leaf)] = 0
    with pytest.raises(gbpf.PFError) as e:
        gbpf.pf_create(bus, bad)
    assert e.value.status == gbpf.PF_ERR_ISLAND


@pytest.mark.parametrize("cfg", [0, 1, 3])
def test_symbolic_bit_exact_vs_oracle(lib, oracle, cfg):
    case = gridgen.config_raw(cfg)
    g = gbpf.Grid(case)
    for which, name in ((gbpf.PF_MAT_BP, "bp"), (gbpf.PF_MAT_BPP, "bpp")):
        ref = oracle.analyze(case, name)
        got = g.symbolic(which)
        assert g.info.n[which] == ref["buses"].shape[0]
        assert np.array_equal(got["perm"], ref["perm"])
        assert np.array_equal(got["Lp"], ref["Lp"])
        assert np.array_equal(got["Li"], ref["Li"])
        assert np.array_equal(got["parent"], ref["parent"])
        assert np.array_equal(got["level"], ref["level"])
        assert g.info.nlevels[which] == ref["nlevels"]
    g.close()


@pytest.mark.parametrize("seed", range(6))
def test_symbolic_small_random_grids(lib, oracle, seed):
    case = gridgen.small_raw(8 + 7 * seed, 300 + seed)
    g = gbpf.Grid(case)
    for which, name in ((gbpf.PF_MAT_BP, "bp"), (gbpf.PF_MAT_BPP, "bpp")):
        ref = oracle.analyze(case, name, literal=True)
        got = g.symbolic(which)
        for k in ("perm", "Lp", "Li", "parent", "level"):
            assert np.array_equal(got[k], ref[k]), k
    g.close()


@pytest.mark.parametrize("which_case", ["cfg0", "cfg1", "small0", "small1", "small2"])
def test_symbolic_sizes_vs_oracle_pattern(lib, oracle, which_case):
    """pf_analyze's sizes against the oracle's filled pattern: strict-lower
    nonzeros, the longest column, and the scalar updates of one numeric
    factor -- for every target (i, c) of L (the diagonal included), one per
    column k < c with L(c,k) and L(i,k) nonzero -- which sizes the factor's
    gather lists."""
    if which_case.startswith("cfg"):
        case = gridgen.config_raw(int(which_case[3:]))
    else:
        s = int(which_case[5:])
        case = gridgen.small_raw(12 + 9 * s, 500 + s)
    g = gbpf.Grid(case)
    for which, name in ((gbpf.PF_MAT_BP, "bp"), (gbpf.PF_MAT_BPP, "bpp")):
        an = oracle.analyze(case, name)
        Lp, Li = an["Lp"], an["Li"]
        n = Lp.shape[0] - 1
        cols = [set(Li[Lp[j]:Lp[j + 1]].tolist()) for j in range(n)]
        rows = [[] for _ in range(n)]
        for j in range(n):
            for i in Li[Lp[j]:Lp[j + 1]]:
                rows[i].append(j)
        assert g.info.nnz_l[which] == Lp[-1]
        assert g.info.max_col[which] == (int(np.max(np.diff(Lp))) if n else 0)
        assert g.info.nupdates[which] == sum(1 + len(cols[c] & cols[k]) for c in range(n) for k in rows[c])
    g.close()


def _tail_tables(lib, g, which):
    f = lib.gbpf_debug_tail_tables
    f.restype = C.c_int
    f.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_int]
    sizes = np.zeros(8, np.int32)
    assert f(g.ctx, which, sizes.ctypes.data, None, 0, None, 0) == 0
    n, t0, ntl, ng, ne, kmax, tmax, nterm = (int(x) for x in sizes)
    tlev = np.zeros((max(1, 2 * ntl), 4), np.int32)
    tinfo = np.zeros((max(1, ng), 4), np.int32)
    assert f(g.ctx, which, sizes.ctypes.data, tlev.ctypes.data, 2 * ntl, tinfo.ctypes.data, ng) == 0
    return (dict(n=n, t0=t0, ntl=ntl, ng=ng, ne=ne, kmax=kmax, tmax=tmax, nterm=nterm),
            tlev[:2 * ntl], tinfo[:ng])


def _oracle_tail_levels(oracle, case, name, narrow=16):
    """Per level of the narrow top of the elimination tree (the run of
    top levels with at most `narrow` columns), from the oracle's own
    symbolic analysis: (columns, targets = entries + diagonals of its
    columns, update terms L(i,k) L(c,k) D(k) with k also in the top run)."""
    an = oracle.analyze(case, name)
    Lp, Li, lev, nl = an["Lp"], an["Li"], an["level"], an["nlevels"]
    n = lev.shape[0]
    cnt = np.bincount(lev, minlength=nl + 1)
    lt = nl
    while lt >= 1 and cnt[lt] <= narrow:
        lt -= 1
    cols = [set(Li[Lp[j]:Lp[j + 1]].tolist()) for j in range(n)]
    rows = [[] for _ in range(n)]
    for j in range(n):
        for i in Li[Lp[j]:Lp[j + 1]]:
            rows[i].append(j)
    out = []
    for L in range(lt + 1, nl + 1):
        cs = np.nonzero(lev == L)[0]
        ntgt = sum(len(cols[c]) + 1 for c in cs)
        nterm = sum(1 + len(cols[c] & cols[k]) for c in cs for k in rows[c] if lev[k] > lt)
        out.append((len(cs), ntgt, nterm))
    return out


@pytest.mark.parametrize("cfg", [0, 1])
def test_tail_factor_tables_vs_oracle(lib, oracle, cfg):
    """The tail factor's level table and target descriptors, built by
    pf_analyze on the host, against counts taken from the oracle's symbolic
    analysis (numbering-independent per level), plus the structural
    invariants the kernel relies on: levels, terms and columns tile their
    ranges, every tail L entry has exactly one target, every tail column
    exactly one diagonal target inside its own level."""
    case = gridgen.config_raw(cfg)
    g = gbpf.Grid(case)
    for which, name in ((gbpf.PF_MAT_BP, "bp"), (gbpf.PF_MAT_BPP, "bpp")):
        sz, tlev, tinfo = _tail_tables(lib, g, which)
        ref = _oracle_tail_levels(oracle, case, name)
        assert sz["ntl"] == len(ref) > 0
        nt = sum(r[0] for r in ref)
        assert sz["n"] - sz["t0"] == nt
        assert sz["ng"] == sum(r[1] for r in ref) and sz["ne"] == sz["ng"] - nt
        assert sz["nterm"] == sum(r[2] for r in ref)
        assert sz["kmax"] == max(r[1] for r in ref) and sz["tmax"] == max(r[2] for r in ref)
        ntask, tasks, tipos = _tail_tasks(lib, g, which, sz["ng"])
        seen_diag = np.zeros(nt, np.int32)
        seen_entry = np.zeros(sz["ne"], np.int32)
        for li, (ncol, ntgt, nterm) in enumerate(ref):
            kb, ke, tb, te = tlev[2 * li]
            cb, ce, q0, q1 = tlev[2 * li + 1]
            assert (ke - kb, te - tb, ce - cb) == (ntgt, nterm, ncol), li
            if li + 1 < len(ref):
                assert tlev[2 * li + 2][0] == ke and tlev[2 * li + 2][2] == te
                assert tlev[2 * li + 3][0] == ce and tlev[2 * li + 3][2] == q1
            info = tinfo[kb:ke]
            # the level's targets (reordered) hold term ranges that tile the level's terms
            rng = info[np.lexsort((info[:, 1], info[:, 0]))]  # by start, empty ranges first
            assert rng[0, 0] == 0 and rng[-1, 1] == te - tb
            assert np.array_equal(rng[1:, 0], rng[:-1, 1]) and np.all(info[:, 1] >= info[:, 0])
            # tipos maps the level's targets one to one onto its positions
            assert np.array_equal(np.sort(tipos[kb:ke]), np.arange(kb, ke))
            # warp tasks: 32 / G positions of one G each, every position once;
            # G the smallest power of two leaving one term to a lane
            # (at most 32); tasks listed by decreasing terms per lane
            cover = np.zeros(ke - kb, np.int32)
            costs = []
            for x, y, G, _ in tasks[q0:q1]:
                assert G in (1, 2, 4, 8, 16, 32) and 1 <= y <= 32 // G
                cover[x:x + y] += 1
                cnt = info[x:x + y, 1] - info[x:x + y, 0]
                assert np.all((G == 32) | (cnt <= G)) and np.all((G == 1) | (cnt > G // 2))
                costs.append(int(np.max((cnt + G - 1) // G)))
            assert np.all(cover == 1), li
            assert costs == sorted(costs, reverse=True)
            assert np.all((info[:, 3] >= cb) & (info[:, 3] < ce))
            d = info[info[:, 2] < 0]
            assert np.all(d[:, 2] == -1) and d.shape[0] == ncol
            np.add.at(seen_diag, d[:, 3], 1)
            np.add.at(seen_entry, info[info[:, 2] >= 0, 2], 1)
        assert tlev[0][0] == 0 and tlev[0][2] == 0 and tlev[1][0] == 0
        assert tlev[-2][1] == sz["ng"] and tlev[-2][3] == sz["nterm"] and tlev[-1][1] == nt
        assert np.all(seen_diag == 1) and np.all(seen_entry == 1)
    g.close()


def _tail_tasks(lib, g, which, ng):
    f = lib.gbpf_debug_tail_tasks
    f.restype = C.c_int
    f.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
    n = np.zeros(1, np.int32)
    assert f(g.ctx, which, n.ctypes.data, None, None, 0) == 0
    ntask = int(n[0])
    tasks = np.zeros((max(1, ntask), 4), np.int32)
    tipos = np.zeros(max(1, ng), np.int32)
    assert f(g.ctx, which, n.ctypes.data, tasks.ctypes.data, tipos.ctypes.data, max(4 * ntask, ng, 1)) == 0
    return ntask, tasks[:ntask], tipos[:ng]


def _scatter_schedules(lib, g, which):
    f = lib.gbpf_debug_scatter_schedules
    f.restype = C.c_int
    f.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
    sizes = np.zeros(6, np.int32)
    assert f(g.ctx, which, sizes.ctypes.data, None, None, None, None, 0) == 0
    t0, ntl, nkf, nif, nkb, nib = (int(x) for x in sizes)
    cap = max(1, nkf, nif, nkb, nib)
    arrs = [np.zeros(cap, np.int32) for _ in range(4)]
    assert f(g.ctx, which, sizes.ctypes.data, *[a.ctypes.data for a in arrs], cap) == 0
    SKf, SIf, SKb, SIb = arrs[0][:nkf], arrs[1][:nif], arrs[2][:nkb], arrs[3][:nib]
    return t0, ntl, SKf, SIf, SKb, SIb


def _oracle_scatter_counts(oracle, case, name, narrow=16):
    """Per level of the narrow top run (bottom first): the forward updates
    (strict-lower entries of the level's columns) and the backward updates
    (strict-lower entries of the level's rows that lie in the top run)."""
    an = oracle.analyze(case, name)
    Lp, Li, lev, nl = an["Lp"], an["Li"], an["level"], an["nlevels"]
    n = lev.shape[0]
    cnt = np.bincount(lev, minlength=nl + 1)
    lt = nl
    while lt >= 1 and cnt[lt] <= narrow:
        lt -= 1
    rowcnt = np.zeros(n, np.int64)
    for j in range(n):
        for i in Li[Lp[j]:Lp[j + 1]]:
            if lev[j] > lt:
                rowcnt[i] += 1
    out = []
    for L in range(lt + 1, nl + 1):
        cs = np.nonzero(lev == L)[0]
        out.append((int(sum(Lp[c + 1] - Lp[c] for c in cs)), int(rowcnt[cs].sum())))
    return out


@pytest.mark.parametrize("cfg", [0, 1])
def test_scatter_tail_schedules_vs_oracle(lib, oracle, cfg):
    """The one-warp scatter schedules of the narrow top (forward and back
    substitution): per level, one slot per update, in the lane that owns the
    target row (row - t0 = lane mod 32), sources inside the level, targets
    below (forward) or above (backward) them, no update twice, and as many
    updates as the oracle's pattern has for that level."""
    case = gridgen.config_raw(cfg)
    g = gbpf.Grid(case)
    for which, name in ((gbpf.PF_MAT_BP, "bp"), (gbpf.PF_MAT_BPP, "bpp")):
        t0, ntl, SKf, SIf, SKb, SIb = _scatter_schedules(lib, g, which)
        _, tlev, _ = _tail_tables(lib, g, which)
        ref = _oracle_scatter_counts(oracle, case, name)
        assert ntl == len(ref) > 0
        for SK, SI, fwd in ((SKf, SIf, True), (SKb, SIb, False)):
            assert SK.shape[0] == ntl + 1 and SK[0] == 0 and SI.shape[0] == 32 * SK[-1]
            for li in range(ntl):
                lv = li if fwd else ntl - 1 - li  # the backward sweep walks the levels top down
                cb, ce = tlev[2 * lv + 1][:2]
                slots = SI[32 * SK[li]:32 * SK[li + 1]]
                lanes = np.arange(slots.shape[0]) % 32
                used = slots >= 0
                tgt, src = slots[used] & 0xFFFF, slots[used] >> 16
                assert np.all(slots[~used] == -1)
                assert np.all(tgt % 32 == lanes[used])
                assert np.all((src >= cb) & (src < ce))
                assert np.all(tgt > src) if fwd else np.all(tgt < src)
                assert np.unique(tgt * 65536 + src).shape[0] == tgt.shape[0]
                assert tgt.shape[0] == ref[lv][0 if fwd else 1], (name, fwd, li)
    g.close()


def _pieces(lib, g, which, lst):
    f = lib.gbpf_debug_pieces
    f.restype = C.c_int
    f.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_int]
    cnt = C.c_int(0)
    assert f(g.ctx, which, lst, C.byref(cnt), None, 0) == 0
    out = np.zeros(max(1, 8 * cnt.value), np.int32)
    assert f(g.ctx, which, lst, C.byref(cnt), out.ctypes.data, out.shape[0]) == 0
    return out[:8 * cnt.value].reshape(-1, 8)


@pytest.mark.parametrize("cfg", [0, 1, 3])
def test_sweep_pieces_tile_levels(lib, oracle, cfg):
    """The staged sweeps' piece lists (forward over CSR rows in ascending
    levels, backward over CSC columns in descending levels): levels in sweep
    order, every row in exactly one piece (or one run of partial-row pieces
    with contiguous entry ranges), pieces of modes 0/1/3 inside one level,
    mode 2 only over narrow levels, per-level entry counts equal to the
    oracle's pattern, and run_end marking the end of each single-warp run."""
    case = gridgen.config_raw(cfg)
    g = gbpf.Grid(case)
    for which, name in ((gbpf.PF_MAT_BP, "bp"), (gbpf.PF_MAT_BPP, "bpp")):
        an = oracle.analyze(case, name)
        Lp, Li, lev, nl = an["Lp"], an["Li"], an["level"], an["nlevels"]
        n = lev.shape[0]
        sizes = np.bincount(lev, minlength=nl + 1)[1:]
        lvl_ptr = np.concatenate([[0], np.cumsum(sizes)])
        colcnt = np.diff(Lp)
        rowcnt = np.bincount(Li, minlength=n) if Li.shape[0] else np.zeros(n, np.int64)
        for lst, fwd in ((0, True), (1, False)):
            per_lev = np.bincount(lev - 1, weights=rowcnt if fwd else colcnt, minlength=nl)
            P = _pieces(lib, g, which, lst)
            covered = np.zeros(n, np.int32)
            got = np.zeros(nl, np.int64)
            last_l = -1 if fwd else nl
            for k, (r0, r1, e0, e1, mode, run_end, l0, l1) in enumerate(P):
                assert mode in (0, 1, 2, 3) and e1 >= e0 and r1 > r0
                if mode == 2:
                    assert r0 == lvl_ptr[l0] and r1 == lvl_ptr[l1 + 1]
                    assert np.all(sizes[l0:l1 + 1] <= 16)
                else:
                    assert l0 == l1 and lvl_ptr[l0] <= r0 < r1 <= lvl_ptr[l0 + 1]
                assert (l0 >= last_l) if fwd else (l1 <= last_l)
                last_l = l1 if fwd else l0
                got[l0] += e1 - e0  # a mode-2 piece's entries are summed over its levels below
                if mode == 2:
                    got[l0] -= e1 - e0
                    assert e1 - e0 == per_lev[l0:l1 + 1].sum()
                    got[l0:l1 + 1] += per_lev[l0:l1 + 1].astype(np.int64)
                if mode == 3:
                    assert r1 == r0 + 1
                    first = not (k > 0 and P[k - 1][4] == 3 and P[k - 1][0] == r0)
                    if not first:
                        assert e0 == P[k - 1][3]
                    covered[r0] += 1 if first else 0
                else:
                    covered[r0:r1] += 1
                single = 2 <= mode <= 4
                if single:
                    nxt = k + 1
                    while nxt < P.shape[0] and 2 <= P[nxt][4] <= 4:
                        nxt += 1
                    assert run_end == nxt
            assert np.all(covered == 1)
            assert np.array_equal(got, per_lev.astype(np.int64)), (name, fwd)
    g.close()


@pytest.mark.parametrize("cfg", [0, 1])
def test_sweep_pieces_with_scatter_tail(lib, oracle, cfg):
    """The sweeps used when the narrow top runs as a scatter tail.  Forward:
    pieces over the levels below the tail (rows [0, t0) once, ascending),
    then block-wide pieces over the tail rows' entries in columns below the
    tail (their count from the oracle's pattern), then scatter pieces tiling
    the forward schedule.  Backward: pieces over the tail rows (inverse
    diagonal), scatter pieces tiling the backward schedule, then the levels
    below the tail, descending."""
    case = gridgen.config_raw(cfg)
    g = gbpf.Grid(case)
    for which, name in ((gbpf.PF_MAT_BP, "bp"), (gbpf.PF_MAT_BPP, "bpp")):
        an = oracle.analyze(case, name)
        Lp, Li, lev, nl = an["Lp"], an["Li"], an["level"], an["nlevels"]
        n = lev.shape[0]
        t0, ntl, SKf, _, SKb, _ = _scatter_schedules(lib, g, which)
        lt = nl - ntl  # levels 1..lt (oracle numbering) lie below the tail
        cols = np.repeat(np.arange(n), np.diff(Lp))
        below = int(np.sum((lev[Li] > lt) & (lev[cols] <= lt)))  # tail rows' entries left of t0
        for lst, fwd in ((2, True), (3, False)):
            P = _pieces(lib, g, which, lst)
            modes = P[:, 4]
            wide = np.isin(modes, (0, 1, 2, 3))
            if fwd:
                order = [(0, 1, 2, 3), (5,), (4,)]
            else:
                order = [(6,), (4,), (0, 1, 2, 3)]
            groups = []
            for ms in order:
                k = 0 if not groups else groups[-1][1]
                e = k
                while e < P.shape[0] and P[e][4] in ms:
                    e += 1
                groups.append((k, e))
            assert groups[-1][1] == P.shape[0], (name, fwd)
            covered = np.zeros(n, np.int32)
            for r0, r1 in P[wide][:, :2]:
                if r1 > r0:
                    covered[r0:r1] += 1
            for (r0, r1, _e0, _e1, mode, *_r) in P[wide]:
                if mode == 3:
                    covered[r0] -= 1
            for k in np.nonzero(wide & (modes == 3))[0]:
                if not (k > 0 and P[k - 1][4] == 3 and P[k - 1][0] == P[k][0]):
                    covered[P[k][0]] += 1
            assert np.all(covered[:t0] == 1) and np.all(covered[t0:] == 0)
            k0, k1 = groups[1] if fwd else groups[0]
            rows = P[k0:k1]
            assert rows[0][0] == t0 and rows[-1][1] == n and np.array_equal(rows[1:, 0], rows[:-1, 1])
            if fwd:
                assert int(np.sum(rows[:, 3] - rows[:, 2])) == below
            k0, k1 = groups[2] if fwd else groups[1]
            sc = P[k0:k1]
            SK = SKf if fwd else SKb
            assert sc[0][2] == 0 and sc[-1][3] == 32 * SK[-1] and np.array_equal(sc[1:, 2], sc[:-1, 3])
    g.close()


@pytest.mark.parametrize("cfg", [0, 1])
def test_admittance_tables_and_mismatch_orders(lib, cfg):
    """The per-entry admittance tables list, for every off-diagonal Ybus entry
    (i, j) exactly once, the branches between buses i and j in ascending
    order (out-of-service ones included: the kernel skips them); the
    mismatch's thread orders are permutations that keep every bus in its
    window of 1,024 (mis_ord) or its cluster slice (mis_ord_cl) and order
    each window or slice by Ybus row length, stably."""
    case = gridgen.config_raw(cfg)
    g = gbpf.Grid(case)
    f = lib.gbpf_debug_net_tables
    f.restype = C.c_int
    f.argtypes = [C.c_void_p, C.c_void_p] + [C.c_void_p] * 6 + [C.c_longlong]
    sz = np.zeros(4, np.int64)
    assert f(g.ctx, sz.ctypes.data, None, None, None, None, None, None, 0) == 0
    nbus, nnz, noff, nref = (int(v) for v in sz)
    cap = max(nbus + 1, nnz, 4 * noff, nref)
    rowptr, col, yoff, ybr, mo, mc = (np.zeros(cap, np.int32) for _ in range(6))
    assert f(g.ctx, sz.ctypes.data, rowptr.ctypes.data, col.ctypes.data, yoff.ctypes.data, ybr.ctypes.data,
             mo.ctypes.data, mc.ctypes.data, cap) == 0
    rowptr, col, ybr, mo, mc = rowptr[:nbus + 1], col[:nnz], ybr[:nref], mo[:nbus], mc[:nbus]
    yoff = yoff[:4 * noff].reshape(noff, 4)
    assert noff == nnz - nbus
    row = np.repeat(np.arange(nbus), np.diff(rowptr))
    offd = np.nonzero(col != row)[0]
    assert np.array_equal(np.sort(yoff[:, 0]), offd)
    between = {}
    for e, (a, b) in enumerate(zip(case.f, case.t)):
        between.setdefault((int(a), int(b)), []).append(e)
        between.setdefault((int(b), int(a)), []).append(e)
    for p, lo, hi, _ in yoff:
        assert list(ybr[lo:hi]) == sorted(between.get((int(row[p]), int(col[p])), []))
    length = np.diff(rowptr)
    assert np.array_equal(np.sort(mo), np.arange(nbus)) and np.array_equal(np.sort(mc), np.arange(nbus))
    for i0 in range(0, nbus, 1024):
        w = mo[i0:i0 + 1024]
        assert w.min() >= i0 and w.max() < i0 + 1024
        assert np.all(np.diff(length[w]) >= 0)
    sl = (nbus + 15) // 16
    for r in range(16):
        w = mc[r * sl:(r + 1) * sl]
        if w.size:
            assert w.min() >= r * sl and w.max() < (r + 1) * sl
            assert np.all(np.diff(length[w]) >= 0)
            eq = np.diff(length[w]) == 0
            assert np.all(np.diff(w)[eq] > 0)  # stable: equal lengths keep bus order
    g.close()


def _gather(lib, g, which):
    f = lib.gbpf_debug_gather
    f.restype = C.c_int
    f.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                  C.c_longlong]
    sizes = np.zeros(3, np.int64)
    assert f(g.ctx, which, sizes.ctypes.data, None, None, None, None, 0) == 0
    n, nnz, nterm = (int(x) for x in sizes)
    Cp = np.zeros(n + 1, np.int32)
    Cr = np.zeros(max(1, nnz), np.int32)
    gp = np.zeros(n + nnz + 1, np.int32)
    gl = np.zeros((max(1, nterm), 4), np.int32)
    cap = max(n + nnz + 1, 4 * nterm)
    assert f(g.ctx, which, sizes.ctypes.data, Cp.ctypes.data, Cr.ctypes.data, gp.ctypes.data,
             gl.ctypes.data, cap) == 0
    return n, nnz, Cp, Cr[:nnz], gp, gl[:nterm]


@pytest.mark.parametrize("cfg", [0, 1])
def test_factor_gather_lists(lib, oracle, cfg):
    """The dependency-driven factor's gather lists: for every target (i, c)
    of L in level order (the diagonal first), one term per column k < c with
    L(c,k) and L(i,k) nonzero -- both positions inside column k, one in row i
    and one in row c, no k twice, none missing -- and per level as many terms
    as the oracle's pattern gives."""
    case = gridgen.config_raw(cfg)
    g = gbpf.Grid(case)
    for which, name in ((gbpf.PF_MAT_BP, "bp"), (gbpf.PF_MAT_BPP, "bpp")):
        n, nnz, Cp, Cr, gp, gl = _gather(lib, g, which)
        assert g.info.nupdates[which] == gl.shape[0] == gp[-1]
        tcol = np.repeat(np.arange(n), np.diff(Cp) + 1)
        toff = np.arange(n + nnz) - (Cp[tcol] + tcol)
        trow = tcol.copy()
        off = toff > 0
        trow[off] = Cr[Cp[tcol[off]] + toff[off] - 1]
        tt = np.repeat(np.arange(n + nnz), np.diff(gp))
        x, y, z = gl[:, 0], gl[:, 1], gl[:, 2]
        pcol = np.repeat(np.arange(n), np.diff(Cp))
        assert np.all(pcol[x] == z) and np.all(pcol[y] == z)
        assert np.all(Cr[y] == tcol[tt]) and np.all(Cr[x] == trow[tt])
        assert np.all(z < tcol[tt])
        assert np.unique(tt.astype(np.int64) * n + z).shape[0] == tt.shape[0]
        rowset = [set() for _ in range(n)]
        for k in range(n):
            for i in Cr[Cp[k]:Cp[k + 1]]:
                rowset[i].add(k)
        want = np.array([len(rowset[c]) if i == c else len(rowset[c] & rowset[i])
                         for i, c in zip(trow, tcol)])
        assert np.array_equal(np.diff(gp), want)
        an = oracle.analyze(case, name)
        Lp, Li, lev, nl = an["Lp"], an["Li"], an["level"], an["nlevels"]
        cols = [set(Li[Lp[j]:Lp[j + 1]].tolist()) for j in range(n)]
        rows = [[] for _ in range(n)]
        for j in range(n):
            for i in Li[Lp[j]:Lp[j + 1]]:
                rows[i].append(j)
        ref = np.zeros(nl, np.int64)
        for c in range(n):
            ref[lev[c] - 1] += sum(1 + len(cols[c] & cols[k]) for k in rows[c])
        lvl_ptr = np.concatenate([[0], np.cumsum(np.bincount(lev, minlength=nl + 1)[1:])])
        got = np.array([gp[Cp[lvl_ptr[l + 1]] + lvl_ptr[l + 1]] - gp[Cp[lvl_ptr[l]] + lvl_ptr[l]]
                        for l in range(nl)])
        assert np.array_equal(got, ref)
    g.close()


def _csr(lib, g, which):
    f = lib.gbpf_debug_csr
    f.restype = C.c_int
    f.argtypes = [C.c_void_p, C.c_int, C.c_void_p] + [C.c_void_p] * 7 + [C.c_int]
    sizes = np.zeros(4, np.int32)
    assert f(g.ctx, which, sizes.ctypes.data, *([None] * 7), 0) == 0
    n, nnz, offLc, na = (int(x) for x in sizes)
    arrs = [np.zeros(max(1, k), np.int32) for k in (n + 1, nnz, nnz, nnz, n + 1, na, na)]
    cap = max(n + 1, nnz, na)
    assert f(g.ctx, which, sizes.ctypes.data, *[a.ctypes.data for a in arrs], cap) == 0
    Fp, Fc, Fpos, Cpos, Ap, Aj, Apos = arrs
    return offLc, Fp, Fc[:nnz], Fpos[:nnz], Cpos[:nnz], Ap, Aj[:na], Apos[:na]


@pytest.mark.parametrize("cfg", [0, 1])
def test_csr_maps_and_residual_pattern(lib, oracle, cfg):
    """The CSR copy of L's pattern (strict lower, ascending columns) maps one
    to one onto the CSC pattern (Fpos, with Cpos its inverse), and the
    off-diagonal pattern of A used by the FP64 residuals is symmetric, points
    at the L slot of each entry, and has the degree sequence of the oracle's
    bus graph of the matrix."""
    case = gridgen.config_raw(cfg)
    g = gbpf.Grid(case)
    for which, name in ((gbpf.PF_MAT_BP, "bp"), (gbpf.PF_MAT_BPP, "bpp")):
        n, nnz, Cp, Cr, _, _ = _gather(lib, g, which)
        offLc, Fp, Fc, Fpos, Cpos, Ap, Aj, Apos = _csr(lib, g, which)
        pcol = np.repeat(np.arange(n), np.diff(Cp))
        rowF = np.repeat(np.arange(n), np.diff(Fp))
        assert Fp[-1] == nnz and np.all(Fc < rowF)
        same = rowF[1:] == rowF[:-1]
        assert np.all(Fc[1:][same] > Fc[:-1][same])
        assert np.all(pcol[Fpos] == Fc) and np.all(Cr[Fpos] == rowF)
        assert np.array_equal(np.sort(Fpos), np.arange(nnz)) and np.all(Cpos[Fpos] == np.arange(nnz))
        rowA = np.repeat(np.arange(n), np.diff(Ap))
        pa = Apos - offLc
        assert np.all(Aj != rowA)
        assert np.all(pcol[pa] == np.minimum(rowA, Aj)) and np.all(Cr[pa] == np.maximum(rowA, Aj))
        sa = rowA[1:] == rowA[:-1]
        assert np.all(Aj[1:][sa] > Aj[:-1][sa])
        fwd = set(zip(rowA.tolist(), Aj.tolist()))
        assert fwd == set(zip(Aj.tolist(), rowA.tolist()))
        _, ogp, _ = oracle.local_graph(case, name)
        assert np.array_equal(np.sort(np.diff(Ap)), np.sort(np.diff(ogp)))
    g.close()


def test_outage_keeps_pattern(lib):
    case = gridgen.config_raw(0)
    c2 = case.copy()
    c2.status[7] = 0
    a, b = gbpf.Grid(case), gbpf.Grid(c2)
    for w in (0, 1):
        sa, sb = a.symbolic(w), b.symbolic(w)
        assert np.array_equal(sa["Li"], sb["Li"]) and np.array_equal(sa["perm"], sb["perm"])
    a.close(); b.close()


def test_device_calls_fail_cleanly_without_gpu(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    g = gbpf.Grid(gridgen.config_raw(0))
    with pytest.raises(gbpf.PFError) as e:
        g.set_cases(1)
    assert e.value.status in (gbpf.PF_ERR_CUDA, gbpf.PF_ERR_OOM)
    g.close()


def test_tuning_fields_validated(lib):
    case = gridgen.config_raw(0)
    ctx = gbpf.pf_create(*_tables(case))
    gbpf.pf_analyze(ctx)
    assert gbpf.pf_get_tuning(ctx) == {"engine": 0, "cluster": 0, "factor": 0, "tail": 0, "outage": 0,
                                       "threads": 0, "ms": 0.0}
    gbpf.pf_set_tuning(ctx, engine=gbpf.PF_ENGINE_LANES, cluster=8, factor=1, tail=2, outage=2, threads=256)
    t = gbpf.pf_get_tuning(ctx)
    assert (t["engine"], t["cluster"], t["factor"], t["tail"], t["outage"], t["threads"]) == \
        (gbpf.PF_ENGINE_LANES, 8, 1, 2, 2, 256)
    for bad in ({"cluster": 3}, {"factor": 3}, {"tail": -1}, {"engine": 7}, {"outage": 3}, {"threads": 64},
                {"threads": 1024}):
        with pytest.raises(gbpf.PFError) as e:
            gbpf.pf_set_tuning(ctx, **bad)
        assert e.value.status == gbpf.PF_ERR_ARG
    gbpf.pf_destroy(ctx)


def test_pack_create_validates(lib):
    case = gridgen.config_raw(0)
    ctx = gbpf.pf_create(*_tables(case))
    arr = (C.c_void_p * 2)(ctx, ctx)
    h = C.c_void_p()
    assert lib.pf_pack_create(arr, 2, C.byref(h)) == gbpf.PF_ERR_STATE  # not analysed
    gbpf.pf_analyze(ctx)
    assert lib.pf_pack_create(arr, 2, C.byref(h)) == gbpf.PF_ERR_ARG  # repeated
    assert lib.pf_pack_create(arr, 0, C.byref(h)) == gbpf.PF_ERR_ARG
    assert lib.pf_pack_create(arr, 1, C.byref(h)) == gbpf.PF_OK
    lib.pf_pack_destroy(h)
    gbpf.pf_destroy(ctx)


def _cluster_program(lib, g, which):
    f = lib.gbpf_debug_cluster
    f.restype = C.c_int
    f.argtypes = [C.c_void_p, C.c_int] + [C.c_void_p] * 12 + [C.c_longlong]
    sz = np.zeros(12, np.int64)
    assert f(g.ctx, which, sz.ctypes.data, *([None] * 11), 0) == 0
    Cc, nt, nstep, nx, ntask, nref, nval = (int(v) for v in sz[:7])
    cap = max(4 * ntask, 4 * nval, 4 * nstep, nref, g.nbus, nt, Cc + 1, 1)
    arrs = [np.zeros(cap, np.int32) for _ in range(11)]
    assert f(g.ctx, which, sz.ctypes.data, *(a.ctypes.data for a in arrs), cap) == 0
    tasks, tptr, steps, refs, eptr, vsrc, vptr, sptr, rhsref, xref, tnode = arrs
    return dict(C=Cc, nt=nt, nx=nx, smem=int(sz[7]), offDi=int(sz[8]), offLc=int(sz[9]),
                offLr=int(sz[10]), ok=int(sz[11]),
                tasks=tasks[:4 * ntask].reshape(-1, 4), tptr=tptr[:Cc + 1],
                steps=steps[:4 * nstep].reshape(-1, 4), sptr=sptr[:Cc + 1], refs=refs[:nref],
                eptr=eptr[:Cc + 1], vsrc=vsrc[:4 * nval].reshape(-1, 4), vptr=vptr[:Cc + 1],
                rhsref=rhsref[:g.nbus], xref=xref[:g.nbus], tnode=tnode[:nt])


def _cluster_groups(lib, g, which):
    f = lib.gbpf_debug_cluster_groups
    f.restype = C.c_int
    f.argtypes = [C.c_void_p, C.c_int] + [C.c_void_p] * 6 + [C.c_longlong]
    sz = np.zeros(6, np.int32)
    assert f(g.ctx, which, sz.ctypes.data, *([None] * 5), 0) == 0
    group, ncol, ngw, ngm, nupd, nterm = (int(v) for v in sz)
    cap = max(4 * max(ncol, nupd, ngw + ngm), 2 * nterm, ngm + 1, 1)
    arrs = [np.zeros(cap, np.int32) for _ in range(5)]
    assert f(g.ctx, which, sz.ctypes.data, *(a.ctypes.data for a in arrs), cap) == 0
    gw_col, gw_upd, gm_ptr, gm_term, gv_info = arrs
    return dict(group=group, n_gw=ngw, n_gm=ngm, gw_col=gw_col[:4 * ncol].reshape(-1, 4),
                gw_upd=gw_upd[:4 * nupd].reshape(-1, 4), gm_ptr=gm_ptr[:ngm + 1],
                gm_term=gm_term[:2 * nterm].reshape(-1, 2), gv_info=gv_info[:4 * (ngw + ngm)].reshape(-1, 4))


@pytest.mark.parametrize("cfg,group", [(0, 0), (0, 2), (1, 0), (1, 1), (1, 4), (1, 6)])
def test_cluster_program_solves_like_oracle(lib, oracle, cfg, group):
    """The cluster engine's substitution program, run on the CPU with the
    device's synchronisation: the oracle's factor is placed in the library's
    level-order layout and the top set's inverse is formed densely from it.
    Between two cluster barriers a CTA runs its steps in order; a step reads
    its own CTA's words as they stood before the step and every other CTA's
    words as they stood at the last cluster barrier, so a dependence that the
    barriers do not cover would read a stale value.  The result equals the
    oracle's LDL^T solve; the top set is closed under parents, every CTA
    passes the same number of cluster barriers, every index stays inside its
    buffer, and the programs of the 10,000-bus grid fit one CTA's shared
    memory.  The subtree levels run `group` at a time (0: the default)
    through the groups' inverses, whose values are formed here from the
    host's value programs as the device forms them."""
    import scipy.sparse as sp
    case = gridgen.config(cfg)
    g = gbpf.Grid(case)
    gbpf.pf_set_tuning(g.ctx, engine=gbpf.PF_ENGINE_CLUSTER, cluster=group)
    rng = np.random.default_rng(7 + cfg)
    for which, name in ((gbpf.PF_MAT_BP, "bp"), (gbpf.PF_MAT_BPP, "bpp")):
        P = _cluster_program(lib, g, which)
        assert P["ok"] == 1
        an, Lx, d, _ = oracle.factor_bmatrix(case, name)
        n = an["buses"].shape[0]
        lev = an["level"]
        order = np.lexsort((np.arange(n), lev))  # level order: (level, step)
        new = np.empty(n, np.int64)
        new[order] = np.arange(n)
        cols = np.repeat(np.arange(n), np.diff(an["Lp"]))
        L = sp.csc_matrix((Lx, (new[an["Li"]], new[cols])), shape=(n, n))
        L.sort_indices()
        dl = np.empty(n)
        dl[new] = d
        nnz = L.nnz
        F = np.zeros(P["offLr"] + nnz + 64)
        F[:n] = dl
        F[P["offDi"]:P["offDi"] + n] = 1.0 / dl
        F[P["offLc"]:P["offLc"] + nnz] = L.data
        Lr = L.tocsr()
        Lr.sort_indices()
        F[P["offLr"]:P["offLr"] + nnz] = Lr.data
        nt, T = P["nt"], P["tnode"]
        Wd = np.zeros(max(1, nt * nt))
        if nt:
            inT = np.zeros(n, bool)
            inT[T] = True
            parent = np.array([L[:, j].indices[0] if L.indptr[j + 1] > L.indptr[j] else -1 for j in range(n)])
            assert np.all((parent[T] < 0) | inT[np.maximum(parent[T], 0)])  # closed under parents
            W = np.linalg.inv(L[T][:, T].toarray() + np.eye(nt))
            Wd = W.flatten()  # W(it, jt) at it * nt + jt
        # the grouped subtree steps' values, as the device forms them from the
        # host's lists (the solve below checks them against the oracle)
        GR = _cluster_groups(lib, g, which)
        ngw, ngm = GR["n_gw"], GR["n_gm"]
        GV = np.zeros(max(1, ngw + ngm))
        for ub, ue, base, Pn in GR["gw_col"]:
            w = np.zeros(8)
            w[0] = 1.0
            for p_, q_, fpos, _ in GR["gw_upd"][ub:ue]:
                assert 0 <= p_ < q_ < Pn <= 8
                w[q_] -= F[fpos] * w[p_]
            GV[base:base + Pn - 1] = w[1:Pn]
        for e in range(ngm):
            acc = 0.0
            for wi, fpos in GR["gm_term"][GR["gm_ptr"][e]:GR["gm_ptr"][e + 1]]:
                assert wi < ngw and fpos < P["offLr"] + nnz
                acc += (1.0 if wi < 0 else GV[wi]) * F[fpos]
            GV[ngw + e] = acc
        # what every value is: an inverse entry W(a, j) has a in j's group
        # above j; a combined entry's k lies below (forward) or above
        # (backward) its row's group
        lev0 = np.empty(n, np.int64)
        lev0[new] = lev - 1  # level of every level-order row, leaves 0
        inT0 = np.zeros(n, bool)
        inT0[P["tnode"]] = True
        gsz = GR["group"]
        for typ, i, jk, _ in GR["gv_info"]:
            assert not inT0[i]
            if typ == 0:
                assert lev0[i] // gsz == lev0[jk] // gsz and lev0[i] > lev0[jk]
            elif typ == 1:
                assert lev0[jk] // gsz < lev0[i] // gsz
            else:
                assert inT0[jk] or lev0[jk] // gsz > lev0[i] // gsz
        vs = P["vsrc"]
        vals = np.empty(vs.shape[0])
        kinds = [vs[:, 0] == q for q in range(6)]
        assert np.all(np.logical_or.reduce(kinds))
        assert np.all(vs[kinds[0], 1] < P["offLr"] + nnz) and np.all(vs[kinds[1] | kinds[2], 1] < max(1, nt * nt))
        assert np.all(vs[kinds[3] | kinds[4], 1] < max(1, ngw)) and np.all(vs[kinds[5], 1] < ngw + max(1, ngm))
        vals[kinds[0]] = F[vs[kinds[0], 1]]
        vals[kinds[1]] = -Wd[vs[kinds[1], 1]]
        vals[kinds[2]] = -Wd[vs[kinds[2], 1]] * F[vs[kinds[2], 2]]
        vals[kinds[3]] = -GV[vs[kinds[3], 1]]
        vals[kinds[4]] = -GV[vs[kinds[4], 1]] * F[vs[kinds[4], 2]]
        vals[kinds[5]] = GV[vs[kinds[5], 1]]
        Cc, nx = P["C"], P["nx"]
        # every index the device program uses stays inside its buffers
        assert np.all((P["refs"] >> 16) < Cc) and np.all((P["refs"] & 0xffff) < max(1, nx))
        prog = []
        for r in range(Cc):
            T_ = P["tasks"][P["tptr"][r]:P["tptr"][r + 1]]
            S_ = P["steps"][P["sptr"][r]:P["sptr"][r + 1]]
            ne = P["eptr"][r + 1] - P["eptr"][r]
            nv = P["vptr"][r + 1] - P["vptr"][r]
            assert T_[-1][3] == ne and np.all(np.diff(T_[:, 3]) >= 0)
            assert np.all(T_[:-1, 0] < nx) and np.all(T_[:-1, 1] < nx) and np.all(T_[:-1, 2] < nv)
            assert np.all(S_[:, 0] <= S_[:, 1]) and np.all(S_[:, 1] <= T_.shape[0] - 1)
            assert np.all(S_[1:, 0] == S_[:-1, 1]) and np.all(np.isin(S_[:, 2], [1, 2, 4, 8, 16, 32]))
            prog.append((T_, S_, P["refs"][P["eptr"][r]:P["eptr"][r + 1]], vals[P["vptr"][r]:P["vptr"][r + 1]]))
        nbar = {int(np.sum(p[1][:, 3])) for p in prog}
        assert len(nbar) == 1
        b_loc = rng.standard_normal(n)
        X = np.zeros((Cc, max(1, nx)))
        rr = P["rhsref"][an["buses"]]
        assert np.all(rr >= 0) and np.all(P["rhsref"][np.setdiff1d(np.arange(g.nbus), an["buses"])] == -1)
        X[rr >> 16, rr & 0xffff] = b_loc
        pos = [0] * Cc
        for _ in range(nbar.pop()):
            snapC = X.copy()
            for r in range(Cc):
                T_, S_, R, V = prog[r]
                while True:
                    tb, te, G, cl = S_[pos[r]]
                    pos[r] += 1
                    snapR = X[r].copy()
                    for t in range(tb, te):
                        out, inn, dg, e0 = T_[t]
                        e1 = T_[t + 1][3]
                        rf = R[e0:e1]
                        o, w = rf >> 16, rf & 0xffff
                        xs = np.where(o == r, snapR[w], snapC[o, w])
                        X[r, out] = snapR[inn] * (V[dg] if dg >= 0 else 1.0) - np.dot(V[e0:e1], xs)
                    if cl:
                        break
        assert all(pos[r] == prog[r][1].shape[0] for r in range(Cc))
        xr = P["xref"][an["buses"]]
        assert np.all(xr >= 0)
        x = X[xr >> 16, xr & 0xffff]
        xs = oracle.lu_solve(n, an["Lp"], an["Li"], Lx, Lx * d[cols], d, b_loc[an["perm"]])
        ref = np.empty(n)
        ref[an["perm"]] = xs
        assert np.max(np.abs(x - ref)) <= 1e-11 * max(1.0, np.max(np.abs(ref))), (name, np.max(np.abs(x - ref)))
        if cfg == 1 and group <= 4:  # larger groups may outgrow a CTA (the engine then does not apply)
            assert P["smem"] + 4096 <= 232448, P["smem"]
    g.close()


def _tail_inverse(lib, g, which):
    f = lib.gbpf_debug_tail_inverse
    f.restype = C.c_int
    f.argtypes = [C.c_void_p, C.c_int, C.c_void_p] + [C.c_void_p] * 10 + [C.c_int]
    sizes = np.zeros(10, np.int32)
    assert f(g.ctx, which, sizes.ctypes.data, *([None] * 10), 0) == 0
    n, t0, nt, nfc, nbc, nfe, nbe, npf3, npb3, ne = (int(x) for x in sizes)
    shapes = (nt, nt + 1, 2 * nfc, nfe, nfe, nt + 1, 2 * nbc, nbe, nbe, nbe)
    arrs = [np.zeros(max(1, k), np.int32) for k in shapes]
    assert f(g.ctx, which, sizes.ctypes.data, *[a.ctypes.data for a in arrs], max(shapes + (1,))) == 0
    par, fr, fc, fj, fs, br, bc, bj, bs, bd = (a[:k] for a, k in zip(arrs, shapes))
    return dict(n=n, t0=t0, nt=nt, nfc=nfc, nbc=nbc, nfe=nfe, nbe=nbe, npf3=npf3, npb3=npb3, ne=ne), \
        par, fr, fc.reshape(-1, 2), fj, fs, br, bc.reshape(-1, 2), bj, bs, bd


@pytest.mark.parametrize("cfg", [0, 1])
def test_tail_inverse_gathers(lib, oracle, cfg):
    """Tail form 3 (the narrow top solved through W = L_TT^-1): the parents
    within the top are the elimination tree's (first row of each column of
    L, from the CSR pattern); the forward gather of row i lists exactly its
    descendants and the backward gather exactly its ancestors, each pair once,
    chunked in order; the dense-W sources and diagonal indices point at
    (ancestor, descendant); the counts agree with the oracle's own symbolic
    analysis (numbering-independent: the number of ancestor/descendant pairs
    in the top run of narrow levels); and the chunk partial sums with the
    top's vector fit the staging ring."""
    case = gridgen.config_raw(cfg)
    g = gbpf.Grid(case)
    for which, name in ((gbpf.PF_MAT_BP, "bp"), (gbpf.PF_MAT_BPP, "bpp")):
        sz, par, fr, fc, fj, fs, br, bc, bj, bs, bd = _tail_inverse(lib, g, which)
        nt, t0 = sz["nt"], sz["t0"]
        assert nt > 0 and sz["npf3"] > 0 and sz["npb3"] > 0
        offLc, Fp, Fc, *_ = _csr(lib, g, which)
        n = sz["n"]
        first_row = np.full(n, -1)
        for i in range(n - 1, -1, -1):  # the smallest row of each column
            first_row[Fc[Fp[i]:Fp[i + 1]]] = i
        for it in range(nt):
            p = first_row[t0 + it]
            assert par[it] == (p - t0 if p >= 0 else -1)
        anc = [[] for _ in range(nt)]
        for it in range(nt):
            a = par[it]
            while a >= 0:
                anc[it].append(a)
                a = par[a]
        desc = [[] for _ in range(nt)]
        for j in range(nt):
            for a in anc[j]:
                desc[a].append(j)
        assert np.all(np.diff(fr) >= 0) and fr[0] == 0 and fr[-1] == sz["nfc"]
        assert np.all(np.diff(br) >= 0) and br[0] == 0 and br[-1] == sz["nbc"]
        for rows, rp, ch, cj, src, fwd in ((desc, fr, fc, fj, fs, True), (anc, br, bc, bj, bs, False)):
            assert ch[0, 0] == 0 if len(ch) else True
            for it in range(nt):
                got = []
                for k in range(rp[it], rp[it + 1]):
                    a, b = ch[k]
                    assert 0 < b - a <= 4096 and (k == 0 or a == ch[k - 1, 1])
                    got.extend(cj[a:b].tolist())
                    for e in range(a, b):
                        assert src[e] == (it * nt + cj[e] if fwd else cj[e] * nt + it)
                assert got == sorted(rows[it])
        assert np.array_equal(bd, t0 + bj)
        # the oracle's count: ancestor/descendant pairs inside its top run
        an = oracle.analyze(case, name)
        Lp, Li, lev, nl = an["Lp"], an["Li"], an["level"], an["nlevels"]
        cnt = np.bincount(lev, minlength=nl + 1)
        lt = nl
        while lt >= 1 and cnt[lt] <= 16:
            lt -= 1
        parent = np.array([Li[Lp[j]] if Lp[j + 1] > Lp[j] else -1 for j in range(lev.shape[0])])
        pairs = 0
        for j in np.nonzero(lev > lt)[0]:
            a = parent[j]
            while a >= 0:
                pairs += 1
                a = parent[a]
        assert sz["nfe"] == sz["nbe"] == pairs
        assert (nt + max(sz["nfc"], sz["nbc"])) * 8 <= 4 * 8192
    g.close()
