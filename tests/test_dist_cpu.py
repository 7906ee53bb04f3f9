"""The multi-rank path of bench.py on CPU: gloo ranks on 127.0.0.1.

A batch shards by case (paper_1811_02512_gb300.shard): every rank solves its
own contiguous slice of the cases and the results are gathered at the end.
Here each rank runs the oracle as a host stand-in for the per-case solve;
the gathered results must equal a single process's, every case must be
counted exactly once, and the job time is the slowest rank's."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _batch():
    from paper_1811_02512_gb300 import gridgen
    base = gridgen.config(0)
    return base, gridgen.scenarios(base, n_load=4, n_outage=3, seed=9)  # 7 cases: an uneven split


def _solve(base, sc, c):
    from oracle import oracle as O
    from paper_1811_02512_gb300 import gridgen
    rc, vm, va, _, _ = O.power_flow(gridgen.apply_scenario(base, sc, c), O.FDPF, tol=1e-10)
    return rc, vm, va


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1811_02512_gb300 import shard
    base, sc = _batch()
    lo, hi = shard.case_range(rank, world, sc.ncase)
    vm = torch.zeros((hi - lo, base.n), dtype=torch.float64)
    va = torch.zeros_like(vm)
    st = torch.zeros(hi - lo, dtype=torch.int32)
    for c in range(lo, hi):
        rc, v, a = _solve(base, sc, c)
        vm[c - lo] = torch.from_numpy(v)
        va[c - lo] = torch.from_numpy(a)
        st[c - lo] = rc
    vm_all, va_all, st_all = shard.gather_cases(vm, va, st, sc.ncase, rank, world)
    ms, solves, value = shard.job_throughput(100.0 + 50.0 * rank, int((st == 0).sum()), world, "cpu")
    out.put((rank, lo, hi, vm_all.numpy(), va_all.numpy(), st_all.numpy(), ms, solves, value))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_cases_partitioned_gathered_and_counted_once(oracle, world):
    import torch.multiprocessing as mp
    base, sc = _batch()
    ref = [_solve(base, sc, c) for c in range(sc.ncase)]
    assert all(r[0] == oracle.OK for r in ref)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # the slices tile the cases exactly once
    assert [r[1] for r in res] == sorted(r[1] for r in res) and res[0][1] == 0 and res[-1][2] == sc.ncase
    assert all(res[k][2] == res[k + 1][1] for k in range(world - 1))
    for rank, lo, hi, vm, va, st, ms, solves, value in res:
        assert vm.shape == (sc.ncase, base.n)
        for c in range(sc.ncase):
            assert np.array_equal(vm[c], ref[c][1]) and np.array_equal(va[c], ref[c][2])
        assert np.all(st == 0)
        assert ms == 100.0 + 50.0 * (world - 1)
        assert solves == sc.ncase  # distinct cases, none counted twice
        assert abs(value - sc.ncase / (ms / 1e3)) < 1e-9


def test_case_ranges_cover_every_case_once():
    sys.path.insert(0, ROOT)
    from paper_1811_02512_gb300 import shard
    for ncase in (0, 1, 7, 1024):
        for world in (1, 2, 3, 8):
            seen = []
            for r in range(world):
                lo, hi = shard.case_range(r, world, ncase)
                assert 0 <= lo <= hi <= ncase and hi - lo in (ncase // world, ncase // world + 1)
                seen.extend(range(lo, hi))
            assert seen == list(range(ncase))
    with pytest.raises(ValueError):
        shard.case_range(2, 2, 5)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    from paper_1811_02512_gb300 import shard
    assert shard.job_throughput(200.0, 5, 1, "cpu") == (200.0, 5.0, 25.0)
    vm = torch.ones((3, 4), dtype=torch.float64)
    st = torch.zeros(3, dtype=torch.int32)
    assert shard.gather_cases(vm, vm, st, 3, 0, 1)[0] is vm
