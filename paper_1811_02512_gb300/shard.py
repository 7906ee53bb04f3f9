"""Case partition of a batch over the ranks of a job.

The batched workloads shard by case: the cases of one topology (load
scenarios, single-branch outages) are independent power flows, so every rank
solves its own contiguous slice of them with the symbolic analysis repeated
on each rank, and the only collective is the gather of the results at the
end.  A single power flow does not shard: a job of several ranks runs
independent replicas of it.  This module holds the host logic of that
partition (no arithmetic of the method); the per-case solves run in the
CUDA library.
"""
from __future__ import annotations


def case_range(rank: int, world: int, ncase: int) -> tuple[int, int]:
    """Cases [lo, hi) of `rank` among `world` ranks: contiguous slices whose
    sizes differ by at most one, covering 0..ncase-1 exactly once."""
    if world < 1 or not 0 <= rank < world or ncase < 0:
        raise ValueError("bad rank/world/ncase")
    return rank * ncase // world, (rank + 1) * ncase // world


def gather_cases(vm, va, status, ncase: int, rank: int, world: int):
    """All-gathers every rank's slice of the results.

    vm, va: [n_local, nbus] float64 tensors and status: [n_local] int32 tensor
    of this rank's cases (those of case_range(rank, world, ncase)), on the
    device of the process group's backend.  Returns the full (vm, va,
    status) of all ncase cases, in case order, on every rank.  With one rank
    the inputs are returned as they are."""
    import torch
    if world == 1:
        return vm, va, status
    import torch.distributed as dist
    width = max(case_range(r, world, ncase)[1] - case_range(r, world, ncase)[0] for r in range(world))
    nbus = vm.shape[1]
    lo, hi = case_range(rank, world, ncase)
    n = hi - lo

    def padded(t, shape, dtype):
        out = torch.zeros(shape, dtype=dtype, device=t.device)
        out[:n] = t
        return out

    pv = padded(vm, (width, nbus), vm.dtype)
    pa = padded(va, (width, nbus), va.dtype)
    ps = padded(status, (width,), status.dtype)
    gv = [torch.empty_like(pv) for _ in range(world)]
    ga = [torch.empty_like(pa) for _ in range(world)]
    gs = [torch.empty_like(ps) for _ in range(world)]
    dist.all_gather(gv, pv)
    dist.all_gather(ga, pa)
    dist.all_gather(gs, ps)
    parts_v, parts_a, parts_s = [], [], []
    for r in range(world):
        a, b = case_range(r, world, ncase)
        parts_v.append(gv[r][:b - a])
        parts_a.append(ga[r][:b - a])
        parts_s.append(gs[r][:b - a])
    return torch.cat(parts_v), torch.cat(parts_a), torch.cat(parts_s)


def job_throughput(total_ms: float, solves_local: float, world: int, device):
    """Whole-job throughput: the job time is the slowest rank's (max over
    ranks), the solves are summed over ranks -- distinct cases when the ranks
    hold disjoint slices of a batch, replicas when each rank runs the same
    single case.  Returns (max ms, total solves, solves per second)."""
    import torch
    t = torch.tensor([total_ms, float(solves_local)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        tmax = t[:1].clone()
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
        tsum = t[1:].clone()
        dist.all_reduce(tsum, op=dist.ReduceOp.SUM)
        total_ms, solves = float(tmax.item()), float(tsum.item())
    else:
        solves = float(solves_local)
    return total_ms, solves, solves / (total_ms / 1e3)
