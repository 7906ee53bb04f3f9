"""Write the loading factor of every named synthetic grid using only the oracle.

The raw grids (paper_1811_02512_gb300.gridgen) carry loads and generation drawn
from the stated distributions; at full size such grids have no power-flow
solution.  The loading factor of a grid is lam = lam_star / 2, where lam_star
is the largest 2^-k (k >= 0) at which the oracle's flat-start Newton-Raphson
converges to 1e-8 p.u. within 10 iterations.  On the grids of the uneven multi-grid batch
(grids "multigrid<g>", 2,000 to 80,000 buses) flat-start Newton-Raphson and
the fast decoupled iteration diverge at every injection scaling once a grid
has more than about 15,000 buses: the line charging, off-nominal taps and
PV set-points alone drive flows the flat start cannot reach.  For those grids
the same rule is applied to the whole network (Case.scaled_network: the
injections, the line charging, the tap and set-point deviations from 1).
The result is stored in
paper_1811_02512_gb300/data/loading_factors.json, keyed by grid name, seed,
bus and branch count.

Usage: python -m oracle.find_loading_factors [--configs 0,1,3,4] [--jobs N]
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from oracle import oracle as O  # noqa: E402
from paper_1811_02512_gb300 import gridgen  # noqa: E402


def loading_factor(raw, kmax=20):
    network = gridgen.network_scaled(raw.name)
    for k in range(kmax + 1):
        lam = 2.0 ** -k
        case = raw.scaled_network(lam) if network else raw.scaled(lam)
        rc, _, _, it, _ = O.power_flow(case, O.NR, tol=1e-8, max_iter=10)
        if rc == O.OK and it <= 10:
            return lam / 2.0
    raise RuntimeError(f"no loading factor found for {raw.name}")


def _one(spec):
    kind, a, b, name = spec
    raw = gridgen.config0_raw() if kind == "c0" else gridgen.delaunay_raw(a, b, name=name)
    return gridgen.loading_key(raw), loading_factor(raw)


def specs(configs):
    out = []
    if 0 in configs:
        out.append(("c0", 0, 0, "grid120"))
    if 1 in configs or 2 in configs:
        out.append(("d", 10000, gridgen.SEED_BASE + 1, "delaunay10k"))
    if 3 in configs:
        out.append(("d", 20000, gridgen.SEED_BASE + 3, "delaunay20k"))
    if 4 in configs:
        for g, (n, s) in enumerate(gridgen.config4_sizes()):
            out.append(("d", n, s, f"multigrid{g}"))
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--configs", default="0,1,3,4")
    ap.add_argument("--jobs", type=int, default=os.cpu_count() or 1)
    args = ap.parse_args()
    configs = {int(x) for x in args.configs.split(",")}
    table = gridgen.load_loading_factors()
    todo = sorted(specs(configs), key=lambda sp: -sp[1])  # largest grids first
    ctx = mp.get_context("spawn")
    os.makedirs(os.path.dirname(gridgen.LOADING_FACTOR_FILE), exist_ok=True)
    with ctx.Pool(args.jobs) as pool:
        for key, lam in pool.imap_unordered(_one, todo):
            table[key] = lam
            print(key, lam, flush=True)
            with open(gridgen.LOADING_FACTOR_FILE, "w") as fh:
                json.dump(dict(sorted(table.items())), fh, indent=1)


if __name__ == "__main__":
    main()
