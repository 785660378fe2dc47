"""Writes reference_counts.json: the oracle's own outer FGMRES step count for the benchmark
workload (64^3 Gaussian bumps, J = 8, FGMRES(30), 4 inner steps, rtol 1e-8), so that the timed
CPU baseline can run a bounded sample of steps and scale it to a whole solve.  Calls only
oracle/ and workloads/.  Test infrastructure, like the rest of oracle/."""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import workloads as W  # noqa: E402
from oracle import hz_oracle as O  # noqa: E402


def main():
    out = {}
    for wl in (W.gaussian_bumps_64(), W.point_source_32()):
        op = O.make_operator(wl.c, wl.h, wl.omega, wl.layer_cells, wl.sigma_max)
        _, nodes = O.setup_nodes(op, wl.J, wl.t, wl.eps)
        t0 = time.time()
        res = O.solve(op, op.s * wl.f[0], nodes, wl.restart, wl.k_in, wl.rtol, 50)
        out[wl.name] = {"its": res.its, "cycles": res.cycles, "rel_res_true": res.rel_res_true,
                        "converged": bool(res.converged),
                        "poly_matvecs_per_fci": sum(n.q * n.sweeps for n in nodes),
                        "seconds_here": round(time.time() - t0, 1)}
        print(wl.name, out[wl.name], flush=True)
    with open(os.path.join(HERE, "reference_counts.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
