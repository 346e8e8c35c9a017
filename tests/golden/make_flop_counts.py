"""Writes flops_per_unit.json: algorithmic FP64 operations of one step, per unit
of work of each kernel group, counted by the flop-counting build of the CPU
oracle (an add/sub/mul with an exact-zero operand is not counted; a division,
square root or pow counts as one operation; compares are listed apart).

Workload: the 64x32x16 magnetised torus block (seed 1912), second step (the
first settles the inversions' guesses). Calls only oracle/ and the input
generator.
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
sys.path.insert(0, os.path.dirname(HERE))

import oracle as O  # noqa: E402
from helpers import torus_case  # noqa: E402


def count(n1=64, n2=32, n3=16, seed=1912):
    geo, d, prim, bf = torus_case(n1, n2, n3, seed=seed)
    g = O.Grid(d, counting=True)
    g.set(prim, bf)
    g.step()
    O.flops_reset()
    g.step()
    ph = O.flops_phase()
    flops = {k: sum(v[:4]) for k, v in ph.items()}
    ncell = n1 * n2 * n3
    faces = ((n1 + 1) * (n2 + 2) * (n3 + 2) + (n1 + 2) * (n2 + 1) * (n3 + 2) + (n1 + 2) * (n2 + 2) * (n3 + 1))
    recon_cells = 3 * (n1 + 2) * (n2 + 2) * (n3 + 2)
    edges = (n1 + 1) * (n2 + 1) * (n3 + 1)
    stages = 2
    return {
        "workload": "torus %dx%dx%d seed %d, one midpoint step" % (n1, n2, n3, seed),
        "per_zone_cycle": sum(flops.values()) / ncell,
        "flux_per_face": flops["flux"] / (stages * faces),
        "recon_per_cell_dir": flops["recon"] / (stages * recon_cells),
        "update_per_cell_stage": flops["update"] / (stages * ncell),
        "cfl_per_cell": flops["cfl"] / ncell,
        "emf_per_edge_stage": flops["emf"] / (stages * edges),
        "ct_per_edge_stage": flops["ct"] / (stages * edges),
        "raw_per_phase": ph,
    }


if __name__ == "__main__":
    out = count()
    with open(os.path.join(HERE, "flops_per_unit.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps({k: v for k, v in out.items() if k != "raw_per_phase"}, indent=1))
