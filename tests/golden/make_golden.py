"""Writes the stored expected values under tests/golden/ from the CPU oracle only.

uc3bus_2periods.json: the 3-bus, 3-line, 3-generator, 2-period instance (seed 0)
  lp_optimum   -- dense simplex optimum of the LP relaxation
  milp_optimum -- best of all 2^6 commitment schedules (each LP by the simplex)

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle.brute import milp_by_enumeration  # noqa: E402
from oracle.lp import lp_from_arrays  # noqa: E402
from oracle.simplex import simplex_solve  # noqa: E402
from paper_2512_06715_gb300 import build  # noqa: E402
from paper_2512_06715_gb300.instances import build_instance  # noqa: E402


def main():
    build.build_ucgen()
    inst = build_instance(3, 3, 3, 2, seed=0)
    lp = lp_from_arrays(inst.row_ptr, inst.col, inst.val, inst.q, inst.c, inst.l, inst.u, inst.m_eq)
    sx = simplex_solve(lp)
    best, sched = milp_by_enumeration(lp, inst.idx_u)
    out = dict(instance=dict(n_bus=3, n_line=3, n_gen=3, n_periods=2, seed=0),
               lp_optimum=sx.obj, milp_optimum=best, milp_schedule=sched.tolist(),
               source="oracle.simplex (LP) and oracle.brute (MILP by enumeration)")
    with open(os.path.join(os.path.dirname(__file__), "uc3bus_2periods.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(out)


if __name__ == "__main__":
    main()
