"""Writes tests/golden/oracle_n8.json: oracle outputs for a seeded 8-body case.

Calls only the oracle and the workload generators.  The fixture is a change
detector for the oracle (its physics pins live in tests/test_oracle_pins.py).
Run: python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import oracle  # noqa: E402
import workloads as W  # noqa: E402


def main():
    cl = W.plummer(8, 2024, masses="kroupa")
    a0, j0, tl = W.hermite_state(cl, seed=2024, t_block=0.25, steps=np.full(8, 0.125))
    xp, vp = oracle.predict(0.25, cl.x, cl.v, a0, j0, tl)
    idx = np.array([7, 0, 3, 5], dtype=np.int32)
    rs2 = 0.5
    acc, jerk, pot, cnt, lists = oracle.regular_force(xp, vp, cl.m, idx, rs2, cap=8)
    out = dict(note="oracle outputs, seeded Plummer N=8 (Kroupa masses), written by make_golden.py",
               x=cl.x.tolist(), v=cl.v.tolist(), m=cl.m.tolist(), a=a0.tolist(), jerk0=j0.tolist(),
               t_last=tl.tolist(), t=0.25, idx=idx.tolist(), rs2=rs2, xp=xp.tolist(), vp=vp.tolist(),
               acc=acc.tolist(), jerk=jerk.tolist(), pot=pot.tolist(), nb_count=cnt.tolist(),
               nb_lists=[l.tolist() for l in lists])
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_n8.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
