"""Runs one condense, one K apply and one preconditioner application on a workload, for
kernel profilers (ncu) to capture.

  python -m paper_2207_08481_gb300.profile_case [c2|c3|c3s] [mixed|fp64]
(c3s: the c3 element type on 16^3 x 6 cells, small enough for full ncu captures)
"""
from __future__ import annotations

import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

CASES = {"c2": dict(dim=2, N=256, k=3, nu=1e-2, levels=5), "c3": dict(dim=3, N=32, k=2, nu=1.0, levels=4),
         "c3s": dict(dim=3, N=16, k=2, nu=1.0, levels=3)}


def main(argv):
    import torch

    import paper_2207_08481_gb300.mcs as mcs
    import workloads
    case = CASES[argv[1] if len(argv) > 1 else "c2"]
    prec = mcs.MCS_FP64 if (len(argv) > 2 and argv[2] == "fp64") else mcs.MCS_MIXED
    torch.cuda.set_device(0)
    h = mcs.Handle.structured(case["dim"], case["N"], case["k"], case["nu"], precision=prec,
                              gmg_levels=case["levels"])
    s = h.sizes
    h.condense()
    xq = torch.zeros((s.ne * s.nq_load, case["dim"]), dtype=torch.float64, device="cuda")
    h.load_points(xq)
    F = torch.zeros(s.ndof, dtype=torch.float64, device="cuda")
    h.load_vector(workloads.manufactured_f(case["dim"], case["nu"], xq), F)
    y = torch.zeros_like(F)
    h.apply(F, y)
    h.precond(F, y)
    torch.cuda.synchronize()
    h.close()
    print("profile case done")


if __name__ == "__main__":
    main(sys.argv)
