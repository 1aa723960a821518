"""Writes tiny_plan.json: ten projected implicit-gradient steps (Section 2.2) of the
FP64 oracle on the tiny case (5 buses, T=24), emissions weight kappa = 50 $/t.

Only ``oracle/`` computes anything here; the inputs come from the seeded generator.
Run from the repository root:  python tests/golden/make_tiny_plan.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import dispatch, grad, plan  # noqa: E402
from paper_2410_13055_gb300 import synth  # noqa: E402

KAPPA = 50.0
STEPS = 10


def main():
    nets, scens = synth.tiny()
    opts = synth.default_opts(kappa=KAPPA)
    eta0 = nets[0]["eta_min"].copy()
    sols = dispatch.solve_all(nets, scens, eta0, opts)
    d0 = grad.planner_gradient(nets, scens, sols)
    alpha = 1e-3 * float(np.median(eta0)) / float(np.max(np.abs(d0)))
    traj, objs, deltas = plan.run(nets, scens, eta0, opts, alpha, STEPS)
    out = dict(case="tiny", seed=0, kappa=KAPPA, eps=opts["eps"], voll=opts["voll"], alpha=alpha,
               eta=[list(map(float, e)) for e in traj], objective=list(map(float, objs)),
               delta=[list(map(float, d)) for d in deltas])
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "tiny_plan.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
