"""Write the stored oracle trajectories used by the parity tests.

Calls only `oracle/` and `synth/`. The paper prints no worked example with
values, so every stored number here is an oracle output:

  dd32_k0.json   the 32 x 32 workload (3-component mixtures, eps = (1/32)^2,
                 4 x 4 basic cells, product initial plan, cell tolerance 1e-7),
                 seed pair k = 0, 20 hybrid iterations (Alg. 3): per half-iteration
                 the objective E, the L1 X / Y marginal errors and the maximal
                 Sinkhorn iteration count; per flow update its optimal value.

Usage: python tests/golden/make_golden.py
"""

import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synth  # noqa: E402
from oracle.hybrid import OracleDD  # noqa: E402


def dd32(k=0):
    mu, nu, eps, p = synth.workload("dd32", k)
    o = OracleDD(mu, nu, eps, p["s"], tol=p["tol"])
    steps = []
    for it in range(p["iters"]):
        for part in (0, 1):
            info = o.iterate(part)
            steps.append(dict(kind="A" if part == 0 else "B", E=info["E"], l1_x=info["l1_x"],
                              l1_y=info["l1_y"], iters_max=int(max(info["iters"]))))
        f = o.flow_update()
        steps.append(dict(kind="F", value=f["value"], l1_y=f["l1_y"]))
        print(it, steps[-3]["E"], steps[-2]["E"], f["value"], flush=True)
    out = dict(workload="dd32", k=k, eps=eps, tol=p["tol"], s=p["s"], steps=steps)
    with open(os.path.join(HERE, f"dd32_k{k}.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    dd32(0)
