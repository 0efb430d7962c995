"""Writes the stored expected values under tests/golden/ by calling only the
FP64 oracle (oracle/) on the seeded synthetic workloads.

The paper prints no worked numeric example (its tables need datasets that are
not available here), so every stored value in this folder comes from this
script:

  plain_100_seed{0,1,2}.json   full oracle solve of the n = n' = 100 workload
  attributed_1000_seed0.json   full oracle solve of the n = n' = 1000 attributed
                               workload (iteration trace, objective, accuracy)

Usage: python tests/golden/make_golden.py [--skip-large]
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_1207_1114_gb300 import synth  # noqa: E402


def record(name, g, **kw):
    t0 = time.time()
    r = oracle.solve(g.A, g.A2, g.B, g.B2, lam=g.lam, **kw)
    out = dict(
        workload=name, n_a=int(g.n), n_b=int(g.n2), k=int(g.k), lam=g.lam, params=kw,
        outer_iters=int(r["outer_iters"]), inner=[int(x) for x in r["inner"]],
        delta=[float(x) for x in r["delta"]], converged=bool(r["converged"]),
        objective=float(r["objective"]), error=float(r["error"]),
        accuracy=float((r["perm"] == g.gt).mean()), perm=[int(x) for x in r["perm"]],
        oracle_seconds=round(time.time() - t0, 2), oracle_threads=oracle.num_threads())
    with open(os.path.join(HERE, name + ".json"), "w") as f:
        json.dump(out, f, indent=1)
    print(name, out["outer_iters"], sum(out["inner"]), out["accuracy"], out["oracle_seconds"])


if __name__ == "__main__":
    for seed in (0, 1, 2):
        record(f"plain_100_seed{seed}", synth.plain_100(seed))
    if "--skip-large" not in sys.argv:
        record("attributed_1000_seed0", synth.attributed_1000(0))
