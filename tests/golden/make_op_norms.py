"""Write tests/golden/op_norms.json: ||U^{1/2} Phi||_S^2 of the seeded
benchmark workloads, computed by the FP64 oracle alone.

eta = 1 / ||U^{1/2} Phi||_S^2 (Section 5.1) is what the oracle-timed
benchmark arm runs Algorithm 3 with.  On these strongly non-uniform
coverages the power iteration needs thousands of operator applications to
converge (20 steps still sit 17 % low at 512^2, which breaks the convergence
condition, Eq. "convergence-req-explicit-pd"), so the value is taken by the
oracle's Lanczos routine once, offline, and stored.

Usage: python tests/golden/make_op_norms.py [workload ...]   (default: c2_512 c3_1024)
Single-threaded it takes about 2 minutes for c2_512 and 20 for c3_1024.
"""
from __future__ import annotations

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import nufft, ppd  # noqa: E402
from paper_1701_01748_gb300 import synth  # noqa: E402

OUT = os.path.join(HERE, "op_norms.json")


def main(names):
    table = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for name in names:
        p = synth.make_problem(name)
        P = nufft.Plan(p.omega, p.L, p.L, theta=p.theta)
        U = nufft.uniform_weights(p.omega, P.K0, P.K1)[0]
        t0 = time.time()
        val, napp = ppd.op_norm_sq_lanczos(P, U, tol=1e-8)
        table[name] = {"seed": p.seed, "L": p.L, "M": p.M, "n_blocks": p.n_blocks, "op_norm_sq": val,
                       "method": "oracle.ppd.op_norm_sq_lanczos(tol=1e-8), U = 1/cell count",
                       "operator_applications": napp, "seconds": round(time.time() - t0, 1)}
        print(name, table[name], flush=True)
        with open(OUT, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
            f.write("\n")


if __name__ == "__main__":
    main(sys.argv[1:] or ["c2_512", "c3_1024"])
