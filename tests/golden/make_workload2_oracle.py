"""Writes workload2_oracle.json: the FP64 oracle's W and final marginal error
for workload-2 pairs (N = 2^20, eps = 1e-4, the stabilised form) that run to
the iteration cap of 5000 without meeting tol = 1e-6.  Calls only the oracle
(oracle/cref.py, the sequential C recurrences) and the seeded input
generators; takes about five minutes on two host cores.

    python tests/golden/make_workload2_oracle.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import cref  # noqa: E402
from paper_2202_10042_gb300 import inputs  # noqa: E402

PAIRS = (0, 17)


def main():
    ps = [inputs.workload2(i) for i in PAIRS]
    res = cref.solve_many([(p.a, p.b, p.h[0], p.eps, p.tol, p.itr_max) for p in ps], tau=1e10)
    out = {"workload": "fs1_1d_log_fp32_batch256_n2^20_eps1e-4", "form": "stabilised, FP64 oracle (cref)",
           "pairs": {}}
    for i, p, r in zip(PAIRS, ps, res):
        assert r.status == cref.OK and r.iters == p.itr_max, (i, r)
        out["pairs"][str(i)] = {"n": int(p.a.size), "eps": p.eps, "tol": p.tol, "iters": int(r.iters),
                                "w": r.w, "err": r.err}
    with open(os.path.join(HERE, "workload2_oracle.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
