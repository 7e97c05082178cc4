"""Writes workload4_oracle.json: the FP64 oracle's W, final marginal error and
stop iteration for workload-4 images (512 x 512, eps = 1e-3, tol = 1e-6, cap
5000; the stabilised form): two that run to the cap without meeting tol and
one that stops early.  Calls only the oracle (oracle/cref.py, the sequential C
recurrences) and the seeded input generators; takes a few minutes on three
host cores.

    python tests/golden/make_workload4_oracle.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import cref  # noqa: E402
from paper_2202_10042_gb300 import inputs  # noqa: E402

CAPPED = (8, 10)  # images that reach the cap of 5000 iterations
EARLY = (3,)     # an image that meets tol before the cap


def main():
    images = CAPPED + EARLY
    ps = [inputs.workload4(i) for i in images]
    res = cref.solve_many([(p.a, p.b, tuple(p.h), p.eps, p.tol, p.itr_max) for p in ps], tau=1e10)
    out = {"workload": "fs1_2d_log_fp32_batch64_512x512_eps1e-3", "form": "stabilised, FP64 oracle (cref)",
           "images": {}}
    for i, p, r in zip(images, ps, res):
        assert r.status == cref.OK, (i, r)
        if i in CAPPED:
            assert r.iters == p.itr_max and r.err > p.tol, (i, r)
        else:
            assert r.iters < p.itr_max and r.err <= p.tol, (i, r)
        out["images"][str(i)] = {"side": int(p.a.shape[0]), "eps": p.eps, "tol": p.tol, "itr_max": int(p.itr_max),
                                 "iters": int(r.iters), "w": r.w, "err": r.err}
    with open(os.path.join(HERE, "workload4_oracle.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
