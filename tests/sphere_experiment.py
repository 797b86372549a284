"""Runner for the paper's single-sphere experiment (Sec. 3.1): GPU solve and
field from paper_1910_01011_gb300.experiments.sphere, l2 error of the total
field against the analytic series (oracle.mie) on the 200 x 200 grid.

Run on a GPU:  python tests/sphere_experiment.py [--el 4 6 8 10]
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def measure(material: str, el_per_lambda: float, **kw) -> dict:
    from oracle import mie
    from paper_1910_01011_gb300.experiments import sphere
    r = sphere.run(material, el_per_lambda, **kw)
    ref = mie.total_field(r["points"], r["radius"], r["k0"], r["kj"], r["rho0"], r["rho"])
    r["field_l2_error"] = float(np.linalg.norm(r["field"] - ref) / np.linalg.norm(ref))
    for key in ("points", "field", "k0", "kj"):
        r.pop(key)
    return r


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--el", type=float, nargs="+", default=[4, 6, 8, 10])
    ap.add_argument("--materials", nargs="+", default=["fat", "bone"])
    ap.add_argument("--tol", type=float, default=1e-5)
    args = ap.parse_args()
    for m in args.materials:
        for e in args.el:
            print(json.dumps(measure(m, e, tol=args.tol)))


if __name__ == "__main__":
    main()
