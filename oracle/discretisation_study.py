"""Discretisation study of the 16-disc workload with the FP64 oracle (test infrastructure).

The parity contract is the discrete operator at the named order p and contour size N_S; this
script reports how far that discrete solution is from a refined one (p -> p + 4, N_S doubled up to
2048 nodes with a longer contour), i.e. the physical truncation and contour error of the named
configuration.  It calls only the oracle and prints one line per discretisation:

    python -m oracle.discretisation_study
"""
from __future__ import annotations

import sys

import numpy as np

from oracle import lsms_oracle as O


def study(levels=((10, 256, 141.0), (10, 512, 141.0), (10, 1024, 141.0), (14, 1024, 163.0),
                  (14, 2048, 200.0))):
    from paper_1407_3868_gb300 import inputs
    w = inputs.WORKLOADS["disc16_p10_ns256"]
    m = w.medium
    med = O.Medium(m["k1"], m["k2"], m["k3"], m["d"], m["kp"], m["radius"])
    c = w.centres()
    fields = {}
    for p, ns, t_max in levels:
        lam, wt = O.contour(ns, m["k1"], m["k2"], m["k3"], w.b, t_max)
        pr = O.Problem(med, p, c, lam, wt)
        beta = pr.solve_dense(w.sources[0])
        fields[(p, ns)] = pr.field_layer1(w.sources[0], beta, w.targets, "scattered")
    ref = fields[(levels[-1][0], levels[-1][1])]
    return {k: float(np.linalg.norm(u - ref) / np.linalg.norm(ref)) for k, u in fields.items()}


if __name__ == "__main__":
    for (p, ns), err in study().items():
        print(f"p = {p:2d}  N_S = {ns:5d}  scattered-field difference from the finest level: {err:.2e}")
    sys.exit(0)
