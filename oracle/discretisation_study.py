"""Discretisation study of the 16-disc workload with the FP64 oracle (test infrastructure).

The parity contract is the discrete operator at the named order p and contour size N_S; this
script reports how far that discrete solution is from the solution with every contour sum replaced
by its exact integral over the same truncated contour ("converged mode": adaptive Gauss-Kronrod to
1e-13, oracle.converged_solution), at the named p and at p + 4, which separates the contour
quadrature error (discrete vs converged at the same p) from the truncation error (converged p vs
converged p + 4).  It calls only the oracle and prints one line per comparison:

    python -m oracle.discretisation_study
"""
from __future__ import annotations

import sys

import numpy as np

from oracle import lsms_oracle as O


def study(orders=((10, 141.0), (14, 163.0)), sizes=(256, 512, 1024, 2048)):
    """{(p, N_S): discrete-vs-converged scattered-field difference} and the truncation difference
    between the converged solutions of the two orders."""
    from paper_1407_3868_gb300 import inputs
    w = inputs.WORKLOADS["disc16_p10_ns256"]
    m = w.medium
    med = O.Medium(m["k1"], m["k2"], m["k3"], m["d"], m["kp"], m["radius"])
    c, src = w.centres(), w.sources[0]
    out, conv = {}, {}
    for p, t_max in orders:
        lam, wt = O.contour(sizes[0], m["k1"], m["k2"], m["k3"], w.b, t_max)
        _, conv[p] = O.converged_solution(O.Problem(med, p, c, lam, wt), src, w.targets, w.b, t_max, tol=1e-13)
        for ns in sizes:
            lam, wt = O.contour(ns, m["k1"], m["k2"], m["k3"], w.b, t_max)
            pr = O.Problem(med, p, c, lam, wt)
            u = pr.field_layer1(src, pr.solve_dense(src), w.targets, "scattered")
            out[(p, ns)] = float(np.linalg.norm(u - conv[p]) / np.linalg.norm(conv[p]))
    (p0, _), (p1, _) = orders[0], orders[-1]
    trunc = float(np.linalg.norm(conv[p0] - conv[p1]) / np.linalg.norm(conv[p1]))
    return out, trunc


if __name__ == "__main__":
    errs, trunc = study()
    for (p, ns), err in errs.items():
        print(f"p = {p:2d}  N_S = {ns:5d}  contour error (discrete vs converged, same p): {err:.2e}")
    print(f"truncation error (converged p = 10 vs converged p = 14): {trunc:.2e}")
    sys.exit(0)
