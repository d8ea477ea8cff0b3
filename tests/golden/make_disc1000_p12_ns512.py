"""Write the oracle's solution of the 1000-disc workload (p = 12, 512 contour nodes, one source at
(0, 1)) to tests/golden/disc1000_p12_ns512_oracle.txt.

Calls only the oracle and the seeded input generators.  The dense (N P) x (N P) matrix of
x -> x - S (T + R) x (25,000 unknowns, 10 GB) is assembled row block by row block on every host
core (`Problem.operator_rows`, the formulas of Lemma 3.1, Theorem 5.2, Eq. "sommerfeldsys" and
Lemma 5.1 written out), equilibrated by the order scale |H_n(k2 R)| and solved by LU (LAPACK), as
`Problem.solve_dense` does for small layouts.  The solution is then checked by an independent
route: its residual under the matrix-free operator `Problem.apply` (the per-target sums), which
the file records.

Stored: beta for every tenth disc (and the last), all orders; the fields TOTAL, SCATTERED and
PARTICLE at the workload's 64 targets on y = 1.5.  Takes a few minutes and ~25 GB of host memory.

    python tests/golden/make_disc1000_p12_ns512.py [--workers N]
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import lsms_oracle as O            # noqa: E402
from paper_1407_3868_gb300 import inputs        # noqa: E402

NAME = "disc1000_p12_ns512"
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"{NAME}_oracle.txt")


def problem_of(w):
    m = w.medium
    lam, wt = O.contour(w.n_nodes, m["k1"], m["k2"], m["k3"], w.b, w.t_max)
    med = O.Medium(m["k1"], m["k2"], m["k3"], m["d"], m["kp"], m["radius"])
    return O.Problem(med, w.p, w.centres(), lam, wt)


def stored_discs(n: int) -> list[int]:
    return sorted(set(list(range(0, n, 10)) + [n - 1]))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=os.cpu_count())
    args = ap.parse_args()
    from scipy import linalg

    w = inputs.WORKLOADS[NAME]
    pr = problem_of(w)
    src = w.sources[0]
    N, P = pr.N, pr.P
    n = N * P
    t0 = time.perf_counter()
    a = np.empty((n, n), dtype=complex)
    with O.RowPool(pr, workers=args.workers) as rp:
        for rows, block in rp.iter_operator_rows(chunks=max(1, N // 25)):
            a[rows[0] * P:(rows[-1] + 1) * P] = block
        t1 = time.perf_counter()
        d = np.tile(O.order_scale(pr.p, pr.m.k2, pr.m.radius), N)
        rhs = pr.rhs(src).ravel()
        a *= d[:, None]
        a /= d[None, :]
        lu = linalg.lu_factor(a, overwrite_a=True, check_finite=False)
        beta = (linalg.lu_solve(lu, d * rhs, check_finite=False) / d).reshape(N, P)
        del a, lu
        t2 = time.perf_counter()
        res = rp.apply(beta).ravel() - rhs
        t3 = time.perf_counter()
    rel_res = float(np.linalg.norm(d * res) / np.linalg.norm(d * rhs))
    fields = {k: pr.field_layer1(src, beta, w.targets, k) for k in ("total", "scattered", "particle")}
    with open(OUT, "w") as f:
        f.write(f"# oracle solution of workload {NAME}: {N} discs, p = {pr.p}, {w.n_nodes} contour "
                f"nodes (b = {w.b!r}, t_max = {w.t_max!r}), source {src.tolist()}\n")
        f.write("# written by tests/golden/make_disc1000_p12_ns512.py (oracle only): dense operator "
                "assembled by rows, equilibrated LU\n")
        f.write(f"# scaled residual under the matrix-free oracle operator: {rel_res:.3e}\n")
        f.write(f"# assembly {t1 - t0:.1f} s, LU {t2 - t1:.1f} s, residual {t3 - t2:.1f} s, "
                f"{args.workers} workers\n")
        f.write("# beta rows: 'beta <disc> <order n> <re> <im>'; field rows: "
                "'<total|scattered|particle> <target> <re> <im>'\n")
        for j in stored_discs(N):
            for i, nn in enumerate(range(-pr.p, pr.p + 1)):
                v = beta[j, i]
                f.write(f"beta {j} {nn} {float(v.real)!r} {float(v.imag)!r}\n")
        for k, u in fields.items():
            for t, v in enumerate(u):
                f.write(f"{k} {t} {float(v.real)!r} {float(v.imag)!r}\n")
    print(f"wrote {OUT}: residual {rel_res:.3e}, assembly {t1 - t0:.1f} s, LU {t2 - t1:.1f} s")


if __name__ == "__main__":
    main()
