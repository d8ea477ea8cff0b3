"""GPU solves of the 1000-disc workload (p = 12, 512 contour nodes, one source at (0, 1)) against the
oracle's solution of the same discrete problem, element by element.

The oracle's solution is stored in tests/golden/disc1000_p12_ns512_oracle.txt, written by
tests/golden/make_disc1000_p12_ns512.py from the oracle alone: the dense 25,000 x 25,000 operator of
Sec. 3.2 Eq. "scattmatrix" (with Lemma 3.1, Theorem 5.2, Eq. "sommerfeldsys" and Lemma 5.1 written
out row by row), equilibrated LU, and a residual of 2.6e-14 under the oracle's matrix-free operator
(recorded in the file).  It holds beta for every tenth disc and the three fields at the 64 targets.

Targets: the plain FP64 path within 1e-10, the mixed path with FP64 refinement within 1e-8, both for
beta (in the scaled norm, weights |H_n(k2 R)|) and for the fields.  Each is checked twice: as a
relative 2-norm over the stored entries and element by element, max_i |a_i - b_i| w_i over
max_i |b_i| w_i, so that one wrong disc, order or target cannot hide under the norm.
"""
import os

import numpy as np
import pytest

from oracle import lsms_oracle as O
from paper_1407_3868_gb300 import inputs

pytestmark = pytest.mark.gpu

NAME = "disc1000_p12_ns512"
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", f"{NAME}_oracle.txt")
KINDS = ("total", "scattered", "particle")


def load_golden(path=GOLDEN):
    beta, fields = {}, {k: {} for k in KINDS}
    with open(path) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            tag, a, b, *rest = line.split()
            if tag == "beta":
                re_, im_ = rest
                beta[(int(a), int(b))] = complex(float(re_), float(im_))
            else:
                fields[tag][int(a)] = complex(float(b), float(rest[0]))
    discs = sorted({j for j, _ in beta})
    p = max(n for _, n in beta)
    B = np.array([[beta[(j, n)] for n in range(-p, p + 1)] for j in discs])
    U = {k: np.array([v[t] for t in sorted(v)]) for k, v in fields.items()}
    return discs, B, U


def rel(a, b, w=None):
    a, b = np.asarray(a), np.asarray(b)
    if w is not None:
        a, b = a * w, b * w
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def relmax(a, b, w=None):
    """Largest weighted element error over the largest weighted element of b."""
    a, b = np.asarray(a), np.asarray(b)
    if w is not None:
        a, b = a * w, b * w
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


@pytest.fixture(scope="module")
def L():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1407_3868_gb300 import lsms
    return lsms


@pytest.fixture(scope="module")
def golden():
    return load_golden()


def test_golden_file_matches_the_workload(golden):
    discs, B, U = golden
    w = inputs.WORKLOADS[NAME]
    assert discs[0] == 0 and discs[-1] == w.n - 1 and B.shape == (len(discs), 2 * w.p + 1)
    assert all(U[k].shape == (w.targets.shape[0],) for k in KINDS)
    assert np.all(np.isfinite(B)) and all(np.all(np.isfinite(U[k])) for k in KINDS)


@pytest.mark.parametrize("precision,tol,target", [(0, 1e-13, 1e-10), (1, 1e-11, 1e-8)])
def test_solve_and_fields_match_the_oracle_solution(L, golden, precision, tol, target):
    discs, B, U = golden
    w = inputs.WORKLOADS[NAME]
    m = w.medium
    hs = O.order_scale(w.p, m["k2"], m["radius"])
    ctx = L.context_for(w, precision)
    ctx.set_particles(w.centres())
    beta, info = ctx.solve(w.sources, tol=tol, maxiter=1500)
    assert info["status"] == 0, info
    got = beta[0][discs]
    errs = {"beta": (rel(got, B, hs), relmax(got, B, hs))}
    for k, which in zip(KINDS, (L.FIELD_TOTAL, L.FIELD_SCATTERED, L.FIELD_PARTICLE)):
        u = ctx.eval_field(w.targets, 0, which)
        errs[k] = (rel(u, U[k]), relmax(u, U[k]))
    ctx.close()
    for key, (e2, emax) in errs.items():
        assert e2 < target and emax < target, (precision, key, e2, emax, info["iters"])


def test_mixed_solve_with_box_residuals_matches_the_oracle_solution(L, golden):
    # the FP64 refinement residual through boxes (lsms_set_fmm_scope(LSMS_FMM_RESIDUAL)): the inner
    # solves and every other application keep the all-pairs translation
    discs, B, U = golden
    w = inputs.WORKLOADS[NAME]
    m = w.medium
    hs = O.order_scale(w.p, m["k2"], m["radius"])
    ctx = L.context_for(w, L.LSMS_MIXED)
    ctx.set_particles(w.centres())
    x = inputs.random_coefficients(w.n, w.p, 1, 3) / hs
    y_all_pairs = ctx.apply(x, L.APPLY_MIXED)
    ctx.set_fmm(4.0)
    ctx.set_fmm_scope(L.FMM_RESIDUAL)
    assert ctx.fmm_info()[0] > 2
    ctx.set_timing(True)
    y = ctx.apply(x, L.APPLY_MIXED)                    # applications keep the all-pairs translation:
    assert ctx.fmm_stats()[1:] == (0.0, 0.0)           # the box translation has not run
    assert rel(y, y_all_pairs, hs) < 1e-6               # (same kernels; FP32 atomics in another order)
    beta, info = ctx.solve(w.sources, tol=1e-11, maxiter=1500)
    assert info["status"] == 0 and info["rel_res_fp64"] < 1e-11, info
    assert ctx.fmm_stats()[2] > 0.0                    # the residuals went through the boxes
    ctx.set_timing(False)
    got = beta[0][discs]
    assert rel(got, B, hs) < 1e-8 and relmax(got, B, hs) < 1e-8
    u = ctx.eval_field(w.targets, 0, L.FIELD_SCATTERED)
    assert rel(u, U["scattered"]) < 1e-8 and relmax(u, U["scattered"]) < 1e-8
    ctx.close()
