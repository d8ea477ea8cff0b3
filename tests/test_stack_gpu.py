"""GPU parity of a five-layer medium (lsms_create_stack: the interface conditions of Sec. 2 at every
interface, the per-node system of Sec. 5.2 extended to all layers) against the oracle's Stack.

Layers (top to bottom) k = 2pi, 2.6pi, 3pi, 3.4pi, 4pi; interior thicknesses 0.5, 2.0, 0.7; the discs
(kp = 2.4pi, R = 0.25) in layer 3, 0.5 below the top interface.  The library takes centres in the
global frame (layer 1 is y > 0); the oracle's Problem takes them in the disc layer's own frame (its
top interface at y = 0), so the two differ by the depth 0.5.  Norms and tolerances as in the
three-layer parity tests: 1e-10 (FP64), 2e-5 (mixed operator), 1e-8 (mixed solve).
"""
import math

import numpy as np
import pytest

from oracle import lsms_oracle as O
from paper_1407_3868_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL_MIXED_OP = 2e-5
TOL_MIXED = 1e-8

KS = inputs.STACK5["ks"]
DS = inputs.STACK5["ds"]
LAYER = inputs.STACK5["layer"]
DEPTH = inputs.STACK5_DEPTH
KP, RADIUS = 2.4 * math.pi, 0.25


@pytest.fixture(scope="module")
def L():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1407_3868_gb300 import lsms
    return lsms


def rel(a, b, w=None):
    a, b = np.asarray(a), np.asarray(b)
    if w is not None:
        a, b = a * w, b * w
    return np.linalg.norm(a - b) / np.linalg.norm(b)


class StackCase:
    def __init__(self, L, n, p, n_nodes, seed, precision=0, width=8.0, t_max=60.0):
        self.local = inputs.layout(n, -width / 2, width / 2, seed)        # -2 < y < 0
        self.glob = self.local - np.array([0.0, DEPTH])
        self.p, self.n = p, n
        b = 0.1 * KS[0]
        self.ctx = L.Context(0, 0, 0, 0, KP, RADIUS, p, n_nodes, b=b, t_max=t_max, panel_order=16,
                             precision=precision, stack=(KS, DS, LAYER))
        self.ctx.set_particles(self.glob)
        self.lam, self.wt = O.contour(n_nodes, KS[0], KS[LAYER - 1], KS[-1], b, t_max,
                                      branch_points=KS)
        self.st = O.Stack(KS, DS, LAYER, KP, RADIUS)
        self.pr = O.Problem(self.st, p, self.local, self.lam, self.wt)
        self.hs = O.order_scale(p, KS[LAYER - 1], RADIUS)
        self.src = np.array([[0.3, 1.0], [-1.1, 0.6]])
        self.tgt = inputs.observation_points(-width / 2, width / 2, 12, 1.5)

    def rand_beta(self, seed, nrhs=1):
        return inputs.random_coefficients(self.n, self.p, nrhs, seed) / self.hs[None, None, :]


@pytest.fixture(scope="module")
def case(L):
    c = StackCase(L, 24, 8, 192, 31)
    yield c
    c.ctx.close()


def test_contour_is_graded_to_every_wavenumber(case):
    lam, wt = case.ctx.contour()
    assert np.allclose(lam, case.lam, rtol=0, atol=1e-13)
    assert np.allclose(wt, case.wt, rtol=0, atol=1e-13)


def test_stack_aggregate_reflect_disaggregate_and_incident(case):
    beta = case.rand_beta(5)
    ws = case.hs * np.abs(case.pr.S)
    pp, qm = case.ctx.aggregate(beta)
    pp_o, qm_o = case.pr.aggregate(beta[0])
    assert rel(pp[0], pp_o) < TOL64 and rel(qm[0], qm_o) < TOL64
    sp, sm = case.ctx.reflect(pp_o, qm_o)
    sig_o = case.pr.layer_densities(None, pp_o, qm_o)
    assert rel(sp[0], sig_o[:, 1]) < 1e-12 and rel(sm[0], sig_o[:, 2]) < 1e-12
    a = case.ctx.disaggregate(sig_o[:, 1], sig_o[:, 2])[0]
    assert rel(a, case.pr.disaggregate(sig_o[:, 1], sig_o[:, 2]), ws) < TOL64
    a_inc = case.ctx.incident(case.src)
    for s in range(case.src.shape[0]):
        assert rel(a_inc[s], case.pr.incident_local(case.src[s]), ws) < TOL64, s


@pytest.mark.parametrize("precision,tol", [(0, TOL64), (1, TOL_MIXED_OP)])
def test_stack_apply_matches_the_oracle(L, case, precision, tol):
    beta = case.rand_beta(7, 2)
    y = case.ctx.apply(beta) if precision == 0 else _apply_mixed(L, case, beta)
    for r in range(2):
        assert rel(y[r], case.pr.apply(beta[r]), case.hs) < tol, r


def _apply_mixed(L, case, beta):
    with L.Context(0, 0, 0, 0, KP, RADIUS, case.p, case.lam.size, b=0.1 * KS[0], t_max=60.0,
                   panel_order=16, precision=L.LSMS_MIXED, stack=(KS, DS, LAYER)) as ctx:
        ctx.set_particles(case.glob)
        return ctx.apply(beta)


@pytest.mark.parametrize("precision,tol", [(0, TOL64), (1, TOL_MIXED)])
def test_stack_solve_and_fields_match_the_oracle(L, case, precision, tol):
    with L.Context(0, 0, 0, 0, KP, RADIUS, case.p, case.lam.size, b=0.1 * KS[0], t_max=60.0,
                   panel_order=16, precision=precision, stack=(KS, DS, LAYER)) as ctx:
        ctx.set_particles(case.glob)
        beta, info = ctx.solve(case.src, tol=1e-12 if precision == 0 else 1e-11, maxiter=400)
        assert info["status"] == 0
        for s in range(case.src.shape[0]):
            b_o = case.pr.solve_dense(case.src[s])
            assert rel(beta[s], b_o, case.hs[None, :]) < tol, s
            for which, name in ((L.FIELD_TOTAL, "total"), (L.FIELD_SCATTERED, "scattered"),
                                (L.FIELD_PARTICLE, "particle")):
                u = ctx.eval_field(case.tgt, s, which)
                u_o = case.pr.field_layer1(case.src[s], b_o, case.tgt, name)
                assert rel(u, u_o) < tol, (s, name)


def test_three_layer_stack_equals_the_three_layer_context(L):
    w = inputs.WORKLOADS["disc16_p10_ns256"]
    m = w.medium
    c = w.centres()
    beta = inputs.random_coefficients(w.n, w.p, 1, 3)
    with L.context_for(w) as a, L.Context(0, 0, 0, 0, m["kp"], m["radius"], w.p, w.n_nodes, b=w.b,
                                          t_max=w.t_max, panel_order=16,
                                          stack=([m["k1"], m["k2"], m["k3"]], [m["d"]], 2)) as b:
        a.set_particles(c)
        b.set_particles(c)
        # the same arithmetic; only the order of FP64 atomic additions may differ between runs
        assert rel(b.apply(beta), a.apply(beta)) < 1e-13


# ---------------------------------------------------------------------------------------------
# Absorbing layers (lsms_create_stack_c): a lossy film below the disc layer, over a substrate
# ---------------------------------------------------------------------------------------------
KS_LOSSY = [2 * math.pi, 3 * math.pi, 3.4 * math.pi + 0.5j, 4 * math.pi]
DS_LOSSY = [2.0, 0.7]


@pytest.mark.parametrize("precision,tol_op,tol_solve", [(0, TOL64, TOL64), (1, TOL_MIXED_OP, TOL_MIXED)])
def test_lossy_film_apply_solve_and_fields(L, precision, tol_op, tol_solve):
    n, p, n_nodes, b, t_max = 20, 8, 512, 0.2, 80.0
    local = inputs.layout(n, -3.0, 3.0, 44)
    src = np.array([[0.3, 1.0], [-1.0, 0.7]])
    tg = inputs.observation_points(-3.0, 3.0, 12, 1.5)
    lam, wt = O.contour(n_nodes, KS_LOSSY[0], KS_LOSSY[1], KS_LOSSY[3].real, b, t_max,
                        branch_points=[complex(k).real for k in KS_LOSSY])
    pr = O.Problem(O.Stack(KS_LOSSY, DS_LOSSY, 2, KP, RADIUS), p, local, lam, wt)
    hs = O.order_scale(p, KS_LOSSY[1], RADIUS)
    with L.Context(0, 0, 0, 0, KP, RADIUS, p, n_nodes, b=b, t_max=t_max, panel_order=16,
                   precision=precision, stack=(np.array(KS_LOSSY), DS_LOSSY, 2)) as ctx:
        ctx.set_particles(local)                 # disc layer directly below y = 0: no depth shift
        l2, w2 = ctx.contour()
        assert np.abs(l2 - lam).max() < 1e-12 and np.abs(w2 - wt).max() < 1e-13
        x = inputs.random_coefficients(n, p, 1, 12) / hs[None, None, :]
        assert rel(ctx.apply(x)[0], pr.apply(x[0]), hs) < tol_op
        beta, info = ctx.solve(src, tol=1e-12 if precision == 0 else 1e-11, maxiter=400)
        assert info["status"] == 0
        for s in range(2):
            b_o = pr.solve_dense(src[s])
            assert rel(beta[s], b_o, hs[None, :]) < tol_solve, s
            for which, name in ((L.FIELD_SCATTERED, "scattered"), (L.FIELD_PARTICLE, "particle")):
                u = ctx.eval_field(tg, s, which)
                assert rel(u, pr.field_layer1(src[s], b_o, tg, name)) < tol_solve, (s, name)
