"""GPU parity with the greedy contour panel rule (lsms_contour.panel_rule = 1) in a medium without
guided modes: the library's nodes equal the oracle's greedy contour, and the FP64 operator, solve
and layer-1 field on them match the oracle's Problem on the same nodes (1e-10, scaled norms).  The
kernels are those of the default rule; only the node placement differs.

Collected after the other parity files (with the order-range file), so that a run stopping at the
first failure has run them."""
import numpy as np
import pytest

from oracle import lsms_oracle as O
from paper_1407_3868_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


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


def test_greedy_panel_rule_parity(L):
    w = inputs.WORKLOADS["disc16_p10_ns256"]
    m = w.medium
    n_nodes = 768
    c = w.centres()
    lam, wt = O.contour(n_nodes, m["k1"], m["k2"], m["k3"], w.b, w.t_max, greedy=True)
    pr = O.Problem(O.Medium(m["k1"], m["k2"], m["k3"], m["d"], m["kp"], m["radius"]), w.p, c, lam, wt)
    hs = O.order_scale(w.p, m["k2"], m["radius"])
    with L.Context(m["k1"], m["k2"], m["k3"], m["d"], m["kp"], m["radius"], w.p, n_nodes, b=w.b,
                   t_max=w.t_max, panel_order=16, precision=L.LSMS_FP64, panel_rule=1) as ctx:
        lam_l, wt_l = ctx.contour()
        assert np.max(np.abs(lam_l - lam)) <= 1e-12 * w.t_max
        assert np.max(np.abs(wt_l - wt)) <= 1e-14 * w.t_max
        ctx.set_particles(c)
        beta = inputs.random_coefficients(w.n, w.p, 1, 91) / hs[None, None, :]
        assert rel(ctx.apply(beta)[0], pr.apply(beta[0]), hs) < TOL64
        b_l, info = ctx.solve(w.sources, tol=1e-12, maxiter=1000)
        assert info["status"] == 0
        b_o = pr.solve_dense(w.sources[0])
        assert rel(b_l[0], b_o, hs[None, :]) < TOL64
        u = ctx.eval_field(w.targets, 0, L.FIELD_SCATTERED)
        assert rel(u, pr.field_layer1(w.sources[0], b_o, w.targets, "scattered")) < TOL64
