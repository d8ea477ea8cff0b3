"""GPU parity at the ends of the order range the ABI accepts: p = 0 (the degenerate truncation, one
order per disc), p = 3 (the FP32 translation's variant for p < 6, one output per lane) and p = 15 (the
largest order, P = 31), each on a ragged layout of 19 discs (a full 8-target tile, a ragged tail,
and a source chunk cut short): the FP64 operator and its two parts, the mixed operator, and the
FP64 solve with its fields, against the oracle.  Tolerances as in the other parity files (scaled
norms, 1e-10 FP64, 2e-5 for the mixed operator).

Collected after every other GPU file, so that a run stopping at the first failure has run them."""
import numpy as np
import pytest

from oracle import lsms_oracle as O
from paper_1407_3868_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL_MIXED_OP = 2e-5


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


def workload(p):
    # t_max grows with the order as for the named workloads (141, 152, 163 at p = 10, 12, 14)
    base = inputs.WORKLOADS["disc16_p10_ns256"]
    t_max = {0: 60.0, 3: 60.0, 15: 169.0}[p]
    return inputs.Workload(f"orders_p{p}", 19, p, 256, t_max, -4.0, 4.0, 40 + p, base.sources, base.targets,
                           1e-12)


@pytest.fixture(scope="module", params=[0, 3, 15])
def case(L, request):
    p = request.param
    w = workload(p)
    m = w.medium
    c = w.centres()
    lam, wt = O.contour(w.n_nodes, m["k1"], m["k2"], m["k3"], w.b, w.t_max)
    pr = O.Problem(O.Medium(m["k1"], m["k2"], m["k3"], m["d"], m["kp"], m["radius"]), p, c, lam, wt)
    hs = O.order_scale(p, m["k2"], m["radius"])
    ctx = L.context_for(w)
    ctx.set_particles(c)
    yield w, c, pr, hs, ctx
    ctx.close()


def test_operator_at_the_order_range_ends(L, case):
    w, c, pr, hs, ctx = case
    beta = inputs.random_coefficients(c.shape[0], w.p, 1, 70 + w.p) / hs[None, None, :]
    ws = hs * np.abs(pr.S)
    assert rel(ctx.apply(beta)[0], pr.apply(beta[0]), hs) < TOL64
    aT = ctx.apply(beta, L.APPLY_ALPHA | L.APPLY_NO_REFLECTION)[0]
    aR = ctx.apply(beta, L.APPLY_ALPHA | L.APPLY_NO_TRANSLATION)[0]
    assert rel(aT, pr.translation(beta[0]), ws) < TOL64
    assert rel(aR, pr.reflection(beta[0]), ws) < TOL64
    assert rel(ctx.apply(beta, L.APPLY_MIXED)[0], pr.apply(beta[0]), hs) < TOL_MIXED_OP


def test_solve_at_the_order_range_ends(L, case):
    w, c, pr, hs, ctx = case
    src = w.sources[0]
    beta, info = ctx.solve(w.sources, tol=1e-13, maxiter=1000)
    assert info["status"] == 0
    b_o = pr.solve_dense(src)
    assert rel(beta[0], b_o, hs) < TOL64
    u = ctx.eval_field(w.targets, 0, L.FIELD_SCATTERED)
    assert rel(u, pr.field_layer1(src, b_o, w.targets, "scattered")) < TOL64
