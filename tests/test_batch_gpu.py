"""GPU tests of the batched forms: a batch of independent layouts (design sweep) and the autotuner.

A layout batch must give, layout by layout, what a context holding that layout alone gives (same
kernels, so to rounding), and one of its layouts is also checked against the FP64 oracle.
"""
import numpy as np
import pytest

from oracle import lsms_oracle as O
from paper_1407_3868_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1407_3868_gb300 import lsms
    return lsms


def workload():
    base = inputs.WORKLOADS["disc16_p10_ns256"]
    return inputs.Workload("batch", 0, 8, 192, 60.0, -3.0, 3.0, 0, base.sources, base.targets, 1e-12)


def layouts():
    return [inputs.layout(n, -0.3 * n, 0.3 * n, 40 + n) for n in (7, 20, 33)]


def rel(a, b, w=None):
    a, b = np.asarray(a), np.asarray(b)
    if w is not None:
        a, b = a * w, b * w
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_apply_equals_single_layout_contexts(L, precision):
    w = workload()
    lay = layouts()
    m = w.medium
    hs = O.order_scale(w.p, m["k2"], m["radius"])
    batch = L.context_for(w, precision)
    batch.set_layouts(lay)
    assert L.load().lsms_num_layouts(batch.h) == 3
    x = np.concatenate([inputs.random_coefficients(len(c), w.p, 1, 50 + i)[0] / hs for i, c in enumerate(lay)])
    flags = L.APPLY_MIXED if precision else 0
    y1 = batch.apply(x, flags)[0]
    y2 = batch.apply(x, flags)[0]          # replayed graph
    off = 0
    tol = 1e-12 if precision == 0 else 1e-6
    for i, c in enumerate(lay):
        ctx = L.context_for(w, precision)
        ctx.set_particles(c)
        ys = ctx.apply(x[off:off + len(c)], flags)[0]
        assert rel(y1[off:off + len(c)], ys, hs) < tol
        assert rel(y2[off:off + len(c)], ys, hs) < tol
        if i == 1:
            lam, wt = O.contour(w.n_nodes, m["k1"], m["k2"], m["k3"], w.b, w.t_max)
            pr = O.Problem(O.Medium(m["k1"], m["k2"], m["k3"], m["d"], m["kp"], m["radius"]), w.p, c, lam, wt)
            assert rel(ys, pr.apply(x[off:off + len(c)]), hs) < (1e-10 if precision == 0 else 2e-5)
        ctx.close()
        off += len(c)
    batch.close()


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-8)])
def test_batch_solve_equals_single_layout_solves(L, precision, tol):
    w = workload()
    lay = layouts()
    m = w.medium
    hs = O.order_scale(w.p, m["k2"], m["radius"])
    batch = L.context_for(w, precision)
    batch.set_layouts(lay)
    beta, info = batch.solve(w.sources, tol=1e-12 if precision == 0 else 1e-10, maxiter=300)
    assert info["status"] == 0
    lam, wt = O.contour(w.n_nodes, m["k1"], m["k2"], m["k3"], w.b, w.t_max)
    med = O.Medium(m["k1"], m["k2"], m["k3"], m["d"], m["kp"], m["radius"])
    off = 0
    for i, c in enumerate(lay):
        pr = O.Problem(med, w.p, c, lam, wt)
        b_o = pr.solve_dense(w.sources[0])
        assert rel(beta[off:off + len(c)], b_o, hs) < tol
        u = batch.eval_field(w.targets, i, L.FIELD_SCATTERED)
        assert rel(u, pr.field_layer1(w.sources[0], b_o, w.targets, "scattered")) < tol
        off += len(c)
    batch.close()


def test_autotune_keeps_results(L):
    w = inputs.WORKLOADS["disc1000_p12_ns512"]
    ctx = L.context_for(w)
    ctx.set_particles(w.centres())
    x = inputs.random_coefficients(w.n, w.p, 1, 3)
    a0 = ctx.translate(x, precision=L.LSMS_MIXED)
    mult = ctx.autotune()
    assert mult > 0
    a1 = ctx.translate(x, precision=L.LSMS_MIXED)
    assert rel(a1, a0) < 1e-5
    ctx.close()
    batch = L.context_for(workload())
    batch.set_layouts(layouts())
    assert batch.autotune() > 0
    batch.close()


def test_batch_rejects_per_step_calls(L):
    batch = L.context_for(workload())
    batch.set_layouts(layouts())
    with pytest.raises(L.LsmsError) as e:
        batch.translate(np.zeros((1, 60, 17)))
    assert e.value.code == -1
    batch.close()
