"""GPU tests of the batched forms: a batch of independent layouts (design sweep) and the autotuner.

A layout batch must give, layout by layout, what a context holding that layout alone gives (same
kernels, so to rounding; in mixed precision the batch translates every layout in one launch, whose
source splits differ), and one of its layouts is also checked against the FP64 oracle.
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


def test_batched_translation_with_ragged_layouts(L):
    # layouts of 1, 63, 64, 65 and 130 discs straddle the 64-target tiles of the one-launch
    # translation; every layout against a context holding it alone, one against the oracle
    w = workload()
    sizes = (65, 1, 130, 64, 63)
    lay = [inputs.layout(n, -0.3 * n - 1.0, 0.3 * n + 1.0, 70 + n) for n in sizes]
    m = w.medium
    hs = O.order_scale(w.p, m["k2"], m["radius"])
    x = np.concatenate([inputs.random_coefficients(len(c), w.p, 1, 80 + i)[0] / hs for i, c in enumerate(lay)])
    with L.context_for(w, L.LSMS_MIXED) as batch:
        batch.set_layouts(lay)
        waves, items = batch.batch_translation()
        assert waves == 4 and items >= sum((n + 63) // 64 for n in sizes)
        y = batch.apply(x, L.APPLY_MIXED)[0]
        y_again = batch.apply(x, L.APPLY_MIXED)[0]
    off = 0
    for i, c in enumerate(lay):
        with L.context_for(w, L.LSMS_MIXED) as ctx:
            ctx.set_particles(c)
            ys = ctx.apply(x[off:off + len(c)], L.APPLY_MIXED)[0]
        assert rel(y[off:off + len(c)], ys, hs) < 1e-6, sizes[i]
        assert rel(y_again[off:off + len(c)], ys, hs) < 1e-6, sizes[i]
        if sizes[i] == 65:
            lam, wt = O.contour(w.n_nodes, m["k1"], m["k2"], m["k3"], w.b, w.t_max)
            pr = O.Problem(O.Medium(m["k1"], m["k2"], m["k3"], m["d"], m["kp"], m["radius"]), w.p, c, lam, wt)
            assert rel(y[off:off + len(c)], pr.apply(x[off:off + len(c)]), hs) < 2e-5
        off += len(c)


def test_batch_with_an_empty_layout(L):
    # a layout without discs contributes nothing and leaves the others (and the one-launch mixed
    # translation of the batch) unchanged
    w = workload()
    m = w.medium
    hs = O.order_scale(w.p, m["k2"], m["radius"])
    lay = [inputs.layout(30, -9.0, 9.0, 91), np.zeros((0, 2)), inputs.layout(20, -6.0, 6.0, 92)]
    x = np.concatenate([inputs.random_coefficients(len(c), w.p, 1, 95 + i)[0] / hs if len(c) else
                        np.zeros((0, 2 * w.p + 1), complex) for i, c in enumerate(lay)])
    for precision, flags in ((0, 0), (1, L.APPLY_MIXED)):
        with L.context_for(w, precision) as batch:
            batch.set_layouts(lay)
            y = batch.apply(x, flags)[0]
        assert y.shape == x.shape
        off = 0
        for c in lay:
            if len(c):
                with L.context_for(w, precision) as ctx:
                    ctx.set_particles(c)
                    ys = ctx.apply(x[off:off + len(c)], flags)[0]
                assert rel(y[off:off + len(c)], ys, hs) < (1e-12 if precision == 0 else 1e-6)
            off += len(c)


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


def test_autotune_keeps_results(L, tmp_path):
    # the tuner picks a tile shape and a split factor; both tile shapes give the same translation
    w = inputs.WORKLOADS["disc1000_p12_ns512"]
    ctx = L.context_for(w)
    ctx.set_particles(w.centres())
    x = inputs.random_coefficients(w.n, w.p, 1, 3)
    a0 = ctx.translate(x, precision=L.LSMS_MIXED)
    (shape, mult), = ctx.autotune()
    assert shape in (0, 1, 2) and mult > 0 and ctx.translation_tuning() == (shape, mult)
    a1 = ctx.translate(x, precision=L.LSMS_MIXED)
    assert rel(a1, a0) < 1e-5
    for s in (0, 1, 2):
        ctx.set_translation_tuning(-1, s, 1.0)
        assert rel(ctx.translate(x, precision=L.LSMS_MIXED), a0) < 1e-5, s
    with pytest.raises(L.LsmsError) as e:
        ctx.set_translation_tuning(-1, 3, 1.0)
    assert e.value.code == -1
    ctx.close()
    # a batch: one tuning per size bucket, stored in a JSON cache and applied again from it
    lay = layouts() + [inputs.layout(150, -45.0, 45.0, 99)]
    cache = str(tmp_path / "tuning.json")
    batch = L.context_for(workload(), L.LSMS_MIXED)
    batch.set_layouts(lay)
    xb = np.concatenate([inputs.random_coefficients(len(c), 8, 1, 60 + i)[0] for i, c in enumerate(lay)])
    y0 = batch.apply(xb, L.APPLY_MIXED)[0]
    t1 = batch.autotune(cache=cache)
    assert len(t1) == len(lay) and all(s in (0, 1, 2) and m > 0 for s, m in t1)
    import json
    table = json.load(open(cache))
    assert all(k.startswith("p8_ns192_b") for k in table) and len(table) >= 2
    batch.set_translation_tuning(-1, 1, 3.0)             # overwrite, then restore from the cache
    t2 = batch.autotune(cache=cache)
    assert t2 == t1
    assert rel(batch.apply(xb, L.APPLY_MIXED)[0], y0) < 1e-5
    batch.autotune()                                     # timed again: also the one-launch translation
    waves, items = batch.batch_translation()
    assert waves in (1, 2, 4, 8) and items > 0
    assert rel(batch.apply(xb, L.APPLY_MIXED)[0], y0) < 1e-5
    batch.close()


def test_batch_rejects_per_step_calls(L):
    batch = L.context_for(workload())
    batch.set_layouts(layouts())
    with pytest.raises(L.LsmsError) as e:
        batch.translate(np.zeros((1, 60, 17)))
    assert e.value.code == -1
    batch.close()
