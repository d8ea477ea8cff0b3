"""GPU parity of the translation through boxes (lsms_set_fmm: the FMM acceleration named in Sec. 3.2,
with the multipole shifts of Sec. 5.3) against the oracle.

(a) With a low box order the library reproduces the oracle's own box translation (the same
    approximation, the same boxes) to 1e-10, the rounding of its FFT convolution (~4e-12) far below
    the truncation (> 1e-6); (b) at the default order it matches the all-pairs
    translation of Lemma 3.1 to 1e-10 in the scaled norm (the FP64 bar), on layouts of 400, 600 and
    1000 discs with ragged boxes, for several right-hand sides, with box counts whose transform
    length along the boxes splits evenly and unevenly (n1 = A B, A = B or 2B) and a high box order
    whose transform along the orders is 1024 long; (c) the operator and the solves with boxes
    agree with the all-pairs ones; (d) at 50,000 discs (10x the bench layout, 6136 boxes) sampled rows
    match the oracle's row-by-row translation; (e) batches of layouts carry the setting."""
import numpy as np
import pytest

from oracle import lsms_oracle as O
from paper_1407_3868_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL_MIXED = 1e-8


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


def workload(n, p, seed, n_nodes=256):
    h = inputs.widened_half_width(n)
    return inputs.Workload(f"fmm{n}", n, p, n_nodes, 141.0, -h, h, seed, np.array([[0.0, 1.0]]),
                           inputs.observation_points(-h, h, 16, 1.5), 1e-11)


def weights(w):
    m = w.medium
    hs = O.order_scale(w.p, m["k2"], m["radius"])
    return hs, hs * np.abs(O.mie_coefficients(w.p, m["k2"], m["kp"], m["radius"]))


def test_box_translation_equals_the_oracles_box_translation(L):
    w = workload(160, 8, 51)
    c = w.centres()
    hs, ws = weights(w)
    beta = inputs.random_coefficients(w.n, w.p, 1, 2) / hs[None, None, :]
    with L.context_for(w) as ctx:
        ctx.set_particles(c)
        ctx.set_fmm(4.0, 30)                      # deliberately low order: a visible truncation
        nb, q = ctx.fmm_info()
        assert q == 30 and nb >= 10
        a = ctx.translate(beta)[0]
    a_box = O.box_translate(c, beta[0], w.medium["k2"], w.p, 4.0, 30, -w.medium["d"] / 2)
    a_all = O.translate(c, beta[0], w.medium["k2"], w.p)
    assert rel(a_box, a_all, ws) > 1e-6           # the truncation is visible ...
    assert rel(a, a_box, ws) < TOL64              # ... and the library makes the same one (its FFT
                                                  # convolution rounds near 4e-12 relative)


@pytest.mark.parametrize("n,width,nrhs,order", [(400, 4.0, 3, 0), (1000, 6.0, 1, 0), (1000, 3.0, 1, 0),
                                                (600, 3.0, 1, 140)])
def test_box_translation_matches_all_pairs(L, n, width, nrhs, order):
    w = workload(n, 12, 52)
    c = w.centres()
    hs, ws = weights(w)
    beta = inputs.random_coefficients(w.n, w.p, nrhs, 3) / hs[None, None, :]
    with L.context_for(w) as ctx:
        ctx.set_particles(c)
        dense = ctx.translate(beta)
        ctx.set_fmm(width, order)
        nb, q = ctx.fmm_info()
        assert nb >= 3 and (order == 0 or q == order)
        a = ctx.translate(beta)
    for r in range(nrhs):
        assert rel(a[r], dense[r], ws) < TOL64, r
    rows = [0, 1, n // 2, n - 1]
    a_o = O.translate(c, beta[0], w.medium["k2"], w.p, rows=rows)
    assert rel(a[0][rows], a_o, ws) < TOL64


@pytest.mark.parametrize("n,p,width", [(1000, 12, 4.0), (300, 6, 4.0), (400, 8, 2.0)])
def test_mixed_box_translation_matches_all_pairs(L, n, p, width):
    # mixed precision: the adjacent-box pairs in FP32 (pairs with k rho < 25 through the FP64-accurate
    # near-pair tables), the far field through the FP32 boxes; the mixed-operator tolerance 2e-5.
    # Boxes of width 2 are narrower than the near-pair radius 25 / k2 (2.65): some near pairs lie
    # two boxes apart and belong to the far field, not to the near field as well.
    w = workload(n, p, 56)
    c = w.centres()
    hs, ws = weights(w)
    beta = inputs.random_coefficients(w.n, w.p, 2, 7) / hs[None, None, :]
    with L.context_for(w, L.LSMS_MIXED) as ctx:
        ctx.set_particles(c)
        ctx.set_fmm(width)
        a = ctx.translate(beta, precision=L.LSMS_MIXED)
        a64 = ctx.translate(beta, precision=L.LSMS_FP64)
    rows = [0, 3, n // 2, n - 1]
    for r in range(2):
        a_o = O.translate(c, beta[r], w.medium["k2"], w.p, rows=rows)
        assert rel(a[r][rows], a_o, ws) < 2e-5, r
        assert rel(a[r], a64[r], ws) < 2e-5, r


@pytest.mark.parametrize("precision,tol", [(0, TOL64), (1, TOL_MIXED)])
def test_operator_and_solve_with_boxes(L, precision, tol):
    w = workload(600, 10, 53)
    c = w.centres()
    hs, _ = weights(w)
    x = inputs.random_coefficients(w.n, w.p, 1, 4) / hs[None, None, :]
    with L.context_for(w, precision) as ctx:
        ctx.set_particles(c)
        y0 = ctx.apply(x, L.APPLY_MIXED if precision else 0)
        b0, i0 = ctx.solve(w.sources, tol=1e-11, maxiter=1500)
        u0 = ctx.eval_field(w.targets, 0, L.FIELD_SCATTERED)
        ctx.set_fmm(4.0)
        y1 = ctx.apply(x, L.APPLY_MIXED if precision else 0)
        b1, i1 = ctx.solve(w.sources, tol=1e-11, maxiter=1500)
        u1 = ctx.eval_field(w.targets, 0, L.FIELD_SCATTERED)
    assert i0["status"] == 0 and i1["status"] == 0
    assert rel(y1, y0, hs) < (TOL64 if precision == 0 else 2e-5)
    assert rel(b1, b0, hs) < tol and rel(u1, u0) < tol


def test_fifty_thousand_discs_on_sampled_rows(L):
    n, p = 50000, 14
    h = inputs.widened_half_width(n)
    w = inputs.Workload("disc50000_p14_ns1024", n, p, 1024, 163.0, -h, h, 6, np.array([[0.0, 1.0]]),
                        inputs.observation_points(-h, h, 64, 1.5), 1e-8)
    c = w.centres()
    hs, ws = weights(w)
    beta = inputs.random_coefficients(n, p, 1, 5) / hs[None, None, :]
    with L.context_for(w) as ctx:
        ctx.set_particles(c)
        ctx.set_fmm(4.0)
        nb, q = ctx.fmm_info()
        assert nb > 6000 and q == 54
        a = ctx.translate(beta)[0]
    rows = [0, 1, 7, n // 3, n // 2, n - 2, n - 1]
    a_o = O.translate(c, beta[0], w.medium["k2"], p, rows=rows)
    assert rel(a[rows], a_o, ws) < TOL64


def test_batch_of_layouts_with_boxes(L):
    base = workload(300, 8, 54)
    lay = [inputs.layout(150, -40.0, 40.0, 61), inputs.layout(260, -65.0, 65.0, 62)]
    hs, _ = weights(base)
    x = inputs.random_coefficients(410, base.p, 1, 6)[0] / hs[None, :]
    with L.context_for(base) as ctx:
        ctx.set_layouts(lay)
        y_dense = ctx.apply(x)
        ctx.set_fmm(4.0)
        y_box = ctx.apply(x)
    assert rel(y_box, y_dense, hs) < TOL64


def test_box_settings_are_validated(L):
    w = workload(50, 6, 55)
    with L.context_for(w) as ctx:
        for bw, q in ((1.0, 0), (4.0, 3), (4.0, 401), (float("nan"), 0)):
            with pytest.raises(L.LsmsError) as e:
                ctx.set_fmm(bw, q)
            assert e.value.code == -1, (bw, q)
        ctx.set_fmm(0.0)
        assert ctx.fmm_info() == (0, 0)


@pytest.mark.parametrize("case", ["gap", "one_box", "two_boxes", "single"])
def test_box_translation_edge_layouts(L, case):
    # empty boxes in the middle of a layout, a layout inside one or two boxes (no far field at all),
    # a single disc: both precisions against the all-pairs translation
    p = 8
    if case == "gap":
        c = np.concatenate([inputs.layout(40, -60.0, -40.0, 71), inputs.layout(40, 40.0, 60.0, 72)])
    elif case == "one_box":
        c = inputs.layout(6, -1.5, 1.5, 73)
    elif case == "two_boxes":
        c = inputs.layout(10, -3.5, 3.5, 74)
    else:
        c = inputs.layout(1, -1.0, 1.0, 75)
    w = workload(len(c), p, 57)
    hs, ws = weights(w)
    beta = inputs.random_coefficients(len(c), p, 1, 8) / hs[None, None, :]
    with L.context_for(w, L.LSMS_MIXED) as ctx:
        ctx.set_particles(c)
        dense = ctx.translate(beta, precision=L.LSMS_FP64)
        ctx.set_fmm(4.0)
        a64 = ctx.translate(beta, precision=L.LSMS_FP64)
        a32 = ctx.translate(beta, precision=L.LSMS_MIXED)
    if case == "single":
        assert np.all(a64 == 0) and np.all(a32 == 0)
        return
    assert rel(a64, dense, ws) < TOL64
    assert rel(a32, dense, ws) < 2e-5


def test_boxes_with_a_layer_stack_and_rotated_inclusions(L):
    # the box translation inside the five-layer medium (disc layer 0.5 below y = 0) with rotated
    # star inclusions: the operator through boxes equals the all-pairs one, both precisions
    st = inputs.STACK5
    m = inputs.MEDIUM
    n, p = 500, 10
    h = inputs.widened_half_width(n)
    local = inputs.layout(n, -h, h, 81)
    glob = local - np.array([0.0, inputs.STACK5_DEPTH])
    s = inputs.STAR5
    smat = O.inclusion_scattering_matrix(inputs.star_curve(s["a1"], s["a2"], s["a3"], s["n_pts"]), p, m["k2"], m["kp"])
    theta = inputs.orientations(n, 82)
    hs = O.order_scale(p, m["k2"], m["radius"])
    x = inputs.random_coefficients(n, p, 1, 83) / hs[None, None, :]
    for precision, flags, tol in ((0, 0, TOL64), (1, L.APPLY_MIXED, 2e-5)):
        with L.Context(0, 0, 0, 0, m["kp"], m["radius"], p, 512, b=inputs.contour_b(2 * h), t_max=141.0,
                       panel_order=16, precision=precision, stack=(st["ks"], st["ds"], st["layer"])) as ctx:
            ctx.set_particles(glob)
            ctx.set_scattering_matrix(smat)
            ctx.set_orientations(theta)
            y_all = ctx.apply(x, flags)
            ctx.set_fmm(4.0)
            y_box = ctx.apply(x, flags)
        assert rel(y_box, y_all, hs) < tol, precision
