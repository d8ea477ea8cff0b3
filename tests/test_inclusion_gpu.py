"""GPU parity of inclusions of any shape (Sec. 4): the operator x - S_j (T + R) x with the dense
prototype matrix S of a star-shaped inclusion (Sec. 6 Eq. "par1": five lobes, radius 0.15 +- 0.05
inside enclosing discs of radius 0.25) turned by a seeded angle per particle, S_j = D(-theta_j) S
D(theta_j), against the oracle's Problem with the same matrices.  FP64 (1e-10), mixed operator
(2e-5) and mixed solve (1e-8) tolerances as in the disc tests; batches of layouts carry the matrix
and the angles of every layout."""
import numpy as np
import pytest

from oracle import lsms_oracle as O
from paper_1407_3868_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL_MIXED_OP = 2e-5
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


def medium_of(w):
    m = w.medium
    return O.Medium(m["k1"], m["k2"], m["k3"], m["d"], m["kp"], m["radius"])


def star_matrix(p):
    s, m = inputs.STAR5, inputs.MEDIUM
    return O.inclusion_scattering_matrix(inputs.star_curve(s["a1"], s["a2"], s["a3"], s["n_pts"]), p,
                                         m["k2"], m["kp"])


class Case:
    def __init__(self, L, w, precision=0, seed_theta=11):
        self.w = w
        self.c = w.centres()
        m = w.medium
        self.S = star_matrix(w.p)
        self.theta = inputs.orientations(w.n, seed_theta)
        self.ctx = L.context_for(w, precision)
        self.ctx.set_scattering_matrix(self.S)
        self.ctx.set_particles(self.c)
        self.ctx.set_orientations(self.theta)
        self.lam, self.wt = O.contour(w.n_nodes, m["k1"], m["k2"], m["k3"], w.b, w.t_max)
        self.pr = O.Problem(medium_of(w), w.p, self.c, self.lam, self.wt, smat=self.S, theta=self.theta)
        self.hs = O.order_scale(w.p, m["k2"], m["radius"])


@pytest.fixture(scope="module")
def small(L):
    c = Case(L, inputs.WORKLOADS["disc16_p10_ns256"])
    yield c
    c.ctx.close()


def test_matrix_round_trip_and_reset(L, small):
    assert np.array_equal(small.ctx.scattering_matrix(), small.S)
    assert np.allclose(small.ctx.scattering(), np.diag(small.S), rtol=0, atol=0)


@pytest.mark.parametrize("flags_mixed,tol", [(False, TOL64), (True, TOL_MIXED_OP)])
def test_apply_with_rotated_inclusions(L, small, flags_mixed, tol):
    x = inputs.random_coefficients(small.w.n, small.w.p, 2, 5) / small.hs[None, None, :]
    flags = L.APPLY_MIXED if flags_mixed else 0
    y = small.ctx.apply(x, flags)
    for r in range(2):
        assert rel(y[r], small.pr.apply(x[r]), small.hs) < tol, r


def test_scaled_device_apply_matches_host(L, small):
    import torch
    x = inputs.random_coefficients(small.w.n, small.w.p, 1, 6)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    small.ctx.apply_dev(xd, yd, L.APPLY_SCALED)
    torch.cuda.synchronize()
    # scaled unknowns b = |H| beta: y = b - |H| S_j (T + R)(b / |H|)
    beta = x[0] / small.hs[None, :]
    want = small.hs[None, :] * small.pr.apply(beta)
    assert rel(yd.cpu().numpy()[0], want) < TOL64


@pytest.mark.parametrize("precision,tol", [(0, TOL64), (1, TOL_MIXED)])
def test_solve_and_fields_with_rotated_inclusions(L, small, precision, tol):
    w = small.w
    ctx = L.context_for(w, precision)
    ctx.set_particles(small.c)
    ctx.set_scattering_matrix(small.S)
    ctx.set_orientations(small.theta)
    beta, info = ctx.solve(w.sources, tol=1e-12 if precision == 0 else 1e-11, maxiter=400)
    assert info["status"] == 0
    b_o = small.pr.solve_dense(w.sources[0])
    assert rel(beta[0], b_o, small.hs[None, :]) < tol
    for which, name in ((L.FIELD_SCATTERED, "scattered"), (L.FIELD_PARTICLE, "particle")):
        u = ctx.eval_field(w.targets, 0, which)
        assert rel(u, small.pr.field_layer1(w.sources[0], b_o, w.targets, name)) < tol, name
    ctx.close()


def test_orientations_reset_and_mie_restored(L, small):
    w = small.w
    x = inputs.random_coefficients(w.n, w.p, 1, 8) / small.hs[None, None, :]
    with L.context_for(w) as ctx:
        ctx.set_scattering_matrix(small.S)
        ctx.set_particles(small.c)
        ctx.set_orientations(small.theta)
        ctx.set_particles(small.c)                       # resets the angles to zero
        unrotated = O.Problem(medium_of(w), w.p, small.c, small.lam, small.wt, smat=small.S)
        assert rel(ctx.apply(x)[0], unrotated.apply(x[0]), small.hs) < TOL64
        ctx.set_scattering_matrix(None)                  # back to the disc
        disc = O.Problem(medium_of(w), w.p, small.c, small.lam, small.wt)
        assert rel(ctx.apply(x)[0], disc.apply(x[0]), small.hs) < TOL64
        with pytest.raises(L.LsmsError) as e:
            ctx.set_orientations(np.zeros(w.n + 1))
        assert e.value.code == -1


def test_batch_of_layouts_with_rotated_inclusions(L):
    # two layouts; the matrix set before the layouts, the angles after (one array for both)
    base = inputs.WORKLOADS["disc16_p10_ns256"]
    lay = [inputs.layout(9, -2.0, 2.0, 31), inputs.layout(14, -3.0, 3.0, 32)]
    S = star_matrix(base.p)
    th = inputs.orientations(23, 4)
    m = base.medium
    lam, wt = O.contour(base.n_nodes, m["k1"], m["k2"], m["k3"], base.b, base.t_max)
    hs = O.order_scale(base.p, m["k2"], m["radius"])
    x = inputs.random_coefficients(23, base.p, 1, 9)[0] / hs[None, :]
    with L.context_for(base) as ctx:
        ctx.set_scattering_matrix(S)
        ctx.set_layouts(lay)
        ctx.set_orientations(th)
        y = ctx.apply(x)
        y = y.reshape(23, -1)
        off = 0
        for l, c in enumerate(lay):
            pr = O.Problem(medium_of(base), base.p, c, lam, wt, smat=S, theta=th[off:off + len(c)])
            assert rel(y[off:off + len(c)], pr.apply(x[off:off + len(c)]), hs) < TOL64, l
            off += len(c)


def test_perfectly_conducting_discs(L, small):
    # PEC discs (Sec. 3.1 remark): the library's diagonal through lsms_set_scattering_matrix, solved
    # and compared with the oracle's problem with the same diagonal
    w = small.w
    m = w.medium
    s_pec = L.pec_scattering_diagonal(w.p, m["k2"], m["radius"])
    pr = O.Problem(medium_of(w), w.p, small.c, small.lam, small.wt, smat=np.diag(O.pec_coefficients(w.p, m["k2"],
                                                                                                    m["radius"])))
    with L.context_for(w) as ctx:
        ctx.set_particles(small.c)
        ctx.set_scattering_matrix(np.diag(s_pec))
        beta, info = ctx.solve(w.sources, tol=1e-12, maxiter=400)
        assert info["status"] == 0
        b_o = pr.solve_dense(w.sources[0])
        assert rel(beta[0], b_o, small.hs[None, :]) < TOL64
        u = ctx.eval_field(w.targets, 0, L.FIELD_SCATTERED)
        assert rel(u, pr.field_layer1(w.sources[0], b_o, w.targets, "scattered")) < TOL64


@pytest.mark.parametrize("loss", [0.5, 7.5])
def test_absorbing_discs(L, small, loss):
    # discs with a lossy interior (complex k_p in Sec. 3.1's mode system): the library's diagonal
    # (lsms_scattering_diagonal_c) through lsms_set_scattering_matrix, solved and compared with the
    # oracle's problem built on its own complex-k_p Mie coefficients
    w = small.w
    m = w.medium
    kp = m["kp"] + 1j * loss
    s_abs = L.scattering_diagonal(w.p, m["k2"], kp, m["radius"])
    pr = O.Problem(medium_of(w), w.p, small.c, small.lam, small.wt,
                   smat=np.diag(O.mie_coefficients(w.p, m["k2"], kp, m["radius"])))
    b_o = pr.solve_dense(w.sources[0])
    u_o = pr.field_layer1(w.sources[0], b_o, w.targets, "scattered")
    with L.context_for(w) as ctx:
        ctx.set_particles(small.c)
        ctx.set_scattering_matrix(np.diag(s_abs))
        beta, info = ctx.solve(w.sources, tol=1e-12, maxiter=1000)
        assert info["status"] == 0
        assert rel(beta[0], b_o, small.hs[None, :]) < TOL64
        assert rel(ctx.eval_field(w.targets, 0, L.FIELD_SCATTERED), u_o) < TOL64
        # the same diagonal through lsms_set_scattering_diagonal (the diagonal combine)
        ctx.set_scattering_matrix(None)
        ctx.set_scattering_diagonal(s_abs)
        assert np.array_equal(ctx.scattering(), s_abs)
        beta, info = ctx.solve(w.sources, tol=1e-12, maxiter=1000)
        assert info["status"] == 0
        assert rel(beta[0], b_o, small.hs[None, :]) < TOL64
        assert rel(ctx.eval_field(w.targets, 0, L.FIELD_SCATTERED), u_o) < TOL64
        ctx.set_scattering_diagonal(None)                 # back to the lossless Mie diagonal
        assert np.allclose(ctx.scattering(), O.mie_coefficients(w.p, m["k2"], m["kp"], m["radius"]),
                           rtol=1e-11, atol=0)


def test_absorbing_diagonal_reaches_every_layout(L, small):
    # a batch of two layouts created after lsms_set_scattering_diagonal carries the diagonal
    base = small.w
    m = base.medium
    kp = m["kp"] + 0.5j
    s_abs = L.scattering_diagonal(base.p, m["k2"], kp, m["radius"])
    lay = [inputs.layout(9, -2.0, 2.0, 31), inputs.layout(14, -3.0, 3.0, 32)]
    x = inputs.random_coefficients(23, base.p, 1, 12)[0] / small.hs[None, :]
    with L.context_for(base) as ctx:
        ctx.set_scattering_diagonal(s_abs)
        ctx.set_layouts(lay)
        y = ctx.apply(x).reshape(23, -1)
        off = 0
        for l, c in enumerate(lay):
            pr = O.Problem(medium_of(base), base.p, c, small.lam, small.wt,
                           smat=np.diag(O.mie_coefficients(base.p, m["k2"], kp, m["radius"])))
            assert rel(y[off:off + len(c)], pr.apply(x[off:off + len(c)]), small.hs) < TOL64, l
            off += len(c)


def test_absorbing_rotated_inclusions(L, small):
    # lossy five-lobed inclusions (complex k_p in Muller's system, the library's own matrix from
    # lsms_inclusion_scattering_matrix_c), each turned by its angle: FP64 solve and fields against
    # the oracle's problem built on its own absorbing matrix
    w = small.w
    m = w.medium
    s = inputs.STAR5
    kp = m["kp"] * (1 + 0.3j)
    cur = inputs.star_curve(s["a1"], s["a2"], s["a3"], s["n_pts"])
    S_lib = L.inclusion_scattering_matrix(w.p, m["k2"], kp, m["radius"], cur)
    S_o = O.inclusion_scattering_matrix(cur, w.p, m["k2"], kp)
    pr = O.Problem(medium_of(w), w.p, small.c, small.lam, small.wt, smat=S_o, theta=small.theta)
    with L.context_for(w) as ctx:
        ctx.set_particles(small.c)
        ctx.set_scattering_matrix(S_lib)
        ctx.set_orientations(small.theta)
        beta, info = ctx.solve(w.sources, tol=1e-12, maxiter=400)
        assert info["status"] == 0
        b_o = pr.solve_dense(w.sources[0])
        assert rel(beta[0], b_o, small.hs[None, :]) < TOL64
        u = ctx.eval_field(w.targets, 0, L.FIELD_SCATTERED)
        assert rel(u, pr.field_layer1(w.sources[0], b_o, w.targets, "scattered")) < TOL64
