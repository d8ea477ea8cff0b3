"""GPU parity: every step of the operator, the operator, the solve and the fields, through the C ABI,
against the FP64 oracle on the same seeded inputs.

Norms.  Coefficient errors are measured in the scaled norm in which every order is O(1): outgoing
coefficients beta_n weighted by |H_n(k2 R)|, incoming coefficients alpha_nu weighted by
|S_nu| |H_nu(k2 R)| (the size of the outgoing coefficient they produce).  Tolerances: 1e-10 relative
for the FP64 path, 1e-8 for the mixed path after refinement (the stated targets); the mixed operator
itself (FP32 translation) is checked at 2e-5.
"""

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


def medium_of(w):
    m = w.medium
    return O.Medium(m["k1"], m["k2"], m["k3"], m["d"], m["kp"], m["radius"])


class Case:
    """One workload: library context, oracle problem, weights."""

    def __init__(self, L, w, centres=None, precision=0):
        self.w = w
        self.c = w.centres() if centres is None else np.asarray(centres, dtype=float).reshape(-1, 2)
        m = w.medium
        self.ctx = L.context_for(w, precision)
        self.ctx.set_particles(self.c)
        self.lam, self.wt = O.contour(w.n_nodes, m["k1"], m["k2"], m["k3"], w.b, w.t_max)
        self.pr = O.Problem(medium_of(w), w.p, self.c, self.lam, self.wt)
        self.hs = O.order_scale(w.p, m["k2"], m["radius"])
        self.ws = self.hs * np.abs(self.pr.S)      # weight of incoming coefficients

    def rand_beta(self, seed, nrhs=1):
        b = inputs.random_coefficients(self.c.shape[0], self.w.p, nrhs, seed)
        return b / self.hs[None, None, :]


def rel(a, b, w=None):
    a, b = np.asarray(a), np.asarray(b)
    if w is not None:
        a, b = a * w, b * w
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def ragged_workload(n, p, n_nodes, seed, width=6.0):
    base = inputs.WORKLOADS["disc16_p10_ns256"]
    w = inputs.Workload(f"ragged{n}", n, p, n_nodes, 60.0, -width / 2, width / 2, seed,
                        base.sources, base.targets, 1e-12)
    return w


@pytest.fixture(scope="module")
def small(L):
    return Case(L, inputs.WORKLOADS["disc16_p10_ns256"])


@pytest.fixture(scope="module")
def ragged(L):
    # 37 discs: one full 32-disc source chunk plus a ragged tail; 4 + 1 target tiles
    w = ragged_workload(37, 6, 144, 21, width=14.0)
    return Case(L, w)


# ---------------------------------------------------------------------------------------------
# a0: setup tables
# ---------------------------------------------------------------------------------------------
def test_contour_and_scattering_tables(small):
    lam, wt = small.ctx.contour()
    assert np.max(np.abs(lam - small.lam)) < 1e-12 * small.w.t_max
    assert np.max(np.abs(wt - small.wt)) < 1e-13
    assert np.allclose(small.ctx.scattering(), small.pr.S, rtol=1e-11, atol=0)


# ---------------------------------------------------------------------------------------------
# a2 translation, a3 aggregate, a4 reflection, a5 disaggregate, a8 incident
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("which", ["small", "ragged"])
def test_translation_fp64(which, small, ragged):
    case = small if which == "small" else ragged
    beta = case.rand_beta(1, nrhs=2)
    a = case.ctx.translate(beta)
    for r in range(2):
        a_o = case.pr.translation(beta[r])
        assert rel(a[r], a_o, case.ws) < TOL64


@pytest.mark.parametrize("which", ["small", "ragged"])
def test_translation_mixed(which, small, ragged, L):
    case = small if which == "small" else ragged
    beta = case.rand_beta(2)
    a = case.ctx.translate(beta, precision=L.LSMS_MIXED)[0]
    assert rel(a, case.pr.translation(beta[0]), case.ws) < TOL_MIXED_OP


@pytest.mark.parametrize("which", ["small", "ragged"])
def test_aggregate_reflect_disaggregate(which, small, ragged):
    case = small if which == "small" else ragged
    beta = case.rand_beta(3)
    pp, qm = case.ctx.aggregate(beta)
    pp_o, qm_o = case.pr.aggregate(beta[0])
    assert rel(pp[0], pp_o) < TOL64 and rel(qm[0], qm_o) < TOL64
    sp, sm = case.ctx.reflect(pp_o, qm_o)
    sig_o = case.pr.layer_densities(None, pp_o, qm_o)
    assert rel(sp[0], sig_o[:, 1]) < 1e-12 and rel(sm[0], sig_o[:, 2]) < 1e-12
    a = case.ctx.disaggregate(sig_o[:, 1], sig_o[:, 2])[0]
    a_o = case.pr.disaggregate(sig_o[:, 1], sig_o[:, 2])
    assert rel(a, a_o, case.ws) < TOL64


@pytest.mark.parametrize("which", ["small", "ragged"])
def test_tensor_core_aggregate_and_disaggregate(which, small, ragged, L):
    # split-BF16 (3 planes, 6 products) tcgen05 contractions are FP32-accurate
    case = small if which == "small" else ragged
    beta = case.rand_beta(13, nrhs=2)
    pp, qm = case.ctx.aggregate(beta, precision=L.LSMS_MIXED)
    for r in range(2):
        pp_o, qm_o = case.pr.aggregate(beta[r])
        assert rel(pp[r], pp_o) < 1e-6 and rel(qm[r], qm_o) < 1e-6
    pp_o, qm_o = case.pr.aggregate(beta[0])
    sig_o = case.pr.layer_densities(None, pp_o, qm_o)
    a = case.ctx.disaggregate(sig_o[:, 1], sig_o[:, 2], precision=L.LSMS_MIXED)[0]
    assert rel(a, case.pr.disaggregate(sig_o[:, 1], sig_o[:, 2]), case.ws) < 1e-6
    # the reflected coupling composes both contractions with an FP32 intermediate (P+, Q-)
    aR = case.ctx.apply(beta[:1], L.APPLY_ALPHA | L.APPLY_NO_TRANSLATION | L.APPLY_MIXED)[0]
    assert rel(aR, case.pr.reflection(beta[0]), case.ws) < 4e-6


def test_incident_local_expansion(small):
    src = np.array([[0.0, 1.0], [0.7, 0.4]])
    a = small.ctx.incident(src)
    for s in range(2):
        assert rel(a[s], small.pr.incident_local(src[s]), small.ws) < TOL64


# ---------------------------------------------------------------------------------------------
# a6: the whole operator
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("which", ["small", "ragged"])
def test_apply_fp64(which, small, ragged, L):
    case = small if which == "small" else ragged
    beta = case.rand_beta(4)
    y = case.ctx.apply(beta)[0]
    y_o = case.pr.apply(beta[0])
    assert rel(y, y_o, case.hs) < TOL64
    # scaled basis: y_b = D y_beta for x_b = D x_beta
    yb = case.ctx.apply(beta * case.hs, L.APPLY_SCALED)[0]
    assert rel(yb, y_o * case.hs) < TOL64
    # the parts separately
    aT = case.ctx.apply(beta, L.APPLY_ALPHA | L.APPLY_NO_REFLECTION)[0]
    aR = case.ctx.apply(beta, L.APPLY_ALPHA | L.APPLY_NO_TRANSLATION)[0]
    assert rel(aT, case.pr.translation(beta[0]), case.ws) < TOL64
    assert rel(aR, case.pr.reflection(beta[0]), case.ws) < TOL64


@pytest.mark.parametrize("which", ["small", "ragged"])
def test_apply_mixed(which, small, ragged, L):
    case = small if which == "small" else ragged
    beta = case.rand_beta(5)
    y = case.ctx.apply(beta, L.APPLY_MIXED)[0]
    assert rel(y, case.pr.apply(beta[0]), case.hs) < TOL_MIXED_OP


def test_apply_device_pointers_match_host(small, L):
    import torch
    beta = small.rand_beta(6, nrhs=3)
    x = torch.from_numpy(beta).cuda()
    y = torch.empty_like(x)
    small.ctx.apply_dev(x, y, L.APPLY_SCALED)
    torch.cuda.synchronize()
    y_host = small.ctx.apply(beta, L.APPLY_SCALED)
    assert np.allclose(y.cpu().numpy(), y_host, rtol=0, atol=1e-13 * np.abs(y_host).max())


# ---------------------------------------------------------------------------------------------
# a7 GMRES, a8 RHS, a9 fields
# ---------------------------------------------------------------------------------------------
@pytest.fixture(scope="module")
def small_solution(small):
    src = small.w.sources[0]
    return small.pr.solve_dense(src)


def test_solve_fp64_matches_dense_lu(small, small_solution, L):
    beta, info = small.ctx.solve(small.w.sources, tol=1e-13, maxiter=300, history=300)
    assert info["status"] == 0
    assert rel(beta[0], small_solution, small.hs) < TOL64
    assert info["rel_res_fp64"] < 1e-12
    assert len(info["history"]) == info["iters"]
    for which, name in ((L.FIELD_TOTAL, "total"), (L.FIELD_SCATTERED, "scattered"),
                        (L.FIELD_PARTICLE, "particle")):
        u = small.ctx.eval_field(small.w.targets, 0, which)
        u_o = small.pr.field_layer1(small.w.sources[0], small_solution, small.w.targets, name)
        assert rel(u, u_o) < TOL64, name


def test_solve_mixed_with_refinement(L, small, small_solution):
    w = small.w
    ctx = L.context_for(w, L.LSMS_MIXED)
    ctx.set_particles(small.c)
    beta, info = ctx.solve(w.sources, tol=1e-11, maxiter=300)
    assert info["status"] == 0 and info["outer_iters"] >= 1
    assert rel(beta[0], small_solution, small.hs) < TOL_MIXED
    u = ctx.eval_field(w.targets, 0, L.FIELD_SCATTERED)
    u_o = small.pr.field_layer1(w.sources[0], small_solution, w.targets, "scattered")
    assert rel(u, u_o) < TOL_MIXED
    ctx.close()


SOURCES3 = np.array([[0.0, 1.0], [-1.3, 0.6], [1.7, 1.4]])


@pytest.mark.parametrize("precision,tol", [(0, TOL64), (1, TOL_MIXED)])
def test_solve_several_sources_in_lockstep(L, small, precision, tol):
    w = small.w
    ctx = L.context_for(w, precision)
    ctx.set_particles(small.c)
    beta, info = ctx.solve(SOURCES3, tol=1e-13 if precision == 0 else 1e-11, maxiter=300)
    assert info["status"] == 0
    for s in range(3):
        b_o = small.pr.solve_dense(SOURCES3[s])
        assert rel(beta[s], b_o, small.hs) < tol
        u = ctx.eval_field(w.targets, s, L.FIELD_SCATTERED)
        assert rel(u, small.pr.field_layer1(SOURCES3[s], b_o, w.targets, "scattered")) < tol
    ctx.close()


@pytest.mark.parametrize("nrhs", [4, 6])
def test_translation_mixed_block_of_right_hand_sides(L, small, nrhs):
    # four right-hand sides share each generated Hankel sequence; 6 = 4 + a partial block of 2
    beta = small.rand_beta(21, nrhs=nrhs)
    a = small.ctx.translate(beta, precision=L.LSMS_MIXED)
    a1 = small.ctx.translate(beta[:1], precision=L.LSMS_MIXED)[0]
    for r in range(nrhs):
        assert rel(a[r], small.pr.translation(beta[r]), small.ws) < TOL_MIXED_OP
    assert rel(a[0], a1, small.ws) < 1e-6
    y = small.ctx.apply(beta, L.APPLY_MIXED)
    for r in range(nrhs):
        assert rel(y[r], small.pr.apply(beta[r]), small.hs) < TOL_MIXED_OP


def test_solve_with_initial_guess_and_maxiter_cap(small, small_solution, L):
    # warm start at the solution converges at once; a cap of 2 iterations reports NOT_CONVERGED
    beta, info = small.ctx.solve(small.w.sources, tol=1e-12, maxiter=50, x0=small_solution[None])
    assert info["status"] == 0 and info["iters"] <= 1
    beta2, info2 = small.ctx.solve(small.w.sources, tol=1e-14, maxiter=2, raise_on_error=False)
    assert info2["status"] == -3 and info2["iters"] == 2
    assert np.all(np.isfinite(beta2))


# ---------------------------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------------------------
def test_no_discs_gives_the_layered_response(L):
    w = inputs.WORKLOADS["disc16_p10_ns256"]
    case = Case(L, w, centres=np.zeros((0, 2)))
    beta, info = case.ctx.solve(w.sources, tol=1e-12, maxiter=10)
    assert beta.shape == (1, 0, 21)
    u = case.ctx.eval_field(w.targets, 0, L.FIELD_SCATTERED)
    u_o = case.pr.field_layer1(w.sources[0], None, w.targets, "scattered")
    assert rel(u, u_o) < TOL64
    assert np.allclose(case.ctx.eval_field(w.targets, 0, L.FIELD_PARTICLE), 0.0, atol=1e-300)


@pytest.mark.parametrize("n", [1, 2])
def test_one_and_two_discs(L, n):
    w = ragged_workload(n, 8, 128, 3, width=2.0)
    case = Case(L, w)
    beta = case.rand_beta(7)
    assert rel(case.ctx.apply(beta)[0], case.pr.apply(beta[0]), case.hs) < TOL64
    b, info = case.ctx.solve(w.sources, tol=1e-13, maxiter=100)
    assert rel(b[0], case.pr.solve_dense(w.sources[0]), case.hs) < TOL64


def test_error_codes(L):
    w = inputs.WORKLOADS["disc16_p10_ns256"]
    ctx = L.context_for(w)
    with pytest.raises(L.LsmsError) as e:
        ctx.apply(np.zeros((1, 1, 21)))
    assert e.value.code == -7                     # before set_particles
    with pytest.raises(L.LsmsError) as e:
        ctx.set_particles([[0.0, -1.0], [0.3, -1.0]])
    assert e.value.code == -2                     # overlapping discs
    ctx.set_particles(w.centres())
    with pytest.raises(L.LsmsError) as e:
        ctx.solve([[0.0, -0.5]])
    assert e.value.code == -1                     # source not in layer 1
    with pytest.raises(L.LsmsError) as e:
        ctx.eval_field([[0.0, 1.0]], 3)
    assert e.value.code == -7                     # no solution for that source
    with pytest.raises(L.LsmsError) as e:
        L.Context(-1.0, 3.0, 1.0, 2.0, 2.0, 0.25, 5, 128)
    assert e.value.code == -1
    ctx.close()


# ---------------------------------------------------------------------------------------------
# full-size workloads: sampled rows the oracle computes one by one
# ---------------------------------------------------------------------------------------------
def sampled_rows(n, k=6, seed=0):
    rng = np.random.default_rng(seed)
    return sorted(set([0, n - 1] + list(rng.choice(n, k - 2, replace=False))))


@pytest.mark.parametrize("name", ["disc1000_p12_ns512", "disc5000_p14_ns1024"])
def test_full_size_apply_on_sampled_rows(L, name):
    w = inputs.WORKLOADS[name]
    case = Case(L, w)
    beta = case.rand_beta(11)
    rows = sampled_rows(w.n)
    y64 = case.ctx.apply(beta)[0][rows]
    ymx = case.ctx.apply(beta, L.APPLY_MIXED)[0][rows]
    y_o = case.pr.apply(beta[0], rows=rows)
    assert rel(y64, y_o, case.hs) < TOL64
    assert rel(ymx, y_o, case.hs) < TOL_MIXED_OP
    case.ctx.close()


def test_full_size_solve_satisfies_the_equations_on_sampled_rows(L):
    w = inputs.WORKLOADS["disc1000_p12_ns512"]
    case = Case(L, w)
    beta, info = case.ctx.solve(w.sources, tol=1e-11, maxiter=1000)
    assert info["status"] == 0, info
    rows = sampled_rows(w.n, 8, 1)
    r = case.pr.apply(beta[0], rows=rows) - case.pr.rhs(w.sources[0])[rows]
    rhs = case.pr.rhs(w.sources[0])
    # residual on the sampled rows, relative to the rhs scale (scaled norm)
    assert np.linalg.norm(r * case.hs) / np.linalg.norm(rhs * case.hs) < 1e-9
    ctx_m = L.context_for(w, L.LSMS_MIXED)
    ctx_m.set_particles(case.c)
    beta_m, info_m = ctx_m.solve(w.sources, tol=1e-11, maxiter=1000)
    assert info_m["status"] == 0, info_m
    assert rel(beta_m[0], beta[0], case.hs) < TOL_MIXED
    ctx_m.close()
    case.ctx.close()


def test_fma_probe_is_plausible(L):
    # the benchmark's measured FMA ceilings sit near the derived peaks (152 SMs x 128 FP32 lanes,
    # or x 2 FP64 FMA units, x 2 flop x clock): between a quarter of them and a little above
    import bench
    f32 = bench.fma_probe(False)
    f64 = bench.fma_probe(True)
    assert 0.25 * 80.5 < f32 < 1.1 * 80.5, f32
    assert 0.25 * 1.26 < f64 < 1.1 * 1.26, f64
