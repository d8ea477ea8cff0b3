"""GPU parity of the tensor-core translation of blocks of right-hand sides (Sec. 3.2 Lemma 3.1
applied to every column; split-BF16 tcgen05 MMAs with FP32 accumulation) against the FP64 oracle,
through the C ABI.

The tensor cores sum in FP32 with less than round-to-nearest accuracy, so the error grows with
the number of MMAs summed in one accumulator; draining every 32 source discs (the default) keeps
it near 6e-6 in the scaled norm (the CUDA-core FP32 path: ~8e-7), inside the mixed-operator
tolerance, and the FP64 refinement of the solve removes it.

The layouts are ragged on purpose: target groups of 16 discs with a partial last group, right-hand
side counts that are not multiples of the 64-column MMA block (40) or span two blocks (72), the
smallest and largest orders the kernel is built for (p = 6 and 15), near pairs (k2 rho < 25, added
by the CUDA-core near-pair kernel) and the self pair.  Tolerances are those of the mixed operator
(2e-5 in the scaled norm) and, after FP64 refinement, of the mixed solve (1e-8).
"""
import numpy as np
import pytest

from oracle import lsms_oracle as O
from paper_1407_3868_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL_MIXED_OP = 2e-5
TOL_MIXED = 1e-8


@pytest.fixture(scope="module")
def L():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1407_3868_gb300 import lsms
    return lsms


def workload(n, p, seed, n_nodes=256, n_src=1):
    h = inputs.widened_half_width(n)
    src = np.stack([np.linspace(-h, h, n_src), np.full(n_src, 1.0)], axis=1)
    return inputs.Workload(f"tc{n}_p{p}", n, p, n_nodes, 141.0, -h, h, seed, src,
                           inputs.observation_points(-h, h, 16, 1.5), 1e-11)


def weights(w):
    m = w.medium
    hs = O.order_scale(w.p, m["k2"], m["radius"])
    return hs, hs * np.abs(O.mie_coefficients(w.p, m["k2"], m["kp"], m["radius"]))


def rel(a, b, wt):
    return np.linalg.norm((a - b) * wt) / np.linalg.norm(b * wt)


@pytest.mark.parametrize("nrhs", [40, 72])
def test_tc_translation_matches_the_oracle_and_the_cuda_core_path(L, nrhs):
    w = workload(300, 12, 41)
    c = w.centres()
    hs, ws = weights(w)
    ctx = L.context_for(w, L.LSMS_MIXED)
    ctx.set_particles(c)
    beta = inputs.random_coefficients(w.n, w.p, nrhs, 7) / hs[None, None, :]
    ctx.set_tc_translation(1)
    a_tc = ctx.translate(beta, precision=L.LSMS_MIXED)
    ctx.set_tc_translation(0)
    a_cc = ctx.translate(beta, precision=L.LSMS_MIXED)
    ctx.close()
    assert np.all(np.isfinite(a_tc))
    for r in sorted({0, 33, nrhs - 1}):
        a_o = O.translate(c, beta[r], w.medium["k2"], w.p)
        e_tc, e_cc = rel(a_tc[r], a_o, ws), rel(a_cc[r], a_o, ws)
        print(f"nrhs {nrhs} r {r}: tensor cores {e_tc:.2e}, CUDA cores {e_cc:.2e}")
        assert e_tc < TOL_MIXED_OP and e_cc < TOL_MIXED_OP, r
    assert rel(a_tc, a_cc, ws) < TOL_MIXED_OP


@pytest.mark.parametrize("p", [6, 15])
def test_tc_translation_smallest_and_largest_order(L, p):
    w = workload(53, p, 43)
    c = w.centres()
    hs, ws = weights(w)
    ctx = L.context_for(w, L.LSMS_MIXED)
    ctx.set_particles(c)
    ctx.set_tc_translation(1)
    beta = inputs.random_coefficients(w.n, p, 16, 9) / hs[None, None, :]
    a = ctx.translate(beta, precision=L.LSMS_MIXED)
    ctx.close()
    for r in (0, 15):
        assert rel(a[r], O.translate(c, beta[r], w.medium["k2"], p), ws) < TOL_MIXED_OP


def test_tc_block_solve_matches_the_oracle(L):
    # 18 sources: the inner mixed GMRES applies the operator to 18 columns at once (tensor cores)
    w = workload(40, 7, 45, n_src=18)
    c = w.centres()
    hs, _ = weights(w)
    m = w.medium
    lam, wt = O.contour(w.n_nodes, m["k1"], m["k2"], m["k3"], w.b, w.t_max)
    pr = O.Problem(O.Medium(m["k1"], m["k2"], m["k3"], m["d"], m["kp"], m["radius"]), w.p, c, lam, wt)
    ctx = L.context_for(w, L.LSMS_MIXED)
    ctx.set_particles(c)
    ctx.set_tc_translation(16)
    beta, info = ctx.solve(w.sources, tol=1e-11, maxiter=400)
    assert info["status"] == 0
    dense = pr.dense_operator()
    for s in (0, 9, 17):
        b_o = np.linalg.solve(dense, pr.rhs(w.sources[s]).ravel()).reshape(w.n, w.p * 2 + 1)
        assert rel(beta[s], b_o, hs[None, :]) < TOL_MIXED, s
        u = ctx.eval_field(w.targets, s, L.FIELD_SCATTERED)
        u_o = pr.field_layer1(w.sources[s], b_o, w.targets, "scattered")
        assert np.linalg.norm(u - u_o) / np.linalg.norm(u_o) < TOL_MIXED, s
    ctx.close()


def test_tc_translation_setting_is_validated(L):
    w = workload(20, 6, 47)
    ctx = L.context_for(w, L.LSMS_MIXED)
    with pytest.raises(L.LsmsError) as e:
        ctx.set_tc_translation(-1)
    assert e.value.code == -1
    ctx.close()
