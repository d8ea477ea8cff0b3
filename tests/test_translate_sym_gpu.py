"""GPU parity of the FP32 translation that generates one Hankel sequence per unordered disc pair
(tile shape 2, the default for one layout) against the FP64 oracle and the two-lanes-per-target
kernel (shape 0), through the C ABI.

Turning the pair's angle by pi gives the reversed pair's sequence, h_s(m <- l) = (-1)^s h_s(l <- m)
(Sec. 3.2 Lemma 3.1), so the kernel contracts each sequence twice: into the target's outputs and,
with the signs (-1)^nu on the coefficients and the outputs, into the source's.  The layouts are
chosen for the kernel's blocking: 16-disc groups with a partial last group (17, 33, 257), a single
partial group (2, 16), diagonal blocks, both rows of a double row (odd and even group counts), near
pairs (k2 rho < 25, left to the near-pair kernel in both directions) and the smallest and largest
orders built.  Tolerances: the mixed operator's 2e-5 in the scaled norm, element by element (the
largest weighted element error over the largest weighted element) as well as over the vector, and
the mixed solve's 1e-8 after FP64 refinement.
"""
import numpy as np
import pytest

from oracle import lsms_oracle as O
from paper_1407_3868_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL_MIXED_OP = 2e-5
TOL_MIXED = 1e-8
SYM = 2


@pytest.fixture(scope="module")
def L():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1407_3868_gb300 import lsms
    return lsms


def workload(n, p, seed, n_nodes=256):
    h = inputs.widened_half_width(n)
    src = np.array([[0.3, 1.0]])
    return inputs.Workload(f"sym{n}_p{p}", n, p, n_nodes, 141.0, -h, h, seed, src,
                           inputs.observation_points(-h, h, 16, 1.5), 1e-11)


def weights(w):
    m = w.medium
    hs = O.order_scale(w.p, m["k2"], m["radius"])
    return hs, hs * np.abs(O.mie_coefficients(w.p, m["k2"], m["kp"], m["radius"]))


def rel(a, b, wt):
    return np.linalg.norm((a - b) * wt) / np.linalg.norm(b * wt)


def relmax(a, b, wt):
    return np.max(np.abs((a - b) * wt)) / np.max(np.abs(b * wt))


def near_pairs(c, k2):
    d = np.hypot(c[:, None, 0] - c[None, :, 0], c[:, None, 1] - c[None, :, 1])
    return int(np.sum((k2 * d < 25.0) & (d > 0)))


@pytest.mark.parametrize("n,p,seed", [(2, 3, 1), (16, 10, 2), (17, 6, 3), (33, 14, 4), (100, 15, 5),
                                      (257, 12, 6)])
def test_symmetric_translation_matches_the_oracle(L, n, p, seed):
    w = workload(n, p, seed)
    c = w.centres()
    hs, ws = weights(w)
    ctx = L.context_for(w, L.LSMS_MIXED)
    ctx.set_particles(c)
    beta = inputs.random_coefficients(w.n, p, 3, 10 + seed) / hs[None, None, :]
    assert ctx.translation_tuning()[0] == SYM            # the default shape
    ctx.set_translation_tuning(-1, 0, 1.0)
    a_h2 = ctx.translate(beta, precision=L.LSMS_MIXED)
    ctx.set_translation_tuning(-1, SYM, 1.0)
    assert ctx.translation_tuning() == (SYM, 1.0)
    a = ctx.translate(beta, precision=L.LSMS_MIXED)
    a1 = ctx.translate(beta[:1], precision=L.LSMS_MIXED)
    ctx.close()
    assert np.all(np.isfinite(a))
    for r in range(3):
        a_o = O.translate(c, beta[r], w.medium["k2"], p)
        e, em = rel(a[r], a_o, ws), relmax(a[r], a_o, ws)
        print(f"n {n} p {p} r {r}: {e:.2e} (elements {em:.2e}), near pairs {near_pairs(c, w.medium['k2'])}")
        assert e < TOL_MIXED_OP and em < TOL_MIXED_OP, r
    assert relmax(a1[0], a[0], ws) < TOL_MIXED_OP
    assert relmax(a, a_h2, ws) < TOL_MIXED_OP


@pytest.mark.parametrize("mult", [1e-4, 1e-3, 1.0])
def test_symmetric_translation_any_run_length(L, mult):
    # the split multiplier sets the run of blocks per warp (300 discs: 19 groups, double rows of 20
    # blocks): runs of a whole double row, of 7 blocks and of one block give the same sums (a row
    # change inside a run flushes the forward outputs)
    w = workload(300, 8, 7)
    c = w.centres()
    hs, ws = weights(w)
    ctx = L.context_for(w, L.LSMS_MIXED)
    ctx.set_particles(c)
    beta = inputs.random_coefficients(w.n, w.p, 1, 77) / hs[None, None, :]
    ctx.set_translation_tuning(-1, SYM, mult)
    a = ctx.translate(beta, precision=L.LSMS_MIXED)[0]
    ctx.close()
    rows = [0, 1, 15, 16, 150, 298, 299]
    a_o = O.translate(c, beta[0], w.medium["k2"], w.p, rows=rows)
    assert relmax(a[rows], a_o, ws) < TOL_MIXED_OP
    assert rel(a[rows], a_o, ws) < TOL_MIXED_OP


def test_symmetric_translation_in_the_mixed_solve(L):
    w = workload(100, 10, 9)
    c = w.centres()
    hs, _ = weights(w)
    m = w.medium
    lam, wt = O.contour(w.n_nodes, m["k1"], m["k2"], m["k3"], w.b, w.t_max)
    pr = O.Problem(O.Medium(m["k1"], m["k2"], m["k3"], m["d"], m["kp"], m["radius"]), w.p, c, lam, wt)
    ctx = L.context_for(w, L.LSMS_MIXED)
    ctx.set_particles(c)
    ctx.set_translation_tuning(-1, SYM, 1.0)
    beta, info = ctx.solve(w.sources, tol=1e-10, maxiter=500)
    ctx.close()
    assert info["status"] == 0, info
    b_o = pr.solve_dense(w.sources[0])
    assert rel(beta[0], b_o, hs) < TOL_MIXED


def test_symmetric_translation_full_size_on_sampled_rows(L):
    w = inputs.WORKLOADS["disc5000_p14_ns1024"]
    c = w.centres()
    hs, ws = weights(w)
    ctx = L.context_for(w, L.LSMS_MIXED)
    ctx.set_particles(c)
    beta = inputs.random_coefficients(w.n, w.p, 1, 5) / hs[None, None, :]
    ctx.set_translation_tuning(-1, 0, 1.0)
    a_h2 = ctx.translate(beta, precision=L.LSMS_MIXED)[0]
    ctx.set_translation_tuning(-1, SYM, 1.0)
    a = ctx.translate(beta, precision=L.LSMS_MIXED)[0]
    ctx.close()
    rng = np.random.default_rng(3)
    rows = sorted({0, 15, 16, w.n - 1, *rng.choice(w.n, 4, replace=False).tolist()})
    a_o = O.translate(c, beta[0], w.medium["k2"], w.p, rows=rows)
    assert relmax(a[rows], a_o, ws) < TOL_MIXED_OP
    assert relmax(a, a_h2, ws) < TOL_MIXED_OP
