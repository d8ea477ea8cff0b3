"""lsms_apply_rows_dev, the block of the operator one GPU owns when the discs are split by rows: on
one GPU every block (ragged, empty, the whole range) equals the same rows of the whole application,
in FP64 and in mixed precision, for discs and rotated inclusions; the blocks of a two-rank split put
together equal the whole operator; and GMRES on split vectors driven by the library's rows
(one rank) reproduces the library's own solve and the oracle."""
import numpy as np
import pytest

from oracle import lsms_oracle as O
from paper_1407_3868_gb300 import inputs, shard

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1407_3868_gb300 import lsms
    return lsms


def rel(a, b, w):
    return np.linalg.norm((a - b) * w) / np.linalg.norm(b * w)


@pytest.mark.parametrize("dense", [False, True])
def test_row_blocks_equal_the_whole_application(L, dense):
    import torch
    w = inputs.Workload("ragged150", 150, 8, 192, 60.0, -40.0, 40.0, 12, np.array([[0.0, 1.0]]),
                        inputs.observation_points(-40.0, 40.0, 8, 1.5), 1e-10)
    m = w.medium
    hs = O.order_scale(w.p, m["k2"], m["radius"])
    ctx = L.context_for(w, L.LSMS_MIXED)
    ctx.set_particles(w.centres())
    if dense:
        s = inputs.STAR5
        smat = L.inclusion_scattering_matrix(w.p, m["k2"], m["kp"], m["radius"],
                                             inputs.star_curve(s["a1"], s["a2"], s["a3"], 128))
        ctx.set_scattering_matrix(smat)
        ctx.set_orientations(inputs.orientations(w.n, 4))
    x = torch.from_numpy(inputs.random_coefficients(w.n, w.p, 2, 9)).cuda()
    for flags, tol in ((L.APPLY_SCALED, 1e-13), (L.APPLY_SCALED | L.APPLY_MIXED, 1e-6),
                       (L.APPLY_SCALED | L.APPLY_ALPHA, 1e-13), (L.APPLY_SCALED | L.APPLY_NO_REFLECTION, 1e-13)):
        y = torch.empty_like(x)
        ctx.apply_dev(x, y, flags)
        full = y.cpu().numpy()
        for r0, r1 in ((0, w.n), (5, 71), (w.n - 3, w.n), (40, 40), (0, 1)):
            yr = torch.empty((2, r1 - r0, w.p * 2 + 1), dtype=x.dtype, device=x.device)
            ctx.apply_rows_dev(x, yr, r0, r1, flags)
            torch.cuda.synchronize()
            if r1 > r0:
                assert rel(yr.cpu().numpy(), full[:, r0:r1], 1.0) < tol, (flags, r0, r1)
        parts = []
        for r0, r1 in shard.row_blocks(w.n, 2):
            yr = torch.empty((2, r1 - r0, w.p * 2 + 1), dtype=x.dtype, device=x.device)
            ctx.apply_rows_dev(x, yr, r0, r1, flags)
            parts.append(yr.cpu().numpy())
        assert rel(np.concatenate(parts, axis=1), full, 1.0) < tol, flags
    with pytest.raises(L.LsmsError) as e:              # a block past the last disc
        ctx.apply_rows_dev(x, torch.empty((2, w.n - 9, 2 * w.p + 1), dtype=x.dtype, device=x.device), 10, w.n + 1)
    assert e.value.code == -1
    ctx.close()


def test_gmres_on_split_vectors_with_the_library_rows(L):
    import torch
    w = inputs.WORKLOADS["disc16_p10_ns256"]
    m = w.medium
    hs = O.order_scale(w.p, m["k2"], m["radius"])
    ctx = L.context_for(w)
    centres = w.centres()
    ctx.set_particles(centres)
    op = shard.ShardedOperator.from_context(ctx, 0, 1, L.APPLY_SCALED)
    beta_lib, info = ctx.solve(w.sources, tol=1e-13, maxiter=300)
    a_inc = ctx.incident(w.sources)[0]
    rhs = hs[None, :] * ctx.scattering()[None, :] * a_inc            # D S a_inc, the scaled system
    xb, iters, hist = shard.sharded_gmres(op, torch.from_numpy(rhs[None]).cuda(), tol=1e-13, maxiter=300)
    beta = xb[0].cpu().numpy() / hs[None, :]
    lam, wt = O.contour(w.n_nodes, m["k1"], m["k2"], m["k3"], w.b, w.t_max)
    pr = O.Problem(O.Medium(m["k1"], m["k2"], m["k3"], m["d"], m["kp"], m["radius"]), w.p, centres, lam, wt)
    b_o = pr.solve_dense(w.sources[0])
    assert rel(beta, b_o, hs) < 1e-10
    assert rel(beta, beta_lib[0], hs) < 1e-10
    assert abs(iters - info["iters"]) <= 2
    ctx.close()
