"""The operator split by target rows over two ranks (paper_1407_3868_gb300.shard), on the CPU with
the gloo backend and the oracle standing in for each rank's GPU: every rank applies its rows of the
oracle operator to the gathered vector.  Checked: the partition, the split application against the
whole one, and GMRES on the split vectors (all-reduced inner products) against the oracle's dense
LU solution, with both ranks stopping at the same iteration."""
import os
import socket

import numpy as np
import pytest

from paper_1407_3868_gb300 import shard


def test_row_blocks_cover_the_discs_evenly():
    for n, world in ((23, 2), (5000, 8), (3, 4), (0, 2), (7, 1)):
        b = shard.row_blocks(n, world)
        assert len(b) == world and b[0][0] == 0 and b[-1][1] == n
        assert all(b[q][1] == b[q + 1][0] for q in range(world - 1))
        sizes = [r1 - r0 for r0, r1 in b]
        assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.row_blocks(5, 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist

    from oracle import lsms_oracle as O
    from paper_1407_3868_gb300 import inputs
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        m = inputs.MEDIUM
        med = O.Medium(m["k1"], m["k2"], m["k3"], m["d"], m["kp"], m["radius"])
        c = inputs.layout(23, -4.0, 4.0, 8)
        lam, wt = O.contour(96, m["k1"], m["k2"], m["k3"], 0.2, 60.0)
        p = 4
        pr = O.Problem(med, p, c, lam, wt)
        P = 2 * p + 1
        d = O.order_scale(p, m["k2"], m["radius"])
        r0, r1 = shard.row_blocks(pr.N, world)[rank]

        def rows_of(x_full, scaled):
            xf = x_full[0].numpy()
            if scaled:
                y = d[None, :] * pr.apply(xf / d[None, :], rows=range(r0, r1))
            else:
                y = pr.apply(xf, rows=range(r0, r1))
            return torch.from_numpy(np.ascontiguousarray(y))[None]

        op = shard.ShardedOperator(lambda xf: rows_of(xf, False), pr.N, P, rank, world)
        x = inputs.random_coefficients(pr.N, p, 1, 5)[0] / d
        y_local = op.apply(torch.from_numpy(np.ascontiguousarray(x[r0:r1]))[None])[0].numpy()
        y_full = pr.apply(x)
        err_apply = np.abs(y_local - y_full[r0:r1]).max() / np.abs(y_full).max()
        ops = shard.ShardedOperator(lambda xf: rows_of(xf, True), pr.N, P, rank, world)
        src = np.array([0.0, 1.0])
        rhs = d[None, :] * pr.rhs(src)
        xl, iters, hist = shard.sharded_gmres(ops, torch.from_numpy(np.ascontiguousarray(rhs[r0:r1]))[None],
                                              tol=1e-13, maxiter=300)
        beta_local = xl[0].numpy() / d[None, :]
        b_o = pr.solve_dense(src)
        err_solve = np.linalg.norm((beta_local - b_o[r0:r1]) * d) / np.linalg.norm(b_o * d)
        it = torch.tensor([float(iters), -float(iters)])
        dist.all_reduce(it, op=dist.ReduceOp.MAX)
        np.save(os.path.join(out_dir, f"rank{rank}.npy"),
                np.array([err_apply, err_solve, iters, it[0].item(), -it[1].item(), hist[-1]]))
    finally:
        dist.destroy_process_group()


def test_two_ranks_apply_and_solve_like_the_whole_operator(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    for rank in range(world):
        err_apply, err_solve, iters, it_max, it_min, res = np.load(tmp_path / f"rank{rank}.npy")
        assert err_apply < 1e-13, (rank, err_apply)
        assert err_solve < 1e-10, (rank, err_solve)
        assert it_max == it_min == iters and 0 < iters < 300 and res <= 1e-13
