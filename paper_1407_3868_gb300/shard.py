"""The multiple-scattering operator split by target rows over several GPUs (one rank per GPU).

The paper names a parallel implementation as the next step (Sec. 7).  The operator
y = x - S (T + R) x (Sec. 3.2 Eq. "scattmatrix") splits naturally by target disc: rank q owns a
contiguous block of discs and computes their rows of y.  Per application the only exchange is the
all-gather of the coefficient blocks: the translation rows need every source disc's coefficients
(Lemma 3.1), and the reflected coupling is formed whole on every rank from the gathered vector (its
aggregate over all discs is O(N N_S P), about 50 microseconds at 5000 discs) and its rows taken, so
no second collective is needed for the spectral sums.  The rows come from the library
(lsms_apply_rows_dev); this module holds only the partition and the exchange.

GMRES on the split vectors (`sharded_gmres`): every inner product is the sum over ranks of the local
ones, so each Gram-Schmidt pass costs one all-reduce of the projection coefficients (classical
Gram-Schmidt, two passes) and one for the norm; every rank then holds the same Hessenberg matrix,
the same Givens rotations and the same residual estimate and stops at the same iteration.

Collectives go through torch.distributed (NCCL between GPUs, gloo on the CPU).  Complex tensors are
exchanged as their real views.
"""
from __future__ import annotations

import math

import numpy as np


def row_blocks(n: int, world: int) -> list[tuple[int, int]]:
    """Contiguous blocks (row0, row1) of n discs over world ranks, sizes differing by at most one."""
    if world < 1:
        raise ValueError("world must be >= 1")
    base, extra = divmod(n, world)
    out, r0 = [], 0
    for q in range(world):
        r1 = r0 + base + (1 if q < extra else 0)
        out.append((r0, r1))
        r0 = r1
    return out


def _dist():
    import torch.distributed as dist
    return dist


def all_reduce_sum(t, group=None):
    """Sum of a (complex or real) tensor over the ranks of `group` (a no-op for one rank)."""
    dist = _dist()
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size(group) == 1:
        return t
    import torch
    v = torch.view_as_real(t) if t.is_complex() else t
    dist.all_reduce(v, op=dist.ReduceOp.SUM, group=group)
    return t


class ShardedOperator:
    """Rows row0 .. row1 - 1 of the operator on this rank, applied to vectors split by rows.

    apply_rows(x_full) -> y_rows: the rank's rows of the operator applied to the whole vector
    (torch tensors (nrhs, N, P) -> (nrhs, row1 - row0, P)); `from_context` builds it from a library
    context holding every disc (lsms_apply_rows_dev)."""

    def __init__(self, apply_rows, n: int, P: int, rank: int, world: int, group=None):
        self.apply_rows = apply_rows
        self.n, self.P, self.rank, self.world, self.group = n, P, rank, world, group
        self.blocks = row_blocks(n, world)
        self.row0, self.row1 = self.blocks[rank]
        self.rows = self.row1 - self.row0

    @classmethod
    def from_context(cls, ctx, rank: int, world: int, flags: int = 0, group=None, stream=None):
        """The library's rows (lsms_apply_rows_dev) on this rank's GPU; ctx holds every disc."""
        import torch
        blocks = row_blocks(ctx.n, world)
        r0, r1 = blocks[rank]

        def apply_rows(x_full):
            y = torch.empty((x_full.shape[0], r1 - r0, ctx.P), dtype=x_full.dtype, device=x_full.device)
            ctx.apply_rows_dev(x_full, y, r0, r1, flags, stream)
            return y
        return cls(apply_rows, ctx.n, ctx.P, rank, world, group)

    def gather(self, x_local):
        """The whole vector (nrhs, N, P) from every rank's block (nrhs, rows, P)."""
        import torch
        dist = _dist()
        if self.world == 1:
            return x_local
        m = max(r1 - r0 for r0, r1 in self.blocks)
        nrhs = x_local.shape[0]
        pad = torch.zeros((nrhs, m, self.P), dtype=x_local.dtype, device=x_local.device)
        pad[:, :self.rows] = x_local
        parts = [torch.empty_like(pad) for _ in range(self.world)]
        dist.all_gather([torch.view_as_real(q) for q in parts], torch.view_as_real(pad), group=self.group)
        return torch.cat([parts[q][:, :r1 - r0] for q, (r0, r1) in enumerate(self.blocks)], dim=1)

    def apply(self, x_local):
        """This rank's rows of y = x - S (T + R) x for the split vector x."""
        return self.apply_rows(self.gather(x_local))


def sharded_gmres(op: ShardedOperator, rhs_local, tol: float = 1e-10, maxiter: int = 500, x0_local=None):
    """Unrestarted GMRES (Sec. 3.2) for op x = rhs on vectors split by rows: classical Gram-Schmidt
    with a second pass, Givens rotations, stop when the residual estimate over ||rhs|| <= tol.
    rhs_local: this rank's block, (1, rows, P) or (rows, P).  Returns (x_local, iterations,
    residual history) with x_local shaped like rhs_local."""
    import torch
    shape = rhs_local.shape
    b = rhs_local.reshape(-1)
    dev, dt = b.device, b.dtype
    L = b.numel()

    def gdot(V, w):                                   # V^H w summed over ranks
        return all_reduce_sum(V.conj() @ w, op.group)

    def gnorm(w):
        s = all_reduce_sum(torch.sum((w.conj() * w).real).reshape(1), op.group)
        return float(torch.sqrt(s)[0])

    def apply(v):
        return op.apply(v.reshape(1, op.rows, op.P)).reshape(-1)

    x = torch.zeros(L, dtype=dt, device=dev) if x0_local is None else x0_local.reshape(-1).clone()
    r = b - apply(x) if x0_local is not None else b.clone()
    bnorm = gnorm(b)
    beta0 = gnorm(r)
    hist = [beta0 / bnorm if bnorm > 0 else 0.0]
    if beta0 == 0.0 or hist[0] <= tol:
        return x.reshape(shape), 0, hist
    V = torch.zeros((maxiter + 1, L), dtype=dt, device=dev)
    H = np.zeros((maxiter + 1, maxiter), dtype=complex)
    cs = np.zeros(maxiter, dtype=complex)
    sn = np.zeros(maxiter, dtype=complex)
    g = np.zeros(maxiter + 1, dtype=complex)
    g[0] = beta0
    V[0] = r / beta0
    k = 0
    for k in range(maxiter):
        w = apply(V[k])
        h = gdot(V[:k + 1], w)
        w = w - V[:k + 1].T @ h
        h2 = gdot(V[:k + 1], w)
        w = w - V[:k + 1].T @ h2
        hcol = (h + h2).cpu().numpy()
        hn = gnorm(w)
        H[:k + 1, k] = hcol
        H[k + 1, k] = hn
        if hn > 0.0:
            V[k + 1] = w / hn
        for i in range(k):
            t = cs[i] * H[i, k] + sn[i] * H[i + 1, k]
            H[i + 1, k] = -np.conj(sn[i]) * H[i, k] + np.conj(cs[i]) * H[i + 1, k]
            H[i, k] = t
        a, c = H[k, k], H[k + 1, k]
        rr = math.hypot(abs(a), abs(c))
        cs[k] = np.conj(a / rr) if rr else 1.0
        sn[k] = np.conj(c / rr) if rr else 0.0
        H[k, k] = cs[k] * a + sn[k] * c
        H[k + 1, k] = 0.0
        g[k + 1] = -np.conj(sn[k]) * g[k]
        g[k] = cs[k] * g[k]
        hist.append(abs(g[k + 1]) / bnorm)
        if hist[-1] <= tol or hn == 0.0:
            k += 1
            break
    else:
        k = maxiter
    y = np.linalg.solve(np.triu(H[:k, :k]), g[:k])
    x = x + V[:k].T @ torch.from_numpy(y).to(device=dev, dtype=dt)
    return x.reshape(shape), k, hist
