"""Failure detection, with every failure made on the host (no GPU fault, trap or hang).

* Non-finite numbers in what the caller passes (coefficients to lsms_apply / lsms_translate /
  the contour steps, an initial guess, a source, a centre) are refused with LSMS_ERR_ARG before
  any device work.
* Finite inputs whose arithmetic overflows (a scattering diagonal of 1e300) make the solver stop with
  LSMS_ERR_NONFINITE instead of iterating on Inf/NaN.
* A GMRES cap returns LSMS_ERR_NOT_CONVERGED with the iterate.
* Stagnation: a mixed solve asked for a tolerance below what the FP64 residual can reach stops
  refining once its residual has not halved over three refinement steps, and reports
  LSMS_ERR_NOT_CONVERGED ("refinement stagnated") with the best iterate, instead of spending the
  remaining iteration budget.
"""
import numpy as np
import pytest

from oracle import lsms_oracle as O
from paper_1407_3868_gb300 import inputs

pytestmark = pytest.mark.gpu

ARG, NOT_CONVERGED, NONFINITE = -1, -3, -4


@pytest.fixture(scope="module")
def L():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1407_3868_gb300 import lsms
    return lsms


@pytest.fixture(scope="module")
def w():
    return inputs.WORKLOADS["disc16_p10_ns256"]


def message(ctx):
    return ctx.lib.lsms_last_error(ctx.h).decode()


def test_non_finite_inputs_are_refused(L, w):
    ctx = L.context_for(w)
    ctx.set_particles(w.centres())
    P = 2 * w.p + 1
    x = inputs.random_coefficients(w.n, w.p, 2, 5)
    for bad in (np.nan, np.inf, -np.inf):
        xb = x.copy()
        xb[1, 7, 3] = complex(bad, 0.0)
        for call in (lambda: ctx.apply(xb), lambda: ctx.apply(xb, L.APPLY_MIXED),
                     lambda: ctx.translate(xb), lambda: ctx.aggregate(xb)):
            with pytest.raises(L.LsmsError) as e:
                call()
            assert e.value.code == ARG and "non-finite" in str(e.value)
    ns = ctx.contour()[0].size
    s = np.ones(ns, dtype=complex)
    s[ns // 2] = complex(0.0, np.nan)
    with pytest.raises(L.LsmsError) as e:
        ctx.reflect(s, np.ones(ns, dtype=complex))
    assert e.value.code == ARG
    with pytest.raises(L.LsmsError) as e:
        ctx.disaggregate(np.ones(ns, dtype=complex), s)
    assert e.value.code == ARG
    # an initial guess with a NaN, a source at NaN, a centre at Inf
    x0 = np.zeros((1, w.n, P), dtype=complex)
    x0[0, 3, 2] = np.nan
    _, info = ctx.solve(w.sources, tol=1e-10, maxiter=50, x0=x0, raise_on_error=False)
    assert info["status"] == ARG and "initial guess" in message(ctx)
    _, info = ctx.solve([[np.nan, 1.0]], tol=1e-10, maxiter=50, raise_on_error=False)
    assert info["status"] == ARG
    c = w.centres().copy()
    c[4, 0] = np.inf
    with pytest.raises(L.LsmsError) as e:
        ctx.set_particles(c)
    assert e.value.code in (ARG, -2)
    # the context still works afterwards
    ctx.set_particles(w.centres())
    y = ctx.apply(x[:1])
    assert np.all(np.isfinite(y))
    ctx.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_overflow_in_the_iteration_is_reported(L, w, precision):
    ctx = L.context_for(w, precision)
    ctx.set_particles(w.centres())
    ctx.set_scattering_diagonal(np.full(2 * w.p + 1, 1e300 + 0j))      # finite, but overflows
    _, info = ctx.solve(w.sources, tol=1e-10, maxiter=100, raise_on_error=False)
    assert info["status"] == NONFINITE, info
    assert "non-finite" in message(ctx)
    # restoring the Mie diagonal recovers a normal solve on the same context
    ctx.set_scattering_diagonal(None)
    _, info = ctx.solve(w.sources, tol=1e-10, maxiter=300)
    assert info["status"] == 0
    ctx.close()


def test_refinement_stagnation_stops_early_with_the_best_iterate(L, w):
    m = w.medium
    centres = w.centres()
    ctx = L.context_for(w, L.LSMS_MIXED)
    ctx.set_particles(centres)
    beta, info = ctx.solve(w.sources, tol=1e-17, maxiter=4000, raise_on_error=False)
    assert info["status"] == NOT_CONVERGED, info
    assert "stagnated" in message(ctx)
    # it gave up after a few refinement steps at the FP64 floor, far below the iteration budget
    assert info["outer_iters"] <= 10 and info["iters"] < 1000, info
    assert info["rel_res_fp64"] < 1e-13, info
    lam, wt = O.contour(w.n_nodes, m["k1"], m["k2"], m["k3"], w.b, w.t_max)
    pr = O.Problem(O.Medium(m["k1"], m["k2"], m["k3"], m["d"], m["kp"], m["radius"]), w.p, centres, lam, wt)
    b_o = pr.solve_dense(w.sources[0])
    hs = O.order_scale(w.p, m["k2"], m["radius"])
    assert np.linalg.norm((beta[0] - b_o) * hs) / np.linalg.norm(b_o * hs) < 1e-10
    ctx.close()


def test_iteration_cap_returns_the_iterate(L, w):
    ctx = L.context_for(w)
    ctx.set_particles(w.centres())
    beta, info = ctx.solve(w.sources, tol=1e-14, maxiter=3, raise_on_error=False)
    assert info["status"] == NOT_CONVERGED and info["iters"] == 3
    assert "maxiter" in message(ctx)
    assert np.all(np.isfinite(beta)) and np.any(beta != 0)
    ctx.close()
