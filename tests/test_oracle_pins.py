"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test checks one oracle function against a closed form, a table, an invariant of the physics,
a special case that reduces to a textbook result, or brute force on a tiny input.  A plausible
mistake (dropped term, wrong sign or index, transposed operand) in the function fails its test.
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate

from oracle import lsms_oracle as O
from paper_1407_3868_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
MED = inputs.MEDIUM


def medium(k1=None, k2=None, k3=None):
    return O.Medium(k1 or MED["k1"], k2 or MED["k2"], k3 or MED["k3"], MED["d"], MED["kp"],
                    MED["radius"])


def fine_contour(m, n_nodes=3000, t_max=120.0, b=0.2):
    return O.contour(n_nodes, m.k1, m.k2, m.k3, b, t_max)


# ---------------------------------------------------------------------------------------------
# special functions and the branch of gamma
# ---------------------------------------------------------------------------------------------
def test_bessel_table():
    rows = np.loadtxt(os.path.join(GOLDEN, "bessel_table_9_1.txt"))
    for x, j0, j1, y0, y1 in rows:
        assert abs(O.hankel(0, x) - (j0 + 1j * y0)) < 1e-10
        assert abs(O.hankel(1, x) - (j1 + 1j * y1)) < 1e-10
        assert abs(O.bessel(1, x) - j1) < 1e-10


def test_gamma_branch():
    k = 3.0
    lam, _ = O.contour(256, 1.0, k, 2.0, 0.2, 40.0)
    g = O.gamma(lam, k)
    assert np.all(g.real >= 0.0)
    assert np.allclose(g * g, lam * lam - k * k, rtol=1e-13, atol=1e-12)
    # real axis: evanescent above k, outgoing (exp(-gamma |y|) = exp(+i sqrt(k^2 - l^2) |y|)) below
    assert O.gamma(np.array([5.0]), k)[0] == pytest.approx(4.0)
    g_in = O.gamma(np.array([1.0, -1.0]), k)
    assert np.allclose(g_in, -1j * math.sqrt(8.0))


def test_contour_weights_integrate_entire_functions():
    # An entire, decaying integrand integrates to its real-axis value along the deformed path.
    # (k2 > k1, k3 here: first the geometric grading, then the guided-mode panel rule)
    lam, wt = O.contour(512, 1.0, 3.0, 2.0, 0.2, 30.0, graded=True)
    assert np.sum(wt * np.exp(-lam ** 2)) == pytest.approx(math.sqrt(math.pi), rel=1e-13)
    f = lambda z: np.exp(-0.5 * (z - 1.0) ** 2 + 2j * z)
    ref = math.sqrt(2 * math.pi) * np.exp(2j - 2.0)        # Fourier transform of a Gaussian
    assert abs(np.sum(wt * f(lam)) - ref) < 1e-13
    lam_g, wt_g = O.contour(512, 1.0, 3.0, 2.0, 0.2, 30.0)
    assert abs(np.sum(wt_g * f(lam_g)) - ref) < 1e-13
    # reversing Gamma2's orientation (a plausible sign slip) changes the value
    n1 = 16 * ((512 - 16) // 32)
    wt_bad = wt.copy()
    wt_bad[n1:512 - n1] *= -1
    assert abs(np.sum(wt_bad * f(lam)) - ref) > 1e-3


def test_contour_symmetry_and_order():
    lam, wt = O.contour(1024, MED["k1"], MED["k2"], MED["k3"], 9.4e-4, 163.0)
    assert lam.size == 1024
    assert np.allclose(lam, -lam[::-1], rtol=0, atol=1e-13)       # lambda -> -lambda symmetry
    assert np.allclose(wt, wt[::-1], rtol=0, atol=1e-15)
    n1 = 16 * ((1024 - 16) // 32)
    assert np.all(np.diff(lam[n1 + (1024 - 2 * n1):].real) > 0)    # Gamma1 increasing t
    assert np.all(lam[:n1].imag > 0) and np.all(lam[-n1:].imag < 0)


# ---------------------------------------------------------------------------------------------
# Sommerfeld / multipole-to-Sommerfeld (Eq. "sommer", Theorem 5.2)
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("n", [0, 1, 2, -3, 7])
@pytest.mark.parametrize("pt", [(0.7, 0.9), (-1.1, -0.6), (2.5, 0.4)])
def test_m2s_theorem_by_quadrature(n, pt):
    k = 3.0 * math.pi
    m = medium(k, k, k)
    lam, wt = fine_contour(m, 4096, 160.0)
    x, y = pt
    g = O.gamma(lam, k)
    quad = np.sum(wt * O.m2s_factor(n, lam, k, above=y > 0) * np.exp(-g * abs(y) + 1j * lam * x) / g)
    quad /= 4.0 * math.pi
    direct = O.hankel(n, k * math.hypot(x, y)) * np.exp(1j * n * math.atan2(y, x))
    assert abs(quad - direct) <= 1e-11 * abs(direct)


def test_sommerfeld_h0_real_axis_quadrature():
    # The same identity on the undeformed real axis with SciPy's adaptive quadrature
    # (the branch points are integrable singularities): checks the contour-free form of Eq. "sommer".
    k, x, y = 2.0, 0.3, 0.8

    def f(t, part):
        g = O.gamma(np.array([t]), k)[0]
        v = np.exp(-g * y + 1j * t * x) / g / (4 * math.pi)
        return v.real if part == 0 else v.imag

    tot = 0j
    for a, b in ((-60, -k), (-k, k), (k, 60)):
        re = integrate.quad(f, a, b, args=(0,), limit=400, epsabs=1e-12)[0]
        im = integrate.quad(f, a, b, args=(1,), limit=400, epsabs=1e-12)[0]
        tot += re + 1j * im
    direct = 0.25j * O.hankel(0, k * math.hypot(x, y))
    assert abs(tot - direct) < 1e-8


# ---------------------------------------------------------------------------------------------
# Jacobi-Anger (Lemma 5.1, Eq. "JA2") and Graf (Lemma 3.1)
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("downward", [True, False])
def test_jacobi_anger_plane_wave(downward):
    k = 3.0 * math.pi
    lam, _ = O.contour(256, 2.0, k, 4.0, 0.2, 40.0)
    m = np.arange(-80, 81)
    for idx in (3, 100, 130, 200):
        l0 = lam[idx]
        g = O.gamma(l0, k)
        for x, y in ((0.13, -0.21), (-0.2, 0.05)):
            r, th = math.hypot(x, y), math.atan2(y, x)
            direct = np.exp((g if downward else -g) * y + 1j * l0 * x)
            ser = np.sum(O.plane_wave_local_factor(m, l0, k, downward) * O.bessel(m, k * r)
                         * np.exp(1j * m * th))
            assert abs(ser - direct) <= 1e-11 * max(1.0, abs(direct))


def test_graf_translation_against_direct_field():
    k = 3.0 * math.pi
    rng = np.random.default_rng(1)
    p = 8
    for xl, xm in (((0.3, -0.5), (-0.4, -1.2)), ((1.0, -0.4), (0.2, -0.45)), ((0.0, -1.0), (0.0, -0.3))):
        xl, xm = np.array(xl), np.array(xm)
        beta = rng.standard_normal(2 * p + 1) + 1j * rng.standard_normal(2 * p + 1)
        alpha = O.translation_matrix(xl, xm, k, 60, p) @ beta
        nu = np.arange(-60, 61)
        for off in ((0.1, -0.07), (-0.15, 0.1), (0.0, 0.2)):
            pt = xl + np.array(off)
            r, th = math.hypot(*off), math.atan2(off[1], off[0])
            local = np.sum(alpha * O.bessel(nu, k * r) * np.exp(1j * nu * th))
            dm = pt - xm
            n = np.arange(-p, p + 1)
            direct = np.sum(beta * O.hankel(n, k * math.hypot(*dm)) * np.exp(1j * n * math.atan2(dm[1], dm[0])))
            assert abs(local - direct) <= 1e-10 * abs(direct)


def test_reversed_pair_translation_is_the_sign_flipped_one():
    # the identity the unordered-pair kernels rest on: turning the pair's angle by pi multiplies
    # H_s(k rho) e^{i s phi} by (-1)^s, so T^{ml}_{nu n} = (-1)^(n - nu) T^{lm}_{nu n}, i.e.
    # T^{ml} beta = D T^{lm} D beta with D = diag((-1)^k); each direction here is formed on its own
    # (atan2 of its own difference vector)
    k = 3.0 * math.pi
    rng = np.random.default_rng(11)
    p = 10
    sign = (-1.0) ** np.arange(-p, p + 1)
    for _ in range(6):
        xl, xm = rng.uniform(-3.0, 3.0, 2), rng.uniform(-3.0, 3.0, 2)
        t_lm = O.translation_matrix(xl, xm, k, p, p)
        t_ml = O.translation_matrix(xm, xl, k, p, p)
        assert np.max(np.abs(t_ml - sign[:, None] * t_lm * sign[None, :])) <= 1e-12 * np.max(np.abs(t_lm))
        beta = rng.standard_normal(2 * p + 1) + 1j * rng.standard_normal(2 * p + 1)
        assert np.allclose(t_ml @ beta, sign * (t_lm @ (sign * beta)), rtol=1e-12, atol=0.0)


def test_translate_equals_pairwise_brute_force():
    rng = np.random.default_rng(2)
    c = inputs.layout(5, -1.5, 1.5, 7)
    p = 4
    beta = rng.standard_normal((5, 9)) + 1j * rng.standard_normal((5, 9))
    k = 3.0 * math.pi
    fast = O.translate(c, beta, k, p)
    for l in range(5):
        acc = np.zeros(9, dtype=complex)
        for m in range(5):
            if m == l:
                continue
            for a, nu in enumerate(range(-p, p + 1)):
                for b, n in enumerate(range(-p, p + 1)):
                    d = c[l] - c[m]
                    acc[a] += (O.hankel(n - nu, k * math.hypot(*d))
                               * np.exp(1j * (n - nu) * math.atan2(d[1], d[0])) * beta[m, b])
        assert np.allclose(fast[l], acc, rtol=1e-13, atol=0)


# ---------------------------------------------------------------------------------------------
# Disc scattering matrix (Sec. 3.1)
# ---------------------------------------------------------------------------------------------
def test_mie_against_closed_form_and_unitarity():
    k2, kp, R, p = MED["k2"], MED["kp"], MED["radius"], 14
    S = O.mie_coefficients(p, k2, kp, R)
    for n in range(-p, p + 1):
        j2, j2p = O.bessel(n, k2 * R), O.bessel_p(n, k2 * R)
        jp, jpp = O.bessel(n, kp * R), O.bessel_p(n, kp * R)
        h, hp = O.hankel(n, k2 * R), O.hankel_p(n, k2 * R)
        closed = (kp * j2 * jpp - k2 * j2p * jp) / (k2 * hp * jp - kp * jpp * h)
        assert abs(S[n + p] - closed) <= 1e-12 * abs(closed)
    # lossless disc: every partial wave conserves flux, |1 + 2 S_n| = 1
    assert np.allclose(np.abs(1 + 2 * S), 1.0, atol=1e-14)
    assert np.allclose(S, S[::-1], rtol=1e-14, atol=0)                 # S_{-n} = S_n
    assert np.allclose(O.mie_coefficients(5, k2, k2, R), 0.0, atol=1e-15)  # no contrast
    # field continuity on the boundary: exterior J + S H equals the interior gamma_n J_n(kp r)
    for n in (0, 3, -6):
        h, j2 = O.hankel(n, k2 * R), O.bessel(n, k2 * R)
        gam = (j2 + S[n + p] * h) / O.bessel(n, kp * R)
        d_out = k2 * (O.bessel_p(n, k2 * R) + S[n + p] * O.hankel_p(n, k2 * R))
        d_in = gam * kp * O.bessel_p(n, kp * R)
        assert abs(d_out - d_in) <= 1e-12 * abs(d_out)


# ---------------------------------------------------------------------------------------------
# Layered medium (Sec. 2, Eq. "sommerfeldsys")
# ---------------------------------------------------------------------------------------------
def test_particle_free_reflection_is_fresnel_slab():
    m = medium()
    lam, _ = O.contour(256, m.k1, m.k2, m.k3, 0.2, 40.0)
    src = np.array([0.3, 1.0])
    inc = m.incident_density(lam, src)
    sig = m.solve_layers(lam, inc=inc)
    g1, g2, g3 = (O.gamma(lam, k) for k in (m.k1, m.k2, m.k3))
    r12 = (g1 - g2) / (g1 + g2)
    r23 = (g2 - g3) / (g2 + g3)
    e2 = np.exp(-2 * g2 * m.d)
    slab = (r12 + r23 * e2) / (1 + r12 * r23 * e2)                # Airy slab reflection
    assert np.allclose(sig[:, 0] / inc, slab, rtol=1e-12, atol=1e-14)


def test_homogeneous_medium_has_no_layer_response():
    k = 3.0
    m = medium(k, k, k)
    lam, _ = O.contour(128, k, k, k, 0.2, 30.0)
    inc = m.incident_density(lam, np.array([0.0, 1.0]))
    sig = m.solve_layers(lam, inc=inc)
    g = O.gamma(lam, k)
    assert np.allclose(sig[:, 0], 0, atol=1e-13)
    assert np.allclose(sig[:, 1], inc, rtol=1e-13)
    assert np.allclose(sig[:, 2], 0, atol=1e-13)
    assert np.allclose(sig[:, 3], inc * np.exp(-g * m.d), rtol=1e-12, atol=1e-300)
    # and particle sources pass straight through: no reflected density
    sig_p = m.solve_layers(lam, p_plus=np.ones(lam.size), q_minus=np.ones(lam.size))
    assert np.allclose(sig_p[:, 1:3], 0, atol=1e-13)


def test_closed_form_two_interface_response():
    # Unit particle sums through the 4x4 LU against the closed form sigma2+ = R_t (P + R_b e Q)/D,
    # sigma2- = R_b (Q + R_t e P)/D, D = 1 - R_t R_b e^2 (derived independently by hand).
    m = medium()
    lam, _ = O.contour(256, m.k1, m.k2, m.k3, 0.2, 60.0)
    rng = np.random.default_rng(3)
    P = rng.standard_normal(lam.size) + 1j * rng.standard_normal(lam.size)
    Q = rng.standard_normal(lam.size) + 1j * rng.standard_normal(lam.size)
    sig = m.solve_layers(lam, p_plus=P, q_minus=Q)
    g1, g2, g3 = (O.gamma(lam, k) for k in (m.k1, m.k2, m.k3))
    rt, rb = (g2 - g1) / (g2 + g1), (g2 - g3) / (g2 + g3)
    e = np.exp(-g2 * m.d)
    dd = 1 - rt * rb * e * e
    assert np.allclose(sig[:, 1], rt * (P + rb * e * Q) / dd, rtol=1e-12, atol=1e-14)
    assert np.allclose(sig[:, 2], rb * (Q + rt * e * P) / dd, rtol=1e-12, atol=1e-14)


# ---------------------------------------------------------------------------------------------
# The coupled problem (Sec. 5, Eqs. "fullrep", "finalsys", "schur")
# ---------------------------------------------------------------------------------------------
@pytest.fixture(scope="module")
def three_discs():
    m = medium()
    lam, wt = fine_contour(m, 3000, 120.0)
    c = np.array([[0.2, -0.7], [-0.6, -1.3], [0.9, -1.1]])
    pr = O.Problem(m, 6, c, lam, wt)
    src = np.array([0.1, 1.0])
    return pr, src, pr.solve_dense(src)


def test_three_solve_routes_agree(three_discs):
    pr, src, beta = three_discs
    sig, b_block = pr.solve_block(src)
    b_schur = pr.solve_schur(src)
    scale = np.abs(beta).max()
    assert np.abs(b_block - beta).max() <= 1e-12 * scale
    assert np.abs(b_schur - beta).max() <= 1e-12 * scale
    # the block solve's layer densities are the ones the operator form implies
    sig2 = pr.densities(src, beta)
    assert np.allclose(sig, sig2, rtol=1e-10, atol=1e-12 * np.abs(sig).max())


def test_interface_continuity_of_total_field(three_discs):
    pr, src, beta = three_discs
    h = 1e-4
    for x in (-0.5, 0.3, 1.7):
        u1 = lambda y: pr.field_layer1(src, beta, np.array([[x, y]]), "total")[0]
        u2 = lambda y: pr.field_layer2(src, beta, np.array([[x, y]]))[0]
        u3 = lambda y: pr.field_layer3(src, beta, np.array([[x, y]]))[0]
        assert abs(u1(0.0) - u2(0.0)) <= 1e-11 * abs(u1(0.0))
        assert abs(u3(-2.0) - u2(-2.0)) <= 1e-11 * abs(u3(-2.0))
        # one-sided second-order differences for the normal derivative
        d1 = (-3 * u1(0.0) + 4 * u1(h) - u1(2 * h)) / (2 * h)
        d2 = (3 * u2(0.0) - 4 * u2(-h) + u2(-2 * h)) / (2 * h)
        assert abs(d1 - d2) <= 1e-5 * abs(d1)
        d3 = (3 * u3(-2.0) - 4 * u3(-2.0 - h) + u3(-2.0 - 2 * h)) / (2 * h)
        d2b = (-3 * u2(-2.0) + 4 * u2(-2.0 + h) - u2(-2.0 + 2 * h)) / (2 * h)
        assert abs(d3 - d2b) <= 1e-5 * abs(d3)


def test_disc_boundary_conditions_multiple_scattering(three_discs):
    # On each disc boundary the total exterior field has Fourier modes alpha_n J_n + beta_n H_n with
    # alpha the full incoming field; the scattering matrix makes them match an interior field.
    # Check the discrete relation beta = S alpha with alpha from incident + T + R.
    pr, src, beta = three_discs
    alpha = pr.incident_local(src) + pr.translation(beta) + pr.reflection(beta)
    assert np.allclose(beta, pr.S[None, :] * alpha, rtol=1e-10, atol=1e-12 * np.abs(beta).max())


def test_single_disc_homogeneous_contour_route_equals_graf():
    k = 3.0 * math.pi
    m = O.Medium(k, k, k, 2.0, MED["kp"], MED["radius"])
    lam, wt = fine_contour(m, 3000, 120.0)
    c = np.array([[0.35, -0.8]])
    p = 8
    pr = O.Problem(m, p, c, lam, wt)
    src = np.array([-0.4, 1.0])
    a_contour = pr.incident_local(src)[0]
    d = src - c[0]
    n = np.arange(-p, p + 1)
    a_graf = 0.25j * O.hankel(n, k * math.hypot(*d)) * np.exp(-1j * n * math.atan2(d[1], d[0]))
    assert np.allclose(a_contour, a_graf, rtol=1e-10, atol=1e-12)
    beta = pr.solve_dense(src)
    assert np.allclose(beta[0], pr.S * a_graf, rtol=1e-10, atol=1e-16)
    assert np.allclose(pr.reflection(beta), 0.0, atol=1e-14)


def test_homogeneous_particle_field_matches_direct_hankel_sum():
    k = 3.0 * math.pi
    m = O.Medium(k, k, k, 2.0, MED["kp"], MED["radius"])
    lam, wt = fine_contour(m, 3000, 120.0)
    c = np.array([[0.35, -0.8], [-0.5, -1.4]])
    pr = O.Problem(m, 6, c, lam, wt)
    src = np.array([0.0, 1.0])
    beta = pr.solve_dense(src)
    tg = np.array([[-1.0, 1.5], [0.2, 1.5], [1.3, 0.7]])
    u_part = pr.field_layer1(src, beta, tg, "particle")
    direct = np.zeros(len(tg), dtype=complex)
    n = np.arange(-6, 7)
    for j in range(2):
        dd = tg - c[j]
        direct += (O.hankel(n[None, :], k * np.hypot(dd[:, 0], dd[:, 1])[:, None])
                   * np.exp(1j * n[None, :] * np.arctan2(dd[:, 1], dd[:, 0])[:, None])) @ beta[j]
    assert np.allclose(u_part, direct, rtol=1e-10, atol=0)


def test_reciprocity_of_layered_scattering():
    m = medium()
    lam, wt = fine_contour(m, 3000, 120.0)
    c = np.array([[0.2, -0.7], [-0.6, -1.3]])
    pr = O.Problem(m, 6, c, lam, wt)
    a, b = np.array([-0.7, 0.6]), np.array([0.9, 1.1])
    u_ab = pr.field_layer1(a, pr.solve_dense(a), b[None, :], "scattered")[0]
    u_ba = pr.field_layer1(b, pr.solve_dense(b), a[None, :], "scattered")[0]
    assert abs(u_ab - u_ba) <= 1e-6 * abs(u_ab)


def test_energy_flux_balance_for_lossless_media():
    # Lossless layers and discs: the power leaving through y = +-inf equals what the line source
    # emits, 1/4 + Im u^s(x0) (Green's identity around the source; the discs absorb nothing).
    # The fluxes come from the densities on the real axis, Im u^s(x0) from the contour, so the
    # two sides agree to the contour's accuracy only if translation, reflection, the scattering
    # matrix and the solve are all right (a mirrored translation angle or a dropped sigma_2^-
    # term breaks the balance at the 1e-4 level).
    src = np.array([0.3, 1.0])
    m = medium(3 * math.pi, 3 * math.pi, 3 * math.pi)
    lam, wt = O.contour(512, m.k1, m.k2, m.k3, 0.2, 120.0)
    up, down = O.Problem(m, 4, np.zeros((0, 2)), lam, wt).outgoing_power(src, None)
    assert up == pytest.approx(0.125, abs=1e-12) and down == pytest.approx(0.125, abs=1e-12)
    m = medium()
    lam, wt = O.contour(1024, m.k1, m.k2, m.k3, 0.2, 120.0)
    c = np.array([[0.2, -0.7], [-0.6, -1.3], [0.9, -1.0]])
    pr = O.Problem(m, 4, c, lam, wt)
    beta = pr.solve_dense(src)
    up, down = pr.outgoing_power(src, beta)
    u_s = pr.field_layer1(src, beta, src[None, :], "scattered")[0]
    assert abs(up + down - (0.25 + u_s.imag)) < 1e-9 * 0.25


def test_layer_stack_reduces_to_three_layers():
    # Stack (any number of layers) against the pinned three-layer medium: an interface between two
    # layers of equal wavenumber must be invisible.  (a) the disc layer split below the discs;
    # (b) a layer of k_1 inserted above the disc layer (all absolute heights shift by its thickness).
    m = medium()
    p, src = 5, np.array([0.3, 1.0])
    c = np.array([[0.2, -0.7], [-0.6, -1.3], [0.9, -1.0]])          # disc-layer frame
    tg = np.array([[-1.0, 1.5], [0.5, 1.2], [1.5, 2.0]])
    lam, wt = O.contour(512, m.k1, m.k2, m.k3, 0.2, 120.0)
    ref = O.Problem(m, p, c, lam, wt)
    b_ref = ref.solve_dense(src)
    u_ref = ref.field_layer1(src, b_ref, tg, "scattered")
    st = O.Stack([m.k1, m.k2, m.k2, m.k3], [1.6, m.d - 1.6], 2, m.kp, m.radius)
    pa = O.Problem(st, p, c, lam, wt)
    b = pa.solve_dense(src)
    assert np.allclose(b, b_ref, rtol=0, atol=1e-12 * np.abs(b_ref).max())
    assert np.allclose(pa.field_layer1(src, b, tg, "scattered"), u_ref, rtol=0, atol=1e-12 * np.abs(u_ref).max())
    h = 0.8
    st = O.Stack([m.k1, m.k1, m.k2, m.k3], [h, m.d], 3, m.kp, m.radius)
    assert st.depth == h
    pb = O.Problem(st, p, c, lam, wt)
    b = pb.solve_dense(src)
    b2 = ref.solve_dense(src + [0.0, h])
    assert np.allclose(b, b2, rtol=0, atol=1e-12 * np.abs(b2).max())
    u2 = ref.field_layer1(src + [0.0, h], b2, tg + [0.0, h], "scattered")
    assert np.allclose(pb.field_layer1(src, b, tg, "scattered"), u2, rtol=0, atol=1e-12 * np.abs(u2).max())


def test_layer_stack_energy_balance():
    # five lossless layers, discs in the third: the radiated power balance of the energy pin
    ks = [2 * math.pi, 2.6 * math.pi, 3 * math.pi, 3.4 * math.pi, 4 * math.pi]
    st = O.Stack(ks, [0.5, 2.0, 0.7], 3, MED["kp"], MED["radius"])
    lam, wt = O.contour(2048, ks[0], ks[2], ks[-1], 0.2, 120.0, branch_points=ks)
    src = np.array([0.3, 1.0])
    pr = O.Problem(st, 5, np.array([[0.2, -0.7], [-0.6, -1.3], [0.9, -1.0]]), lam, wt)
    beta = pr.solve_dense(src)
    up, down = pr.outgoing_power(src, beta)
    u_s = pr.field_layer1(src, beta, src[None, :], "scattered")[0]
    assert abs(up + down - (0.25 + u_s.imag)) < 1e-9 * 0.25


def test_oracle_gmres_matches_lu():
    m = medium()
    lam, wt = O.contour(256, m.k1, m.k2, m.k3, 0.2, 141.0)
    c = inputs.layout(6, -1.5, 1.5, 11)
    pr = O.Problem(m, 5, c, lam, wt)
    src = np.array([0.0, 1.0])
    beta = pr.solve_dense(src)
    x, it, hist = O.gmres(lambda v: pr.apply(v).ravel(), pr.rhs(src).ravel(), tol=1e-13, maxiter=200)
    assert hist[-1] <= 1e-13
    assert np.allclose(x.reshape(beta.shape), beta, rtol=1e-9, atol=1e-10 * np.abs(beta).max())


# ---------------------------------------------------------------------------------------------
# Inclusions of any smooth shape (Sec. 4): Muller's system, Kress's log quadrature, S matrix
# ---------------------------------------------------------------------------------------------
@pytest.mark.filterwarnings("ignore::scipy.integrate.IntegrationWarning")
def test_kress_log_weights_integrate_the_log_kernel():
    # int_0^2pi ln(4 sin^2((t - tau)/2)) cos(m tau) d tau = -(2 pi / m) cos(m t) (m >= 1), 0 (m = 0)
    n_pts = 32
    w = O.kress_log_weights(n_pts)
    tj = 2 * np.pi * np.arange(n_pts) / n_pts
    for i in (0, 5):
        for m in (0, 1, 4, 15):
            got = np.sum(w[(i - np.arange(n_pts)) % n_pts] * np.cos(m * tj))
            want = 0.0 if m == 0 else -(2 * np.pi / m) * np.cos(m * tj[i])
            assert abs(got - want) < 1e-12, (i, m)
    # a smooth non-polynomial density against adaptive quadrature of the singular integral
    f = lambda s: np.exp(np.cos(s)) * (1 + 0.3 * np.sin(2 * s))
    n_pts = 64
    w = O.kress_log_weights(n_pts)
    tj = 2 * np.pi * np.arange(n_pts) / n_pts
    t0 = tj[3]
    # ln(4 sin^2(u/2)) = 2 ln|u| + ln(4 sin^2(u/2) / u^2), the second smooth for |u| < 2 pi;
    # the log part by QUADPACK's algebraic-logarithmic weights on either side of t0
    q = dict(limit=200, epsabs=1e-14, epsrel=1e-14)
    ref = 2 * (integrate.quad(f, 0, t0, weight="alg-logb", wvar=(0, 0), **q)[0]
               + integrate.quad(f, t0, 2 * np.pi, weight="alg-loga", wvar=(0, 0), **q)[0])
    smooth = lambda s: np.log(4 * np.sin((t0 - s) / 2) ** 2 / (t0 - s) ** 2) if s != t0 else 0.0
    ref += integrate.quad(lambda s: smooth(s) * f(s), 0, 2 * np.pi, points=[t0], **q)[0]
    got = np.sum(w[(3 - np.arange(n_pts)) % n_pts] * f(tj))
    assert abs(got - ref) < 1e-12


@pytest.mark.parametrize("radius,kp", [(0.2, 2.4 * math.pi), (0.25, 1.5 * math.pi), (0.1, 5.0 * math.pi)])
def test_inclusion_matrix_of_a_centred_circle_is_the_mie_diagonal(radius, kp):
    k2, p = MED["k2"], 10
    S = O.inclusion_scattering_matrix(inputs.star_curve(radius, 0.0, 0, 128), p, k2, kp)
    mie = O.mie_coefficients(p, k2, kp, radius)
    assert np.abs(np.diag(S) - mie).max() < 1e-13
    assert np.abs(S - np.diag(np.diag(S))).max() < 1e-13


def test_inclusion_matrix_of_an_off_centre_circle_is_the_translated_mie_matrix():
    # a circle of radius a centred at c: regular waves re-expanded about c, Mie there, outgoing
    # waves re-expanded about the origin (Graf), both addition theorems checked here first
    k2, kp, p, a = MED["k2"], 2.4 * math.pi, 8, 0.12
    c = np.array([0.05, 0.03])
    rc, pc = np.hypot(*c), math.atan2(c[1], c[0])
    x = np.array([0.31, -0.22])
    xr, xth = np.hypot(*x), math.atan2(x[1], x[0])
    xp = x - c
    xpr, xpth = np.hypot(*xp), math.atan2(xp[1], xp[0])
    mm = np.arange(-40, 41)
    for n in (-3, 0, 2):
        lhs = O.bessel(n, k2 * xr) * np.exp(1j * n * xth)
        rhs = np.sum(O.bessel(n - mm, k2 * rc) * np.exp(1j * (n - mm) * pc) * O.bessel(mm, k2 * xpr)
                     * np.exp(1j * mm * xpth))
        assert abs(lhs - rhs) < 1e-13
        lhs = O.hankel(n, k2 * xpr) * np.exp(1j * n * xpth)
        rhs = np.sum(O.bessel(mm - n, k2 * rc) * np.exp(-1j * (mm - n) * pc) * O.hankel(mm, k2 * xr)
                     * np.exp(1j * mm * xth))
        assert abs(lhs - rhs) < 1e-12
    q = 24
    mie = O.mie_coefficients(q, k2, kp, a)
    m = np.arange(-q, q + 1)
    ords = np.arange(-p, p + 1)
    Jin = O.bessel(ords[None, :] - m[:, None], k2 * rc) * np.exp(1j * (ords[None, :] - m[:, None]) * pc)
    Jout = O.bessel(ords[:, None] - m[None, :], k2 * rc) * np.exp(-1j * (ords[:, None] - m[None, :]) * pc)
    want = Jout @ (mie[:, None] * Jin)
    S = O.inclusion_scattering_matrix(inputs.star_curve(a, 0.0, 0, 128, centre=c), p, k2, kp)
    assert np.abs(S - want).max() < 1e-12 * np.abs(want).max()


@pytest.fixture(scope="module")
def star5_matrix():
    k2, kp, p = MED["k2"], MED["kp"], 10
    s = inputs.STAR5
    return O.inclusion_scattering_matrix(inputs.star_curve(s["a1"], s["a2"], s["a3"], 256), p, k2, kp)


def test_inclusion_matrix_symmetries_and_energy(star5_matrix):
    S = star5_matrix
    p = (S.shape[0] - 1) // 2
    l = np.arange(-p, p + 1)
    sg = (-1.0) ** (l[:, None] + l[None, :])
    big = np.abs(S).max()
    # five-fold rotational symmetry: S[l, n] = 0 unless l = n mod 5
    assert np.abs(S[((l[:, None] - l[None, :]) % 5) != 0]).max() < 1e-13 * big
    assert np.abs(S[((l[:, None] - l[None, :]) % 5) == 0]).min() >= 0.0
    # mirror symmetry about the x-axis: S[l, n] = (-1)^(l+n) S[-l, -n]
    assert np.abs(S - sg * S[::-1, ::-1]).max() < 1e-13 * big
    # reciprocity: S[l, n] = (-1)^(l+n) S[-n, -l]
    assert np.abs(S - sg * S[::-1, ::-1].T).max() < 1e-13 * big
    # lossless media: I + 2 S is unitary (outgoing power = incoming power, mode by mode)
    U = np.eye(S.shape[0]) + 2 * S
    assert np.abs(U.conj().T @ U - np.eye(S.shape[0])).max() < 1e-12
    # a genuinely non-circular inclusion couples orders 5 apart
    allowed = (((l[:, None] - l[None, :]) % 5) == 0) & (l[:, None] != l[None, :])
    assert np.abs(S[allowed]).max() > 1e-3 * big


def test_inclusion_matrix_converges_and_rotates(star5_matrix):
    k2, kp, p = MED["k2"], MED["kp"], 10
    s = inputs.STAR5
    S512 = O.inclusion_scattering_matrix(inputs.star_curve(s["a1"], s["a2"], s["a3"], 512), p, k2, kp)
    assert np.abs(S512 - star5_matrix).max() < 1e-12
    th = 0.37
    Sr = O.inclusion_scattering_matrix(inputs.star_curve(s["a1"], s["a2"], s["a3"], 256, rotation=th),
                                       p, k2, kp)
    assert np.abs(Sr - O.rotate_scattering_matrix(star5_matrix, th)).max() < 1e-12
    # a wrong sign in the rotation would be caught: the matrix is not rotation invariant
    assert np.abs(Sr - O.rotate_scattering_matrix(star5_matrix, -th)).max() > 1e-3


def test_problem_with_inclusion_matrices():
    # (i) circles as dense matrices reproduce the disc problem; (ii) rotated star inclusions: the
    # preconditioned system and the block system of Eq. "finalsys" give the same solution
    m = O.Medium(MED["k1"], MED["k2"], MED["k3"], MED["d"], MED["kp"], MED["radius"])
    p, src = 6, np.array([0.1, 1.0])
    c = inputs.layout(5, -1.5, 1.5, 3)
    lam, wt = O.contour(128, m.k1, m.k2, m.k3, 0.2, 80.0)
    disc = O.Problem(m, p, c, lam, wt)
    circ = O.Problem(m, p, c, lam, wt, smat=np.diag(disc.S), theta=inputs.orientations(5, 1))
    x = inputs.random_coefficients(5, p, 1, 2)[0]
    assert np.allclose(circ.apply(x), disc.apply(x), rtol=0, atol=1e-14 * np.abs(x).max())
    s = inputs.STAR5
    S = O.inclusion_scattering_matrix(inputs.star_curve(s["a1"], s["a2"], s["a3"], 128), p, m.k2, m.kp)
    pr = O.Problem(m, p, c, lam, wt, smat=S, theta=inputs.orientations(5, 1))
    b1 = pr.solve_dense(src)
    _, b2 = pr.solve_block(src)
    b3 = pr.solve_schur(src)
    assert np.allclose(b1, b2, rtol=0, atol=1e-11 * np.abs(b1).max())
    assert np.allclose(b1, b3, rtol=0, atol=1e-11 * np.abs(b1).max())
    assert np.abs(b1 - disc.solve_dense(src)).max() > 1e-3 * np.abs(b1).max()


def test_operator_rows_are_the_dense_operator_and_solve_like_the_block_system():
    # the row-by-row assembly (Lemma 3.1 blocks, the reflected coupling as matrices) against the
    # column-by-column matrix of the operator, for discs, rotated inclusions and a five-layer stack;
    # then the independent block system of Eq. "finalsys" solved by LU gives the same beta as LU on
    # the assembled rows (a transposed T block or a dropped reflection term fails both)
    m = O.Medium(MED["k1"], MED["k2"], MED["k3"], MED["d"], MED["kp"], MED["radius"])
    p, src = 5, np.array([0.1, 1.0])
    c = inputs.layout(7, -1.5, 1.5, 4)
    lam, wt = O.contour(128, m.k1, m.k2, m.k3, 0.2, 80.0)
    s = inputs.STAR5
    S = O.inclusion_scattering_matrix(inputs.star_curve(s["a1"], s["a2"], s["a3"], 96), p, m.k2, m.kp)
    st = inputs.STACK5
    stack = O.Stack(st["ks"], st["ds"], st["layer"], MED["kp"], MED["radius"])
    lam5, wt5 = O.contour(128, st["ks"][0], st["ks"][2], st["ks"][-1], 0.2, 80.0)
    probs = [O.Problem(m, p, c, lam, wt),
             O.Problem(m, p, c, lam, wt, smat=S, theta=inputs.orientations(7, 2)),
             O.Problem(stack, p, c, lam5, wt5)]
    for k, pr in enumerate(probs):
        a = pr.dense_operator()
        rows = pr.operator_rows(range(pr.N))
        assert np.abs(rows - a).max() <= 1e-14 * np.abs(a).max(), k
        sub = [5, 0, 6]
        a_sub = a.reshape(pr.N, pr.P, -1)[sub].reshape(len(sub) * pr.P, -1)
        assert np.abs(pr.operator_rows(sub) - a_sub).max() <= 1e-14 * np.abs(a).max(), k
        if k < 2:
            b_rows = np.linalg.solve(rows, pr.rhs(src).ravel()).reshape(pr.N, pr.P)
            _, b_block = pr.solve_block(src)
            assert np.abs(b_rows - b_block).max() <= 1e-11 * np.abs(b_block).max(), k


def test_row_pool_applies_the_operator_over_target_chunks():
    m = O.Medium(MED["k1"], MED["k2"], MED["k3"], MED["d"], MED["kp"], MED["radius"])
    c = inputs.layout(23, -4.0, 4.0, 8)
    lam, wt = O.contour(96, m.k1, m.k2, m.k3, 0.2, 60.0)
    pr = O.Problem(m, 4, c, lam, wt)
    x = inputs.random_coefficients(23, 4, 1, 3)[0]
    y = pr.apply(x)
    with O.RowPool(pr, workers=2, chunks_per_worker=3) as rp:
        assert len(rp.row_chunks()) == 6
        assert np.abs(rp.apply(x) - y).max() <= 1e-13 * np.abs(y).max()
        rows = [22, 1, 9]
        assert np.abs(rp.apply(x, rows=rows) - y[rows]).max() <= 1e-13 * np.abs(y).max()
        blocks = list(rp.iter_operator_rows(chunks=4))
        assert [r for r, _ in blocks][0][0] == 0 and sum(len(r) for r, _ in blocks) == 23
        a = np.concatenate([b for _, b in blocks], axis=0)
        assert np.abs(a @ x.ravel() - y.ravel()).max() <= 1e-12 * np.abs(y).max()


# ---------------------------------------------------------------------------------------------
# Guided-mode media (k2 > k1, k3): poles of the layer response next to the contour
# ---------------------------------------------------------------------------------------------
def _guided_fields(n_nodes, b, graded=False):
    k1, k2, k3, d, kp, R = 1.0, 6.0, 1.0, 3.0, 2.0, 0.25
    m = O.Medium(k1, k2, k3, d, kp, R)
    c = inputs.layout(8, -2.0, 2.0, 5, radius=R, d=d, clearance=0.3)
    src = np.array([0.2, 1.0])
    tg = inputs.observation_points(-3.0, 3.0, 16, 1.5)
    lam, wt = O.contour(n_nodes, k1, k2, k3, b, 40.0, graded=graded)
    pr = O.Problem(m, 6, c, lam, wt)
    beta = pr.solve_dense(src)
    return pr.field_layer1(src, beta, tg, "scattered"), pr.field_layer1(src, beta, tg, "particle")


def test_guided_medium_fields_do_not_depend_on_the_contour():
    # Cauchy: moving Gamma (b, node count) without crossing a pole or branch point leaves every
    # Sommerfeld integral unchanged, so the solved fields must agree between contours; with the
    # poles of the guided modes a distance b below Gamma1 this checks the panel rule as well as
    # the layer response, the coupling and the fields
    ref = _guided_fields(1536, 0.15)
    for n_nodes, b in ((640, 0.3), (768, 0.25), (1024, 0.2)):
        for u, r in zip(_guided_fields(n_nodes, b), ref):
            assert np.linalg.norm(u - r) / np.linalg.norm(r) < 1e-11, (n_nodes, b)
    # the geometric grading (no guided-mode refinement) misses at the same node count
    u, r = _guided_fields(1024, 0.2, graded=True)[0], ref[0]
    assert np.linalg.norm(u - r) / np.linalg.norm(r) > 1e-8


def test_guided_band():
    assert O.guided_band((1.0, 6.0, 1.0)) == (1.0, 6.0)
    assert O.guided_band((1.0, 6.0, 2.0)) == (2.0, 6.0)
    assert O.guided_band((MED["k1"], MED["k2"], MED["k3"])) is None     # k2 < k3: energy leaks down
    assert O.guided_band((1.0, 2.0, 5.0, 3.0, 1.5)) == (1.5, 5.0)


# ---------------------------------------------------------------------------------------------
# Absorbing layers (complex wavenumbers)
# ---------------------------------------------------------------------------------------------
K3_LOSSY = MED["k3"] + 2.0j


def test_lossy_substrate_particle_free_reflection_is_the_airy_slab():
    st = O.Stack([MED["k1"], MED["k2"], K3_LOSSY], [MED["d"]], 2, MED["kp"], MED["radius"])
    lam, _ = O.contour(256, MED["k1"], MED["k2"], MED["k3"], 0.2, 40.0)
    src = np.array([0.3, 1.0])
    inc = st.incident_density(lam, src)
    sig = st.solve_layers(lam, inc=inc)
    g1, g2, g3 = (O.gamma(lam, k) for k in (MED["k1"], MED["k2"], K3_LOSSY))
    assert np.all(g3.real > 0)                                         # decays into the substrate
    r12, r23 = (g1 - g2) / (g1 + g2), (g2 - g3) / (g2 + g3)
    e2 = np.exp(-2 * g2 * MED["d"])
    slab = (r12 + r23 * e2) / (1 + r12 * r23 * e2)
    assert np.allclose(sig[:, 0] / inc, slab, rtol=1e-12, atol=1e-14)
    # the lossless substrate gives another reflection (the loss is felt)
    st0 = O.Stack([MED["k1"], MED["k2"], MED["k3"]], [MED["d"]], 2, MED["kp"], MED["radius"])
    assert np.abs(st0.solve_layers(lam, inc=inc)[:, 0] - sig[:, 0]).max() > 1e-3 * np.abs(sig[:, 0]).max()


def _lossy_fields(n_nodes, b, ks):
    st = O.Stack(ks, [MED["d"]] + [0.9] * (len(ks) - 3), 2, MED["kp"], MED["radius"])
    c = inputs.layout(8, -2.0, 2.0, 5, clearance=0.3)
    src = np.array([0.2, 1.0])
    tg = inputs.observation_points(-3.0, 3.0, 16, 1.5)
    lam, wt = O.contour(n_nodes, MED["k1"], MED["k2"], MED["k3"], b, 50.0,
                        branch_points=[complex(k).real for k in ks])
    pr = O.Problem(st, 6, c, lam, wt)
    return pr.field_layer1(src, pr.solve_dense(src), tg, "scattered")


def test_lossy_fields_do_not_depend_on_the_contour_and_split_layers_are_invisible():
    ks = [MED["k1"], MED["k2"], K3_LOSSY]
    ref = _lossy_fields(3072, 0.15, ks)
    for n_nodes, b in ((1536, 0.25), (2048, 0.3)):
        u = _lossy_fields(n_nodes, b, ks)
        assert np.linalg.norm(u - ref) / np.linalg.norm(ref) < 1e-10, (n_nodes, b)
    # an interface inside the absorbing substrate (equal complex k on both sides) changes nothing
    u4 = _lossy_fields(1536, 0.25, [MED["k1"], MED["k2"], K3_LOSSY, K3_LOSSY])
    assert np.linalg.norm(u4 - ref) / np.linalg.norm(ref) < 1e-10
    # and the loss matters
    u0 = _lossy_fields(1536, 0.25, [MED["k1"], MED["k2"], MED["k3"]])
    assert np.linalg.norm(u0 - ref) / np.linalg.norm(ref) > 1e-2


def test_box_translation_converges_to_the_dense_translation():
    # the far field through box expansions (Graf shifts + Lemma 3.1 between boxes two or more
    # apart) against the all-pairs sum: the error falls geometrically with the box order once it
    # passes k times the box radius (boxes of width 8 and height 2: k r = 38.9)
    k2, p = MED["k2"], 8
    n = 120
    h = inputs.widened_half_width(n)
    c = inputs.layout(n, -h, h, 7)
    hs = O.order_scale(p, k2, MED["radius"])
    beta = inputs.random_coefficients(n, p, 1, 3)[0] / hs[None, :]
    ref = O.translate(c, beta, k2, p)
    ws = hs * np.abs(O.mie_coefficients(p, k2, MED["kp"], MED["radius"]))
    err = lambda a: np.linalg.norm((a - ref) * ws) / np.linalg.norm(ref * ws)
    e50 = err(O.box_translate(c, beta, k2, p, 8.0, 50, -MED["d"] / 2))
    e70 = err(O.box_translate(c, beta, k2, p, 8.0, 70, -MED["d"] / 2))
    assert e70 < 1e-12 < 1e-6 < e50


def test_pec_disc_total_field_vanishes_on_the_boundary():
    # incoming J_n e^{i n theta} plus the scattered S_n H_n e^{i n theta} is zero at r = R for every n,
    # checked by summing a random incoming expansion on points of the circle; the dielectric disc
    # does not satisfy it
    k2, R, p = MED["k2"], MED["radius"], 10
    S = O.pec_coefficients(p, k2, R)
    rng = np.random.default_rng(3)
    alpha = rng.normal(size=2 * p + 1) + 1j * rng.normal(size=2 * p + 1)
    th = np.linspace(0.0, 2 * np.pi, 37)
    n = np.arange(-p, p + 1)
    e = np.exp(1j * np.outer(th, n))
    u = e @ (alpha * (O.bessel(n, k2 * R) + S * O.hankel(n, k2 * R)))
    ref = np.abs(e @ (alpha * O.bessel(n, k2 * R))).max()
    assert np.abs(u).max() < 1e-13 * ref
    # a lossless scatterer: |1 + 2 S_n| = 1
    assert np.allclose(np.abs(1 + 2 * S), 1.0, rtol=0, atol=1e-13)
    Sd = O.mie_coefficients(p, k2, MED["kp"], R)
    u_d = e @ (alpha * (O.bessel(n, k2 * R) + Sd * O.hankel(n, k2 * R)))
    assert np.abs(u_d).max() > 1e-2 * ref


def test_pec_disc_is_the_limit_of_a_good_conductor():
    # a dielectric disc whose interior wavenumber k_p = s (1 + i) has a large imaginary part (a good
    # conductor, skin depth 1/s) tends to the perfectly conducting disc with a gap O(1/s): the gap
    # halves as s doubles and one Richardson step leaves O(1/s^2).  Independent of the PEC formula:
    # the dielectric side solves the pinned 2x2 mode system with complex-argument Bessel functions.
    k2, R, p = MED["k2"], MED["radius"], 10
    pec = O.pec_coefficients(p, k2, R)
    ref = np.abs(pec).max()
    m = {s: O.mie_coefficients(p, k2, s * (1 + 1j), R) for s in (200, 400, 800, 1600)}
    gap = {s: np.abs(m[s] - pec).max() / ref for s in m}
    assert gap[200] < 0.05
    for s in (200, 400, 800):
        assert 1.95 < gap[s] / gap[2 * s] < 2.05
    rich = {s: np.abs(2 * m[2 * s] - m[s] - pec).max() / ref for s in (400, 800)}
    assert rich[800] < 5e-5 and 3.5 < rich[400] / rich[800] < 4.5


@pytest.mark.parametrize("kp", [MED["kp"] + 0.5j, MED["kp"] * (1 + 1j), 300 * (1 + 1j)])
def test_energy_balance_with_absorbing_discs(kp):
    # discs with a lossy or conducting interior (complex k_p) in the lossless three-layer medium: the
    # source's power 1/4 + Im u^s(x0) leaves through y = +-inf or is absorbed inside the discs (the
    # flux of each disc's own expansion, from the Wronskian); lossless discs absorb nothing
    m = O.Medium(MED["k1"], MED["k2"], MED["k3"], MED["d"], kp, MED["radius"])
    c = np.array([[0.1, -0.6], [-0.7, -1.2], [0.8, -1.0]])
    src = np.array([0.3, 0.5])
    lam, wt = O.contour(2048, m.k1, m.k2, m.k3, 0.2, 60.0)
    pr = O.Problem(m, 8, c, lam, wt)
    beta = pr.solve_dense(src)
    absorbed = pr.absorbed_power(src, beta)
    up, down = pr.outgoing_power(src, beta)
    total = 0.25 + pr.field_layer1(src, beta, src[None, :], "scattered")[0].imag
    assert np.all(absorbed > 1e-4)
    assert abs(up + down + absorbed.sum() - total) < 1e-11 * total
    assert abs(up + down - total) > 1e-2 * total
    lossless = O.Problem(O.Medium(MED["k1"], MED["k2"], MED["k3"], MED["d"], MED["kp"], MED["radius"]), 8, c,
                         lam, wt)
    assert np.abs(lossless.absorbed_power(src, lossless.solve_dense(src))).max() < 1e-14


def test_energy_balance_with_perfectly_conducting_discs():
    # PEC discs absorb nothing: radiation through y = +-inf equals the source's power (2e-13), each
    # disc's absorbed power vanishes, and a sign slip in the PEC coefficients breaks the balance
    m = medium()
    c = np.array([[0.1, -0.6], [-0.7, -1.2], [0.8, -1.0]])
    src = np.array([0.3, 0.5])
    lam, wt = O.contour(2048, m.k1, m.k2, m.k3, 0.2, 60.0)
    for sign, ok in ((1.0, True), (-1.0, False)):
        pr = O.Problem(m, 8, c, lam, wt, smat=np.diag(sign * O.pec_coefficients(8, m.k2, m.radius)))
        beta = pr.solve_dense(src)
        up, down = pr.outgoing_power(src, beta)
        total = 0.25 + pr.field_layer1(src, beta, src[None, :], "scattered")[0].imag
        if ok:
            assert abs(up + down - total) < 1e-11 * total
            assert np.abs(pr.absorbed_power(src, beta)).max() < 1e-14
        else:
            assert abs(up + down - total) > 1e-1 * total


@pytest.mark.parametrize("loss", [0.5, 2.0])
def test_energy_balance_with_an_absorbing_substrate(loss):
    # lossless layers 1 and 2 and discs over an absorbing half-space: the source's power
    # 1/4 + Im u^s(x0) leaves upward through y = +inf or crosses into the substrate, where it is
    # absorbed (flux -(1/8pi) int |sigma_3|^2 Im(gamma_3)/|gamma_3|^2 over the whole real axis)
    k3 = MED["k3"] + 1j * loss
    st = O.Stack([MED["k1"], MED["k2"], k3], [MED["d"]], 2, MED["kp"], MED["radius"])
    c = np.array([[0.2, -0.7], [-0.6, -1.3], [0.9, -1.0]])
    src = np.array([0.3, 1.0])
    lam, wt = O.contour(1024, MED["k1"], MED["k2"], MED["k3"], 0.2, 120.0,
                        branch_points=[MED["k1"], MED["k2"], MED["k3"]])
    pr = O.Problem(st, 4, c, lam, wt)
    beta = pr.solve_dense(src)
    up, down = pr.outgoing_power(src, beta)
    u_s = pr.field_layer1(src, beta, src[None, :], "scattered")[0]
    assert up > 0 and down > 0
    assert abs(up + down - (0.25 + u_s.imag)) < 1e-9 * 0.25


@pytest.mark.parametrize("with_discs", [False, True])
def test_energy_balance_in_a_guided_medium(with_discs):
    # k2 above both half-spaces: the source's power 1/4 + Im u^s(x0) (from the contour, which passes
    # a distance b from the guided poles) leaves through y = +-inf (real-axis densities) and along
    # the layer in its guided modes (residues at the real poles)
    k1, k2, k3, d = 1.0, 3.0, 1.5, 1.0
    m = O.Medium(k1, k2, k3, d, 2.0, 0.1)
    assert len(m.guided_poles()) == 1
    src = np.array([0.3, 0.5])
    c = np.array([[0.1, -0.3], [-0.5, -0.7], [0.6, -0.55]]) if with_discs else np.zeros((0, 2))
    lam, wt = O.contour(2048, k1, k2, k3, 0.2, 33.0)
    pr = O.Problem(m, 4, c, lam, wt)
    beta = pr.solve_dense(src) if with_discs else None
    up, down = pr.outgoing_power(src, beta)
    right, left = O.guided_power(pr, src, beta)
    u_s = pr.field_layer1(src, beta, src[None, :], "scattered")[0]
    total = 0.25 + u_s.imag
    assert right > 1e-4 and left > 1e-4
    if not with_discs:
        assert abs(right - left) < 1e-12 * right           # symmetric about the source
    assert abs(up + down + right + left - total) < 1e-10 * total
    # the guided modes are needed: without them the balance misses by their share
    assert abs(up + down - total) > 1e-3 * total


def test_energy_balance_with_many_guided_modes():
    # Sec. 6 Example 1's medium (k = (1, 3, 1), a layer 32 thick): 29 guided modes, the last one
    # 0.0015 below k2; radiation plus the modes' power equals the source's power
    e = inputs.EXAMPLE1
    m = O.Medium(e["k1"], e["k2"], e["k3"], e["d"], e["kp"], e["radius"])
    assert len(m.guided_poles()) == 29
    src = np.array([0.0, 1.0])
    lam, wt = O.contour(2048, e["k1"], e["k2"], e["k3"], 0.2, 33.0)
    pr = O.Problem(m, 4, np.zeros((0, 2)), lam, wt)
    up, down = pr.outgoing_power(src, None)
    right, left = O.guided_power(pr, src, None)
    total = 0.25 + pr.field_layer1(src, None, src[None, :], "scattered")[0].imag
    assert abs(up + down + right + left - total) < 1e-10 * total


@pytest.mark.parametrize("with_discs", [False, True])
def test_energy_balance_in_a_guided_stack(with_discs):
    # four layers (k = 1, 2.5, 3, 1.5), discs in the third: two guided modes, one of them above the
    # second layer's k (evanescent there, so that layer's gamma is continued too); radiation through
    # y = +-inf plus the modes' power equals the source's power
    ks, ds, mi = [1.0, 2.5, 3.0, 1.5], [0.7, 2.0], 3
    st = O.Stack(ks, ds, mi, 2.0, 0.1)
    poles = st.guided_poles()
    assert len(poles) == 2 and ks[1] < poles[1] < ks[2]
    src = np.array([0.3, 0.5])
    c = np.array([[0.1, -0.2], [-0.5, -0.5], [0.6, -0.35]]) if with_discs else np.zeros((0, 2))
    lam, wt = O.contour(2048, ks[0], ks[mi - 1], ks[-1], 0.2, 33.0, branch_points=ks)
    pr = O.Problem(st, 4, c, lam, wt)
    beta = pr.solve_dense(src) if with_discs else None
    up, down = pr.outgoing_power(src, beta)
    right, left = O.guided_power(pr, src, beta)
    total = 0.25 + pr.field_layer1(src, beta, src[None, :], "scattered")[0].imag
    if not with_discs:
        assert abs(right - left) < 1e-12 * right
    assert abs(up + down + right + left - total) < 1e-10 * total
    assert abs(up + down - total) > 1e-2 * total


@pytest.mark.parametrize("kp", [MED["kp"] + 0.5j, MED["kp"] * (1 + 1j), 3 + 23.9j])
def test_absorbing_inclusion_matrix(kp):
    # complex k_p in Muller's system: a centred circle gives the absorbing disc's Mie diagonal (the
    # 2x2 mode system, pinned by the energy balance with absorbing discs); the five-lobed star keeps
    # its selection rule, mirror symmetry and reciprocity, converges in the number of points, and is
    # passive: I - (I + 2S)^H (I + 2S) is positive semidefinite and not zero
    k2, p = MED["k2"], 10
    S = O.inclusion_scattering_matrix(inputs.star_curve(0.2, 0.0, 0, 256), p, k2, kp)
    mie = O.mie_coefficients(p, k2, kp, 0.2)
    assert np.abs(S - np.diag(mie)).max() < 1e-12 * np.abs(mie).max()
    s = inputs.STAR5
    S = O.inclusion_scattering_matrix(inputs.star_curve(s["a1"], s["a2"], s["a3"], 256), p, k2, kp)
    S384 = O.inclusion_scattering_matrix(inputs.star_curve(s["a1"], s["a2"], s["a3"], 384), p, k2, kp)
    big = np.abs(S).max()
    assert np.abs(S384 - S).max() < 1e-12 * big
    l = np.arange(-p, p + 1)
    sg = (-1.0) ** (l[:, None] + l[None, :])
    assert np.abs(S[((l[:, None] - l[None, :]) % 5) != 0]).max() < 1e-13 * big
    assert np.abs(S - sg * S[::-1, ::-1]).max() < 1e-13 * big
    assert np.abs(S - sg * S[::-1, ::-1].T).max() < 1e-13 * big
    U = np.eye(2 * p + 1) + 2 * S
    ev = np.linalg.eigvalsh(np.eye(2 * p + 1) - U.conj().T @ U)
    assert ev.min() > -1e-12 and ev.max() > 1e-2


def test_energy_balance_with_absorbing_rotated_inclusions():
    # lossy five-lobed inclusions, each turned by its own angle, in the three-layer medium: radiation
    # through y = +-inf plus the power each inclusion absorbs (minus the flux of its own expansion)
    # equals the source's power
    s = inputs.STAR5
    m = medium()
    kp = m.kp * (1 + 0.3j)
    S = O.inclusion_scattering_matrix(inputs.star_curve(s["a1"], s["a2"], s["a3"], 128), 6, m.k2, kp)
    c = np.array([[0.2, -0.7], [-0.6, -1.3], [0.9, -1.0]])
    src = np.array([0.3, 1.0])
    lam, wt = O.contour(1024, m.k1, m.k2, m.k3, 0.2, 120.0)
    pr = O.Problem(m, 6, c, lam, wt, smat=S, theta=np.array([0.3, 1.7, 4.0]))
    beta = pr.solve_dense(src)
    up, down = pr.outgoing_power(src, beta)
    absorbed = pr.absorbed_power(src, beta)
    total = 0.25 + pr.field_layer1(src, beta, src[None, :], "scattered")[0].imag
    assert np.all(absorbed > 1e-3)
    assert abs(up + down + absorbed.sum() - total) < 1e-9 * total
    assert abs(up + down - total) > 1e-2 * total


def test_energy_balance_with_rotated_inclusions():
    # lossless five-lobed inclusions (dense scattering matrices, each turned by its own angle) in the
    # three-layer medium: the power through y = +-inf equals the source's power
    s = inputs.STAR5
    m = medium()
    S = O.inclusion_scattering_matrix(inputs.star_curve(s["a1"], s["a2"], s["a3"], 128), 6, m.k2, m.kp)
    c = np.array([[0.2, -0.7], [-0.6, -1.3], [0.9, -1.0]])
    src = np.array([0.3, 1.0])
    lam, wt = O.contour(1024, m.k1, m.k2, m.k3, 0.2, 120.0)
    pr = O.Problem(m, 6, c, lam, wt, smat=S, theta=np.array([0.3, 1.7, 4.0]))
    beta = pr.solve_dense(src)
    up, down = pr.outgoing_power(src, beta)
    u_s = pr.field_layer1(src, beta, src[None, :], "scattered")[0]
    assert abs(up + down - (0.25 + u_s.imag)) < 1e-9 * 0.25


def test_converged_mode_reproduces_the_discrete_sums_and_is_their_limit():
    # converged mode (discretisation studies): its per-node integrands, summed with a contour's own
    # nodes and weights, give Problem's discrete operator, right-hand side and field (scaled); its
    # adaptive integrals over the same truncated contour are what the discrete solutions converge to
    m = medium()
    c = np.array([[0.1, -0.6], [-0.7, -1.2], [0.8, -1.0]])
    src, tg = np.array([0.3, 0.5]), np.array([[0.0, 0.8], [1.0, 1.5], [-2.0, 0.3]])
    p, b, t_max = 3, 0.2, 60.0
    lam, wt = O.contour(256, m.k1, m.k2, m.k3, b, t_max)
    pr = O.Problem(m, p, c, lam, wt)
    N, P = pr.N, pr.P
    hs = np.tile(O.order_scale(p, m.k2, m.radius), N)
    K, r, f, H = O.converged_parts(pr, src, tg, lam)
    R = np.zeros((N * P, N * P), dtype=complex)
    for col in range(N * P):
        e = np.zeros(N * P, dtype=complex)
        e[col] = 1.0 / hs[col]
        R[:, col] = hs * pr.scatter(pr.reflection(e.reshape(N, P))).ravel()
    assert np.abs(np.tensordot(wt, K, axes=1) - R).max() < 1e-14 * np.abs(R).max()
    rhs = hs * pr.rhs(src).ravel()
    assert np.abs(wt @ r - rhs).max() < 1e-14 * np.abs(rhs).max()
    beta = pr.solve_dense(src)
    u = pr.field_layer1(src, beta, tg, "scattered")
    u_parts = wt @ f + np.tensordot(wt, H, axes=1) @ (hs * beta.ravel())
    assert np.abs(u_parts - u).max() < 1e-14 * np.abs(u).max()
    bc, uc = O.converged_solution(pr, src, tg, b, t_max)
    errs = {}
    for ns in (256, 2048):
        lam, wt = O.contour(ns, m.k1, m.k2, m.k3, b, t_max)
        prn = O.Problem(m, p, c, lam, wt)
        bn = prn.solve_dense(src)
        errs[ns] = np.linalg.norm((bn - bc).ravel() * hs) / np.linalg.norm(bc.ravel() * hs)
    assert errs[256] > 1e-6 and errs[2048] < 1e-11


def test_greedy_panel_rule_reaches_the_converged_integral_sooner():
    # the length / (b + distance) panel rule in a medium without guided modes (greedy=True), against
    # converged mode on a narrow three-disc layout: at 768 nodes it is at the converged integral
    # while the geometric grading still misses by 1e-7; at 256 nodes (7 panels a side) they agree
    m = medium()
    c = np.array([[0.1, -0.6], [-0.7, -1.2], [0.8, -1.0]])
    src, tg = np.array([0.3, 0.5]), np.array([[0.0, 0.8], [1.0, 1.5], [-2.0, 0.3]])
    p, b, t_max = 3, 0.2, 60.0
    lam, wt = O.contour(256, m.k1, m.k2, m.k3, b, t_max)
    _, uc = O.converged_solution(O.Problem(m, p, c, lam, wt), src, tg, b, t_max)
    err = {}
    for ns, g in ((256, False), (256, True), (768, False), (768, True)):
        lam, wt = O.contour(ns, m.k1, m.k2, m.k3, b, t_max, greedy=g)
        pr = O.Problem(m, p, c, lam, wt)
        u = pr.field_layer1(src, pr.solve_dense(src), tg, "scattered")
        err[(ns, g)] = np.linalg.norm(u - uc) / np.linalg.norm(uc)
    assert err[(768, True)] < 1e-10 < 1e-8 < err[(768, False)]
    assert abs(err[(256, True)] - err[(256, False)]) < 1e-2 * err[(256, False)]
