"""FP64 CPU oracle for multi-particle scattering in a layered medium.

TEST INFRASTRUCTURE.  Only the test suite, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this module.  The CUDA library never calls it
and shares no code with it: special functions come from SciPy (AMOS), Gauss-Legendre rules from
NumPy, and the interface systems are solved by LAPACK LU (no FFT anywhere: every sum is written out).

It computes, plainly and slowly, what the paper defines (Lai, Kobayashi, Greengard, "A fast solver
for multi-particle scattering in a layered medium"):

* the Sommerfeld representation of the fields in the three layers (Sec. 2, Eqs. "layer1",
  "layer21", "layer22", "layer3") and the 4x4 mode-by-mode interface system A_lambda
  (Eq. "sommerfeldsys") (``Medium``); any number of layers, absorbing ones included, by the same
  continuity conditions at every interface (``Stack``; the extension Sec. 1 names);
* the discretised Sommerfeld contour of Sec. 5.1 (``contour``), with its panels placed around the
  branch points and, where an interior layer guides waves, around the real poles
  (``contour_panel_breaks``, ``guided_band``);
* the scattering matrix of a dielectric disc from its 2x2 mode system (Sec. 3.1, Eq. "linear"),
  lossless or absorbing (complex k_p), and of a perfectly conducting disc (``pec_coefficients``);
* the scattering matrix of an inclusion of any smooth shape from Muller's second-kind system
  (Sec. 4, Eqs. "intg1", "intg2"), discretised by Nystrom with Kress's product rule for the
  logarithmic singularities, and its rotated copies (Sec. 4.1);
* Graf's multipole-to-local translation (Sec. 3.2, Lemma 3.1 / Eq. "trans"), all pairs or through
  one level of boxes (``box_translate``: shift to box centres, box-to-box Graf translation, shift
  back);
* the multipole-to-Sommerfeld map (Sec. 5.3, Theorem 5.2) and the Sommerfeld-to-local map by
  Jacobi-Anger (Sec. 5.2.1, Lemma 5.1, Eq. "JA2");
* the block system [A B; C D] (Eq. "finalsys"), its Schur complement (Eq. "schur") and the
  preconditioned operator I - S(T + R) (Sec. 3.2, Eq. "scattmatrix" and the remark after it),
  solved densely or by GMRES;
* the fields in every layer, and two checks that need no reference solution: the power radiated
  through y = +-inf (``Problem.outgoing_power``, Parseval on the real axis) and the power the
  guided modes carry along the layers (``guided_power``, residues at the real poles), which
  together with the power absorbed inside lossy particles (``Problem.absorbed_power``) equal the
  power the source emits.
* converged mode for discretisation studies: every contour sum replaced by its adaptive integral
  over the same truncated contour (``converged_parts``, ``converged_solution``).

Readings of the paper taken here (each is listed in the design notes with its reason):

* time dependence exp(-i w t): H^(1) is outgoing (Sec. 1 states exp(i w t), but every formula
  that follows fits exp(-i w t));
* gamma_i(lambda) = sqrt(lambda^2 - k_i^2) with Re gamma >= 0, computed as
  -i * sqrt(k_i^2 - lambda^2) with the principal square root (Sec. 2 Remark, Sec. 5.1);
* the contour of Eq. "sommerseg" runs Gamma3 -> Gamma2 -> Gamma1; on Gamma2 d lambda = i ds with
  s running from b down to -b;
* the phase exp(-i lambda x0) is carried by the incident density I(lambda) instead of by every
  representation (absolute x everywhere);
* Lemma 3.1 is used with phi = arg(x_l - x_m), i.e. alpha^l_nu = sum_n beta^m_n H_{n-nu}(k rho)
  exp(i (n - nu) phi) (the lemma as printed, with theta_lm = arg(x_m - x_l), has a wrong angle);
* the Mie denominator uses J_n(k_p R) (Eq. "linear" solved; the printed closed form has J_n(k R));
* Theorem 5.2 is used in the form H_n(k r) e^{i n theta} = (1/4 pi) int 4 (-i)^{n+1} w^n
  exp(-gamma |y - y_j|) exp(i lambda (x - x_j)) / gamma d lambda with w = (lambda - gamma)/k above
  the centre and w = (lambda + gamma)/k below it (the printed base and prefactor are garbled);
* the disc equations are solved in the preconditioned form (I - S(T + R)) beta = S a_inc, where
  S multiplies the incoming (local) coefficients (Sec. 3.2; Eq. "schur" with D = S T - I and C
  including S).
* more than three layers: each interior layer carries a wave leaving its top and one leaving its
  bottom interface, and [u] = [du/dy] = 0 at every interface gives 2(L - 1) equations per node;
* inclusions: Kress's product rule stands in for the Alpert rule Sec. 4 names; the coefficients of
  Sec. 4.1 carry the i/4 of the free-space Green's function and the full normal derivative of the
  incoming wave; a copy turned by theta has S_theta[l][n] = exp(-i l theta) S[l][n] exp(i n theta);
* guided-mode media: Gamma1's panels are placed by length over distance to the nearest
  singularity; absorbing layers (complex k, not in the sources' or the particles' layer) keep the
  principal branch of gamma;
* the fast translation Sec. 3.2 leaves to a wideband FMM is one level of boxes along x: Graf shifts
  to and from box centres and Graf translation between well-separated boxes, direct pairs
  between neighbours.

Notation: P = 2p + 1 orders n = -p..p stored at index n + p; beta has shape (N, P) (or
(nrhs, N, P)); the contour has N_S nodes lambda_nu with weights w_nu (d lambda included).
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special

FOUR_PI = 4.0 * math.pi


# ----------------------------------------------------------------------------------------------
# Special functions and the vertical wavenumber (Sec. 2, Sec. 3.1)
# ----------------------------------------------------------------------------------------------
def hankel(n, x):
    """H_n^(1)(x) (Sec. 3.1: the Hankel function of the first kind)."""
    return special.hankel1(n, x)


def hankel_p(n, x):
    """d/dx H_n^(1)(x)."""
    return special.h1vp(n, x)


def bessel(n, x):
    """J_n(x)."""
    return special.jv(n, x)


def bessel_p(n, x):
    """d/dx J_n(x)."""
    return special.jvp(n, x)


def gamma(lam, k):
    """sqrt(lambda^2 - k^2) on the branch with Re >= 0 (Sec. 2 Remark; Sec. 5.1 branch cuts).

    Written as -i sqrt(k^2 - lambda^2) with the principal square root: on the real axis it is
    positive for |lambda| > k and equals -i sqrt(k^2 - lambda^2) (an outgoing wave) for |lambda| < k.
    """
    lam = np.asarray(lam, dtype=complex)
    return -1j * np.sqrt(k * k - lam * lam)


# ----------------------------------------------------------------------------------------------
# Sommerfeld contour (Sec. 5.1, Eq. "sommerseg")
# ----------------------------------------------------------------------------------------------
def guided_band(branch_points):
    """(lo, hi): the real lambda where the layer response can have poles (guided modes), i.e.
    evanescent in both half-spaces (lambda > max(k_top, k_bottom)) yet propagating in an interior
    layer (lambda < the largest interior k); None when that interval is empty.  branch_points are
    the layers' wavenumbers from top to bottom."""
    ks = [float(k) for k in branch_points]
    if len(ks) < 3:
        return None
    lo, hi = max(ks[0], ks[-1]), max(ks[1:-1])
    return (lo, hi) if hi > lo else None


def contour_panel_breaks(n_panels: int, branch_points, b: float, t_max: float, band=None) -> np.ndarray:
    """Panel breakpoints of Gamma1 on t in [0, t_max].

    Without a guided-mode band: breakpoints sit at 0, t_max and every branch point k_i < t_max,
    and are graded geometrically toward each branch point (k_i +- b 2^j, j < L) with the largest L
    that keeps the panel count at most n_panels.  Remaining panels are made by halving the longest
    panel (first one on ties).  If even the ungraded set has too many panels, the branch points
    are dropped.

    With a guided-mode band (lo, hi) (poles of the layer response on the real axis, a distance b
    from Gamma1): start from 0, t_max and the branch points (0 and t_max alone if there are fewer
    panels than that), then repeatedly halve the panel with the largest length / (b + distance to
    the nearest branch point) (distance 0 for a panel that meets the band; first one on ties) until
    there are n_panels: the length of a Gauss-Legendre panel relative to the distance of its
    nearest singularity sets its error.
    """
    ks = sorted(set(float(k) for k in branch_points if 0.0 < k < t_max))
    if band is not None:
        lo, hi = float(band[0]), float(band[1])
        pts = sorted(set([0.0, float(t_max)] + ks))
        if len(pts) - 1 > n_panels:
            pts = [0.0, float(t_max)]

        def score(a, e):
            if e > lo and a < hi:
                dist = 0.0
            else:
                dist = t_max
                for s in ks:
                    dist = min(dist, 0.0 if a <= s <= e else min(abs(a - s), abs(e - s)))
            return (e - a) / (b + dist)

        while len(pts) - 1 < n_panels:
            best, bs = 0, -1.0
            for i in range(len(pts) - 1):
                sc = score(pts[i], pts[i + 1])
                if sc > bs:
                    best, bs = i, sc
            pts.insert(best + 1, 0.5 * (pts[best] + pts[best + 1]))
        return np.array(pts)
    levels = 0
    while b * 2.0 ** levels < t_max:
        levels += 1
    pts = None
    for lev in range(levels, -1, -1):
        cand = {0.0, float(t_max)}
        for k in ks:
            cand.add(k)
            for j in range(lev):
                for q in (k - b * 2.0 ** j, k + b * 2.0 ** j):
                    if 0.0 < q < t_max:
                        cand.add(q)
        if len(cand) - 1 <= n_panels:
            pts = sorted(cand)
            break
    if pts is None:
        pts = [0.0, float(t_max)]
    while len(pts) - 1 < n_panels:
        lengths = [pts[i + 1] - pts[i] for i in range(len(pts) - 1)]
        i = int(np.argmax(lengths))
        pts.insert(i + 1, 0.5 * (pts[i] + pts[i + 1]))
    return np.array(pts)


def contour(n_nodes: int, k1: float, k2: float, k3: float, b: float, t_max: float,
            panel_order: int = 16, branch_points=None, guided=True, graded=False, greedy=False):
    """Nodes lambda_nu and weights w_nu (d lambda included) of the discretised contour.

    Gamma1 (t - i b, 0 < t < t_max) and Gamma3 (its mirror t + i b, -t_max < t < 0) each carry
    n1 = q * floor((N_S - q) / (2 q)) Gauss-Legendre nodes in panels of order q placed by
    contour_panel_breaks (guided=False or graded=True: the geometric grading even in a
    guided-mode medium, for comparison only; greedy=True: the length over distance rule in every
    medium, with an empty band where there is no guided-mode band); Gamma2 (i s,
    s from b down to -b) carries the remaining N_S - 2 n1 nodes as one Gauss-Legendre rule.
    Returned in path order Gamma3 -> Gamma2 -> Gamma1.
    """
    q = panel_order
    n1 = q * ((n_nodes - q) // (2 * q))
    n2 = n_nodes - 2 * n1
    if n1 <= 0 or n2 <= 0:
        raise ValueError("contour: too few nodes for the panel order")
    bp = (k1, k2, k3) if branch_points is None else branch_points
    band = guided_band(bp) if guided and not graded else None
    if greedy and band is None:
        band = (0.0, 0.0)                                 # no panel meets an empty band
    breaks = contour_panel_breaks(n1 // q, bp, b, t_max, band)
    x, w = np.polynomial.legendre.leggauss(q)
    t1, w1 = [], []
    for a, c in zip(breaks[:-1], breaks[1:]):
        t1.append(0.5 * (a + c) + 0.5 * (c - a) * x)
        w1.append(0.5 * (c - a) * w)
    t1 = np.concatenate(t1)
    w1 = np.concatenate(w1)
    lam1 = t1 - 1j * b
    # Gamma3: lambda -> -lambda, traversed with t increasing from -t_max to 0
    lam3 = -lam1[::-1]
    w3 = w1[::-1]
    xs, ws = np.polynomial.legendre.leggauss(n2)
    s = (b * xs)[::-1]                       # from b down to -b
    lam2 = 1j * s
    w2 = -1j * (b * ws)[::-1]                # d lambda = i ds, ds negative along the path
    lam = np.concatenate([lam3, lam2, lam1])
    wt = np.concatenate([w3.astype(complex), w2, w1.astype(complex)])
    return lam, wt


# ----------------------------------------------------------------------------------------------
# Single disc: scattering matrix (Sec. 3.1, Eq. "linear"; Definition 3.1)
# ----------------------------------------------------------------------------------------------
def mie_coefficients(p: int, k2: float, kp: float, radius: float) -> np.ndarray:
    """Diagonal scattering matrix S_n, n = -p..p, by solving the 2x2 mode system of Eq. "linear".

    For each mode n with alpha_n = 1:  [-H_n(k2 R)  J_n(kp R); -k2 H_n'(k2 R)  kp J_n'(kp R)]
    [beta_n; gamma_n] = [J_n(k2 R); k2 J_n'(k2 R)];  S_n = beta_n.
    """
    out = np.zeros(2 * p + 1, dtype=complex)
    for n in range(-p, p + 1):
        a = np.array([[-hankel(n, k2 * radius), bessel(n, kp * radius)],
                      [-k2 * hankel_p(n, k2 * radius), kp * bessel_p(n, kp * radius)]])
        rhs = np.array([bessel(n, k2 * radius), k2 * bessel_p(n, k2 * radius)])
        out[n + p] = np.linalg.solve(a, rhs)[0]
    return out


def pec_coefficients(p: int, k2: float, radius: float) -> np.ndarray:
    """Scattering diagonal of a perfectly conducting disc (Sec. 3.1, remark after Definition 3.1):
    the total field vanishes on the boundary, J_n(k2 R) alpha_n + H_n(k2 R) beta_n = 0."""
    n = np.arange(-p, p + 1)
    return -bessel(n, k2 * radius) / hankel(n, k2 * radius)


def order_scale(p: int, k2: float, radius: float) -> np.ndarray:
    """|H_n(k2 R)|, n = -p..p: the diagonal that makes every order O(1) on the disc boundary."""
    n = np.arange(-p, p + 1)
    return np.abs(hankel(n, k2 * radius))


# ----------------------------------------------------------------------------------------------
# Inclusions of any smooth shape (Sec. 4: Eqs. "rep1", "rep2", "intg1", "intg2"; Sec. 4.1)
# ----------------------------------------------------------------------------------------------
EULER_GAMMA = 0.57721566490153286061


def kress_log_weights(n_pts: int) -> np.ndarray:
    """Weights R_j of the product rule  int_0^2pi ln(4 sin^2((t_i - tau)/2)) f(tau) d tau
    ~ sum_j R_{(i - j) mod n_pts} f(t_j),  t_j = 2 pi j / n_pts  (exact for trigonometric
    polynomials of degree < n_pts / 2: Kress's quadrature for logarithmic singularities, used here
    in place of Alpert's hybrid Gauss-trapezoidal rule; reading of Sec. 4's remark).

    With n = n_pts / 2:  R_j = -(2 pi / n) sum_{m=1}^{n-1} cos(m t_j) / m - (pi / n^2) cos(n t_j).
    """
    if n_pts < 4 or n_pts % 2:
        raise ValueError("kress_log_weights: need an even number of points >= 4")
    n = n_pts // 2
    tj = 2.0 * np.pi * np.arange(n_pts) / n_pts
    m = np.arange(1, n)
    return (-(2.0 * np.pi / n) * (np.cos(np.outer(tj, m)) / m[None, :]).sum(axis=1)
            - (np.pi / n ** 2) * np.cos(n * tj))


def _kernels(curve, k: float):
    """Parametrised kernels of the four boundary operators for wavenumber k, split as
    M(t, tau) = M1(t, tau) ln(4 sin^2((t - tau)/2)) + M2(t, tau), off the diagonal.

    G = (i/4) H_0(k r);  S: G;  D (at the boundary, principal value): dG/dn_y;  N: dG/dn_x;
    T: d^2 G / dn_x dn_y.  ds_y = |x'(tau)| d tau is folded in.  M1 is the coefficient of ln r
    halved (ln r = ln(4 sin^2)/2 + smooth), taken from the J_0, J_1 parts of H_0 = J_0 (1 +
    (2i/pi) ln(k r / 2)) + ..., H_1 = J_1 (1 + (2i/pi) ln(k r / 2)) - 2i/(pi k r) + ....
    Returns dicts of (n_pts, n_pts) arrays with the diagonal left at zero.
    """
    x, dx, ddx = curve
    n_pts = x.shape[0]
    d = x[:, None, :] - x[None, :, :]                  # x(t_i) - x(t_j)
    r = np.hypot(d[..., 0], d[..., 1])
    off = ~np.eye(n_pts, dtype=bool)
    r_safe = np.where(off, r, 1.0)
    sp = np.hypot(dx[:, 0], dx[:, 1])                  # |x'|
    nu = np.stack([dx[:, 1], -dx[:, 0]], axis=1)       # |x'| n (outward for counterclockwise)
    nx = nu / sp[:, None]
    nx_d = np.einsum("ik,ijk->ij", nx, d)              # n(t_i) . (x_i - x_j)
    nuy_d = np.einsum("jk,ijk->ij", nu, d)             # |x'_j| n(t_j) . (x_i - x_j)
    nx_nuy = nx @ nu.T                                 # n(t_i) . |x'_j| n(t_j)
    z = k * r_safe
    h0, h1 = special.hankel1(0, z), special.hankel1(1, z)
    j0, j1 = special.jv(0, z), special.jv(1, z)
    sp_j = sp[None, :]
    out = {}
    out["S"] = (0.25j * h0 * sp_j, -(1.0 / FOUR_PI) * j0 * sp_j)
    out["D"] = (0.25j * k * h1 * nuy_d / r_safe, -(k / FOUR_PI) * j1 * nuy_d / r_safe)
    out["N"] = (-0.25j * k * h1 * nx_d / r_safe * sp_j, (k / FOUR_PI) * j1 * nx_d / r_safe * sp_j)
    a_full = k * k * h0 / r_safe ** 2 - 2.0 * k * h1 / r_safe ** 3
    a_reg = k * k * j0 / r_safe ** 2 - 2.0 * k * j1 / r_safe ** 3
    out["T"] = (0.25j * (a_full * nx_d * nuy_d + k * h1 / r_safe * nx_nuy),
                -(1.0 / FOUR_PI) * (a_reg * nx_d * nuy_d + k * j1 / r_safe * nx_nuy))
    res = {}
    for key, (m, m1) in out.items():
        m = np.where(off, m, 0.0)
        m1 = np.where(off, m1, 0.0)
        res[key] = (m, m1)
    return res, sp


def muller_matrix(curve, k2: float, kp: float) -> np.ndarray:
    """Nystrom matrix of Eqs. "intg1", "intg2" in the unknowns [mu; sigma] (2 n_pts):

        mu + (S^{k2} - S^{kp}) sigma + (D^{k2} - D^{kp}) mu            = -u_inc
        -sigma + (N^{k2} - N^{kp}) sigma + (T^{k2} - T^{kp}) mu         = -du_inc/dn

    Each difference kernel is at most logarithmically singular; it is integrated with the weights
    R_j against its log part M1 and with the trapezoidal rule (2 pi / n_pts) against M2 = M - M1 L.
    Diagonal limits of the differences (C = Euler's constant, s = |x'(t)|):
      S: M1 = -(s / 4 pi)(J_0 terms cancel to 0 in the difference), M2 = -(s / 2 pi) ln(k2 / kp);
      D, N: M1 = M2 = 0;
      T: M1 = -(k2^2 - kp^2) s / (8 pi),
         M2 = s [ (i/8 + (1 - 2C)/(8 pi)) (k2^2 - kp^2) - (k2^2 ln(k2 s / 2) - kp^2 ln(kp s / 2)) / (4 pi) ].
    """
    x = curve[0]
    n_pts = x.shape[0]
    kw = kress_log_weights(n_pts)
    idx = (np.arange(n_pts)[:, None] - np.arange(n_pts)[None, :]) % n_pts
    Rw = kw[idx]
    tt = 2.0 * np.pi * np.arange(n_pts) / n_pts
    L = np.log(np.where(np.eye(n_pts, dtype=bool), 1.0, 4.0 * np.sin((tt[:, None] - tt[None, :]) / 2) ** 2))
    ka, sp = _kernels(curve, k2)
    kb, _ = _kernels(curve, kp)
    h = 2.0 * np.pi / n_pts
    diag = np.arange(n_pts)
    mats = {}
    dk2 = k2 * k2 - kp * kp
    for key in ("S", "D", "N", "T"):
        m = ka[key][0] - kb[key][0]
        m1 = ka[key][1] - kb[key][1]
        m2 = m - m1 * L
        if key == "S":
            m1[diag, diag] = 0.0
            m2[diag, diag] = -(sp / (2.0 * np.pi)) * np.log(k2 / kp)
        elif key == "T":
            m1[diag, diag] = -dk2 * sp / (8.0 * np.pi)
            m2[diag, diag] = sp * ((0.125j + (1.0 - 2.0 * EULER_GAMMA) / (8.0 * np.pi)) * dk2
                                   - (k2 * k2 * np.log(k2 * sp / 2.0) - kp * kp * np.log(kp * sp / 2.0))
                                   / FOUR_PI)
        else:
            m1[diag, diag] = 0.0
            m2[diag, diag] = 0.0
        mats[key] = Rw * m1 + h * m2
    eye = np.eye(n_pts)
    return np.block([[eye + mats["D"], mats["S"]], [mats["T"], -eye + mats["N"]]])


def regular_wave_traces(curve, k: float, n: int):
    """J_n(k rho) e^{i n theta} and its normal derivative at the curve points (polar coordinates
    about the enclosing disc's centre, the origin)."""
    x, dx, _ = curve
    rho = np.hypot(x[:, 0], x[:, 1])
    th = np.arctan2(x[:, 1], x[:, 0])
    sp = np.hypot(dx[:, 0], dx[:, 1])
    nrm = np.stack([dx[:, 1], -dx[:, 0]], axis=1) / sp[:, None]
    n_rho = (nrm[:, 0] * np.cos(th) + nrm[:, 1] * np.sin(th))
    n_th = (-nrm[:, 0] * np.sin(th) + nrm[:, 1] * np.cos(th))
    e = np.exp(1j * n * th)
    u = bessel(n, k * rho) * e
    du = (k * bessel_p(n, k * rho) * n_rho + 1j * n / rho * bessel(n, k * rho) * n_th) * e
    return u, du


def outgoing_from_densities(curve, k2: float, sigma, mu, p: int) -> np.ndarray:
    """beta_l, l = -p..p, of u^s = S^{k2} sigma + D^{k2} mu outside the enclosing disc (Sec. 4.1):
    beta_l = (i/4) int [J_l(k2 |y|) e^{-i l theta_y} sigma + n_y . grad(J_l(k2 |y|) e^{-i l theta_y}) mu] ds_y
    (Graf's addition theorem for G = (i/4) H_0), by the trapezoidal rule."""
    x, dx, _ = curve
    n_pts = x.shape[0]
    h = 2.0 * np.pi / n_pts
    sp = np.hypot(dx[:, 0], dx[:, 1])
    out = np.zeros(2 * p + 1, dtype=complex)
    for l in range(-p, p + 1):
        u, du = regular_wave_traces(curve, k2, -l)        # J_{-l} e^{-i l theta} = (-1)^l J_l e^{-i l theta}
        sgn = (-1.0) ** l
        out[l + p] = 0.25j * h * np.sum(sgn * (u * sigma + du * mu) * sp)
    return out


def inclusion_scattering_matrix(curve, p: int, k2: float, kp: float) -> np.ndarray:
    """S[l + p, n + p] = beta^n_l: outgoing coefficients of the inclusion for the incoming wave
    J_n(k2 r) e^{i n theta} (Sec. 4.1), by one LU of the Muller matrix and 2p + 1 solves."""
    a = muller_matrix(curve, k2, kp)
    n_pts = curve[0].shape[0]
    S = np.zeros((2 * p + 1, 2 * p + 1), dtype=complex)
    lu = __import__("scipy.linalg", fromlist=["lu_factor"])
    fac = lu.lu_factor(a)
    for n in range(-p, p + 1):
        u, du = regular_wave_traces(curve, k2, n)
        sol = lu.lu_solve(fac, np.concatenate([-u, -du]))
        mu, sigma = sol[:n_pts], sol[n_pts:]
        S[:, n + p] = outgoing_from_densities(curve, k2, sigma, mu, p)
    return S


def rotate_scattering_matrix(S: np.ndarray, theta: float) -> np.ndarray:
    """Scattering matrix of the prototype turned by theta about its centre (Sec. 4.1):
    S_theta[l, n] = e^{-i l theta} S[l, n] e^{i n theta}."""
    p = (S.shape[0] - 1) // 2
    e = np.exp(1j * np.arange(-p, p + 1) * theta)
    return np.conj(e)[:, None] * S * e[None, :]


# ----------------------------------------------------------------------------------------------
# Free-space multiple scattering (Sec. 3.2, Lemma 3.1, Eq. "trans", Eq. "scattmatrix")
# ----------------------------------------------------------------------------------------------
def translation_matrix(xl, xm, k: float, p_out: int, p_in: int) -> np.ndarray:
    """T^{lm}: local coefficients on disc l induced by the H-expansion of disc m (Lemma 3.1).

    T[nu + p_out, n + p_in] = H_{n - nu}(k rho) exp(i (n - nu) phi), rho = |x_l - x_m|,
    phi = arg(x_l - x_m).
    """
    dx, dy = xl[0] - xm[0], xl[1] - xm[1]
    rho = math.hypot(dx, dy)
    phi = math.atan2(dy, dx)
    nu = np.arange(-p_out, p_out + 1)[:, None]
    n = np.arange(-p_in, p_in + 1)[None, :]
    s = n - nu
    return hankel(s, k * rho) * np.exp(1j * s * phi)


def translate(centres: np.ndarray, beta: np.ndarray, k2: float, p: int, rows=None) -> np.ndarray:
    """alpha^l = sum_{m != l} T^{lm} beta^m for the target discs in `rows` (all by default).

    beta: (N, P).  Per target, the Hankel values of all sources are evaluated at once; the sum
    over sources and orders is the plain double sum of Eq. "trans".
    """
    n_disc = centres.shape[0]
    rows = range(n_disc) if rows is None else rows
    nu = np.arange(-p, p + 1)
    s_all = np.arange(-2 * p, 2 * p + 1)
    out = np.zeros((len(rows), 2 * p + 1), dtype=complex)
    for r, l in enumerate(rows):
        m = np.array([j for j in range(n_disc) if j != l], dtype=int)
        if m.size == 0:
            continue
        d = centres[l][None, :] - centres[m]
        rho = np.hypot(d[:, 0], d[:, 1])
        phi = np.arctan2(d[:, 1], d[:, 0])
        h = hankel(s_all[None, :], k2 * rho[:, None]) * np.exp(1j * s_all[None, :] * phi[:, None])
        # h[j, s + 2p] = H_s(k rho_j) e^{i s phi_j};  alpha_nu = sum_j sum_n h[j, n - nu] beta_j,n
        for a, v in enumerate(nu):
            idx = (nu - v) + 2 * p          # n - nu for n = -p..p
            out[r, a] = np.sum(h[:, idx] * beta[m])
    return out


# ----------------------------------------------------------------------------------------------
# Layered medium: the 4x4 mode system (Sec. 2, Eq. "sommerfeldsys")
# ----------------------------------------------------------------------------------------------
def box_translate(centres: np.ndarray, beta: np.ndarray, k2: float, p: int, box_width: float,
                  order: int, y_centre: float) -> np.ndarray:
    """The translation of Lemma 3.1 with the far field compressed by boxes (the FMM remark of
    Sec. 3.2 and the multipole shifts of Sec. 5.3), plainly: discs are grouped into boxes of width
    box_width along x with centres C_i at height y_centre; pairs in the same or adjacent boxes are
    translated directly; for boxes at least two apart the discs' H-expansions are shifted to their
    box centre (Graf: B_q = sum_m sum_n J_{q-n}(k |x_m - C|) e^{-i (q - n) phi_m} beta^m_n),
    translated box to box by Lemma 3.1 truncated at |q|, |nu| <= order, and shifted to each target
    (Graf: alpha_nu = sum_q J_{q - nu}(k |x_l - C|) e^{i (q - nu) phi_l} A_q)."""
    c = np.asarray(centres, dtype=float).reshape(-1, 2)
    n_d = c.shape[0]
    P = 2 * p + 1
    x0 = c[:, 0].min()
    box = np.floor((c[:, 0] - x0) / box_width).astype(int)
    nb = int(box.max()) + 1 if n_d else 0
    C = np.stack([x0 + (np.arange(nb) + 0.5) * box_width, np.full(nb, float(y_centre))], axis=1)
    nn = np.arange(-p, p + 1)
    qq = np.arange(-order, order + 1)
    B = np.zeros((nb, 2 * order + 1), dtype=complex)
    for m in range(n_d):
        d = c[m] - C[box[m]]
        r, ph = math.hypot(d[0], d[1]), math.atan2(d[1], d[0])
        s = qq[:, None] - nn[None, :]
        B[box[m]] += (bessel(s, k2 * r) * np.exp(-1j * s * ph)) @ beta[m]
    A = np.zeros_like(B)
    for i in range(nb):
        for j in range(nb):
            if abs(i - j) >= 2:
                A[i] += translation_matrix(C[i], C[j], k2, order, order) @ B[j]
    alpha = np.zeros((n_d, P), dtype=complex)
    for l in range(n_d):
        d = c[l] - C[box[l]]
        r, ph = math.hypot(d[0], d[1]), math.atan2(d[1], d[0])
        s = qq[None, :] - nn[:, None]
        alpha[l] = (bessel(s, k2 * r) * np.exp(1j * s * ph)) @ A[box[l]]
        for m in np.nonzero(np.abs(box - box[l]) <= 1)[0]:
            if m != l:
                alpha[l] += translation_matrix(c[l], c[m], k2, p, p) @ beta[m]
    return alpha


class Medium:
    """Three layers: k1 (y > 0), k2 (-d < y < 0), k3 (y < -d); discs kp, radius R."""

    def __init__(self, k1, k2, k3, d, kp, radius):
        self.k1, self.k2, self.k3, self.d, self.kp, self.radius = k1, k2, k3, d, kp, radius

    def a_lambda(self, lam, g=None) -> np.ndarray:
        """A_lambda of Eq. "sommerfeldsys" for every node: shape (N_S, 4, 4).

        Unknowns (sigma_1, sigma_2^+, sigma_2^-, sigma_3); rows: [u] = 0 at y = 0, [u] = 0 at
        y = -d, [du/dy] = 0 at y = 0, [du/dy] = 0 at y = -d (Eqs. "cont1", "cont2").  g: the
        vertical wavenumbers (gamma_1, gamma_2, gamma_3) to use instead of `gamma` (another branch).
        """
        lam = np.atleast_1d(lam)
        g1, g2, g3 = g if g is not None else (gamma(lam, self.k1), gamma(lam, self.k2), gamma(lam, self.k3))
        e = np.exp(-g2 * self.d)
        a = np.zeros((lam.size, 4, 4), dtype=complex)
        a[:, 0, 0] = 1.0 / g1
        a[:, 0, 1] = -1.0 / g2
        a[:, 0, 2] = -e / g2
        a[:, 1, 1] = e / g2
        a[:, 1, 2] = 1.0 / g2
        a[:, 1, 3] = -1.0 / g3
        a[:, 2, 0] = 1.0
        a[:, 2, 1] = 1.0
        a[:, 2, 2] = -e
        a[:, 3, 1] = e
        a[:, 3, 2] = -1.0
        a[:, 3, 3] = -1.0
        return a

    def incident_density(self, lam, src, g1=None) -> np.ndarray:
        """I(lambda) = exp(-gamma_1 y0 - i lambda x0): the line source's plane-wave amplitude at
        y = 0 (Eq. "sommer" with y < y0; the exp(-i lambda x0) phase is kept in the density)."""
        g1 = gamma(lam, self.k1) if g1 is None else g1
        return np.exp(-g1 * src[1] - 1j * lam * src[0])

    def rhs(self, lam, inc=None, p_plus=None, q_minus=None, g=None) -> np.ndarray:
        """Right-hand side of A_lambda sigma for the incident density I and the particle sums.

        Incident: (-I/gamma_1, 0, I, 0) (Eq. "sommerfeldsys").  Particles: their field near the
        top interface is (1/4pi) int P^+ e^{-gamma_2 y}/gamma_2 e^{i lambda x}, near the bottom
        interface (1/4pi) int Q^- e^{gamma_2 (y + d)}/gamma_2 e^{i lambda x}; moving these known
        terms of [u] and [du/dy] to the right gives (P^+/gamma_2, -Q^-/gamma_2, P^+, -Q^-).
        """
        lam = np.atleast_1d(lam)
        g1, g2 = (g[0], g[1]) if g is not None else (gamma(lam, self.k1), gamma(lam, self.k2))
        r = np.zeros((lam.size, 4), dtype=complex)
        if inc is not None:
            r[:, 0] += -inc / g1
            r[:, 2] += inc
        if p_plus is not None:
            r[:, 0] += p_plus / g2
            r[:, 2] += p_plus
        if q_minus is not None:
            r[:, 1] += -q_minus / g2
            r[:, 3] += -q_minus
        return r

    def solve_layers(self, lam, inc=None, p_plus=None, q_minus=None, g=None) -> np.ndarray:
        """sigma = A_lambda^{-1} rhs at every node (LAPACK LU); shape (N_S, 4)."""
        a = self.a_lambda(lam, g)
        r = self.rhs(lam, inc, p_plus, q_minus, g)
        return np.linalg.solve(a, r[..., None])[..., 0]

    def guided_poles(self, n_scan: int = 40001) -> list:
        """Real poles lambda_g of the layer response in (max(k1, k3), k2): the guided modes of a
        lossless layer (zeros of det A_lambda)."""
        band = guided_band((self.k1, self.k2, self.k3))
        if band is None:
            return []
        return real_zeros(lambda x: np.linalg.det(self.a_lambda(np.array([complex(x)]))[0]), *band, n_scan)


def real_zeros(det, lo: float, hi: float, n_scan: int = 40001) -> list:
    """Zeros of det(lambda) on the open interval (lo, hi) of the real axis.  On the real axis a
    layer system's determinant is c(lambda) f(lambda) with a slowly turning phase c, so sign changes
    of its real or imaginary part are bracketed on a fine grid and refined by Brent's method,
    keeping those where |det| vanishes against the grid's median (a sign change through a pole of
    det, where an interior layer's gamma passes through 0, is dropped by that test)."""
    from scipy import optimize

    xs = np.linspace(lo + 1e-9, hi - 1e-9, n_scan)
    vals = np.array([det(x) for x in xs])
    ok = np.isfinite(vals)
    ref = np.median(np.abs(vals[ok]))
    zeros = []
    for i in range(n_scan - 1):
        if not (ok[i] and ok[i + 1]):
            continue
        for part in (np.real, np.imag):
            if np.sign(part(vals[i])) != np.sign(part(vals[i + 1])):
                r = optimize.brentq(lambda x: part(det(x)), xs[i], xs[i + 1], xtol=1e-15, rtol=1e-15)
                if abs(det(r)) < 1e-8 * ref:
                    zeros.append(r)
    out = []
    for r in sorted(zeros):
        if not out or r - out[-1] > 1e-9:
            out.append(r)
    return out


class Stack:
    """Any number of layers (the generalisation the paper's introduction names): wavenumbers
    k_1 (top, y > 0) .. k_L (bottom), interior layers 2..L-1 of thicknesses d_2..d_{L-1}, discs in
    layer m (2 <= m <= L-1).  The interfaces are at z_1 = 0, z_i = z_{i-1} - d_i.

    Each interior layer j carries (1/4pi) int [s_j^+ exp(gamma_j (y - z_{j-1})) +
    s_j^- exp(-gamma_j (y - z_j))] / gamma_j exp(i lambda x) d lambda (a wave leaving its top and one
    leaving its bottom interface), layer 1 sigma_1 exp(-gamma_1 y) / gamma_1 and layer L
    sigma_L exp(gamma_L (y - z_{L-1})) / gamma_L, as in the three-layer representation (Sec. 2).
    [u] = [du/dy] = 0 at every interface gives 2(L - 1) equations per node, solved by LAPACK LU.
    The discs' spectral densities enter at the two interfaces of layer m in the particle layer's own
    frame (its top interface at y = 0): the Problem class is used unchanged with disc centres given
    in that frame (y + depth), and solve_layers returns (sigma_1, s_m^+, s_m^-, sigma_L).
    """

    def __init__(self, ks, ds, m, kp, radius):
        # complex k (Im k > 0) makes a layer absorbing; gamma's principal branch keeps Re >= 0
        self.ks = [complex(k) if np.iscomplexobj(k) and complex(k).imag != 0.0 else float(np.real(k)) for k in ks]
        self.ds, self.mi = [float(d) for d in ds], int(m)
        self.L = len(self.ks)
        if self.L < 3 or len(self.ds) != self.L - 2 or not 2 <= self.mi <= self.L - 1:
            raise ValueError("Stack: need L >= 3 layers, L - 2 thicknesses and 2 <= m <= L - 1")
        self.k1, self.k2, self.k3 = self.ks[0], self.ks[self.mi - 1], self.ks[-1]
        self.d = self.ds[self.mi - 2]
        self.depth = sum(self.ds[: self.mi - 2])        # from y = 0 down to the top of layer m
        self.kp, self.radius = kp, radius

    def incident_density(self, lam, src, g1=None) -> np.ndarray:
        g1 = gamma(lam, self.k1) if g1 is None else g1
        return np.exp(-g1 * src[1] - 1j * lam * src[0])

    def interfaces(self):
        """z_1 = 0, z_i = z_{i-1} - d_i: the interface heights (L - 1 values)."""
        z = [0.0]
        for dd in self.ds:
            z.append(z[-1] - dd)
        return z

    def _col(self, j, sign):
        """Unknown index of layer j (1-based): sigma_1, (s_2^+, s_2^-), ..., sigma_L."""
        n = 2 * self.L - 2
        if j == 1:
            return 0
        if j == self.L:
            return n - 1
        return 1 + 2 * (j - 2) + (0 if sign > 0 else 1)

    def _assemble(self, gv, inc=None, p_plus=None, q_minus=None):
        """The interface system of one node: [u] = [du/dy] = 0 at every interface, for the vertical
        wavenumbers gv[j - 1] of layer j and the known densities (scalars or None)."""
        L, m, col = self.L, self.mi, self._col
        n = 2 * L - 2
        E = {j: np.exp(-gv[j - 1] * self.ds[j - 2]) for j in range(2, L)}
        a = np.zeros((n, n), dtype=complex)
        r = np.zeros(n, dtype=complex)
        for i in range(1, L):                                    # interface i: layer i above, i + 1 below
            rv, rd = 2 * (i - 1), 2 * (i - 1) + 1
            gi, gb = gv[i - 1], gv[i]
            if i == 1:                                           # layer above: value, derivative
                a[rv, col(1, 1)] += 1.0 / gi
                a[rd, col(1, 1)] += -1.0
            else:
                a[rv, col(i, 1)] += E[i] / gi
                a[rv, col(i, -1)] += 1.0 / gi
                a[rd, col(i, 1)] += E[i]
                a[rd, col(i, -1)] += -1.0
            if i + 1 == L:                                       # layer below (subtracted)
                a[rv, col(L, 1)] -= 1.0 / gb
                a[rd, col(L, 1)] -= 1.0
            else:
                a[rv, col(i + 1, 1)] -= 1.0 / gb
                a[rv, col(i + 1, -1)] -= E[i + 1] / gb
                a[rd, col(i + 1, 1)] -= 1.0
                a[rd, col(i + 1, -1)] -= -E[i + 1]
            # known fields: rhs = (below) - (above)
            if i == 1 and inc is not None:                       # incident wave in layer 1
                r[rv] -= inc / gi
                r[rd] -= inc
            if i == m - 1 and p_plus is not None:                # discs, below this interface
                r[rv] += p_plus / gb
                r[rd] += -p_plus
            if i == m and q_minus is not None:                   # discs, above this interface
                r[rv] -= q_minus / gi
                r[rd] -= q_minus
        return a, r

    def solve_layers(self, lam, inc=None, p_plus=None, q_minus=None, g=None, full=False) -> np.ndarray:
        """(sigma_1, s_m^+, s_m^-, sigma_L) per node, or with full=True every unknown (sigma_1,
        s_2^+, s_2^-, ..., sigma_L).  g: the vertical wavenumbers of every layer to use instead of
        `gamma` (another branch)."""
        lam = np.atleast_1d(np.asarray(lam, dtype=complex))
        L, m = self.L, self.mi
        n = 2 * L - 2
        g = [gamma(lam, k) for k in self.ks] if g is None else list(g)    # g[j - 1] for layer j
        out = np.zeros((lam.size, n if full else 4), dtype=complex)
        pick = lambda arr, v: None if arr is None else arr[v]
        for v in range(lam.size):
            a, r = self._assemble([gj[v] for gj in g], pick(inc, v), pick(p_plus, v), pick(q_minus, v))
            s = np.linalg.solve(a, r)
            out[v] = s if full else (s[0], s[self._col(m, 1)], s[self._col(m, -1)], s[n - 1])
        return out

    def det(self, lam_real: float) -> complex:
        """det of the interface system at one real node (for locating its poles)."""
        lam = np.array([complex(lam_real)])
        a, _ = self._assemble([gamma(lam, k)[0] for k in self.ks])
        return np.linalg.det(a)

    def guided_poles(self, n_scan: int = 40001) -> list:
        """Real poles of the layer response in the guided band (max(k_1, k_L), max interior k),
        lossless stacks only: zeros of det of the interface system."""
        if any(isinstance(k, complex) for k in self.ks):
            raise ValueError("guided_poles: lossless layers only")
        band = guided_band(self.ks)
        return [] if band is None else real_zeros(self.det, *band, n_scan)


# ----------------------------------------------------------------------------------------------
# Multipole <-> Sommerfeld (Sec. 5.2.1 Lemma 5.1 / Eq. "JA2"; Sec. 5.3 Theorem 5.2)
# ----------------------------------------------------------------------------------------------
def m2s_factor(n, lam, k: float, above: bool):
    """c_n w^n with c_n = 4 (-i)^{n+1}: the spectral coefficient of H_n(k r) e^{i n theta}.

    Theorem 5.2 (read as stated in the module docstring): w = (lambda - gamma)/k for targets above
    the expansion centre, (lambda + gamma)/k below it.
    """
    g = gamma(lam, k)
    w = (lam - g) / k if above else (lam + g) / k
    n = np.asarray(n)
    return 4.0 * (-1j) ** (n + 1) * w ** n


def plane_wave_local_factor(m, lam, k: float, downward: bool):
    """i^m w^m: Jacobi-Anger coefficient of J_m(k r) e^{i m theta} in a layer plane wave.

    exp(gamma (y - y_i) + i lambda (x - x_i)) (decaying downward, from the top interface) uses
    w = (lambda - gamma)/k; exp(-gamma (y - y_i) + i lambda (x - x_i)) uses (lambda + gamma)/k
    (Lemma 5.1 with the direction angle of the complex wave vector (lambda, -+ i gamma)).
    """
    g = gamma(lam, k)
    w = (lam - g) / k if downward else (lam + g) / k
    m = np.asarray(m)
    return (1j) ** m * w ** m


# ----------------------------------------------------------------------------------------------
# The discretised problem
# ----------------------------------------------------------------------------------------------
class Problem:
    """Discs at `centres` in layer 2, order p, contour (lam, wt).

    All linear maps below are the discrete ones: every Sommerfeld integral is the quadrature sum
    (1/4pi) sum_nu w_nu (...) over the same nodes.
    """

    def __init__(self, medium: Medium, p: int, centres: np.ndarray, lam, wt, smat=None, theta=None):
        self.m = medium
        self.p = p
        self.P = 2 * p + 1
        self.c = np.asarray(centres, dtype=float).reshape(-1, 2)
        self.N = self.c.shape[0]
        self.lam = np.asarray(lam, dtype=complex)
        self.wt = np.asarray(wt, dtype=complex)
        self.S = mie_coefficients(p, medium.k2, medium.kp, medium.radius)
        self.orders = np.arange(-p, p + 1)
        # inclusions of another shape (Sec. 4.1): one scattering matrix per particle, the
        # prototype's turned by that particle's angle
        self.smats = None
        if smat is not None:
            th = np.zeros(self.N) if theta is None else np.asarray(theta, dtype=float)
            self.smats = np.stack([rotate_scattering_matrix(np.asarray(smat), a) for a in th]) \
                if self.N else np.zeros((0, self.P, self.P), dtype=complex)

    def scatter(self, alpha, rows=None):
        """S_j alpha^j for every particle j (or the listed rows)."""
        alpha = np.asarray(alpha)
        if self.smats is None:
            return self.S[None, :] * alpha
        sm = self.smats if rows is None else self.smats[list(rows)]
        return np.einsum("jln,jn->jl", sm, alpha)

    # --- (a2) free-space translation --------------------------------------------------------
    def translation(self, beta, rows=None):
        return translate(self.c, beta, self.m.k2, self.p, rows)

    # --- (a3) aggregate: multipole -> Sommerfeld (Theorem 5.2, Eq. "invfft") ------------------
    def aggregate(self, beta):
        """P^+(nu) and Q^-(nu): spectral densities of all H-expansions at the two interfaces.

        For each node and order n: c_n w_-^n sum_j beta^j_n exp(gamma_2 y_j - i lambda x_j)
        (top, w_- = (lambda - gamma_2)/k2) and c_n w_+^n sum_j beta^j_n exp(-gamma_2 (y_j + d)
        - i lambda x_j) (bottom); then summed over n.
        """
        k2, d = self.m.k2, self.m.d
        lam = self.lam[:, None]
        g2 = gamma(lam, k2)
        x, y = self.c[None, :, 0], self.c[None, :, 1]
        e_top = np.exp(g2 * y - 1j * lam * x)             # (N_S, N)
        e_bot = np.exp(-g2 * (y + d) - 1j * lam * x)
        f_top = m2s_factor(self.orders[None, :], lam, k2, above=True)   # (N_S, P)
        f_bot = m2s_factor(self.orders[None, :], lam, k2, above=False)
        p_plus = np.sum(f_top * (e_top @ beta), axis=1)
        q_minus = np.sum(f_bot * (e_bot @ beta), axis=1)
        return p_plus, q_minus

    # --- (a4) per-node layer response (Eq. "sommerfeldsys" with particle terms) -----------------
    def layer_densities(self, inc=None, p_plus=None, q_minus=None):
        return self.m.solve_layers(self.lam, inc, p_plus, q_minus)

    # --- (a5) disaggregate: Sommerfeld -> local (Lemma 5.1, Eq. "JA2") -------------------------
    def disaggregate(self, s2p, s2m, rows=None):
        """alpha^i_m = (1/4pi) sum_nu (w_nu / gamma_2) [sigma_2^+ exp(gamma_2 y_i + i lambda x_i)
        i^m w_-^m + sigma_2^- exp(-gamma_2 (y_i + d) + i lambda x_i) i^m w_+^m]."""
        k2, d = self.m.k2, self.m.d
        c = self.c if rows is None else self.c[list(rows)]
        lam = self.lam[None, :]
        g2 = gamma(lam, k2)
        x, y = c[:, 0:1], c[:, 1:2]
        e_top = np.exp(g2 * y + 1j * lam * x)             # (Nr, N_S)
        e_bot = np.exp(-g2 * (y + d) + 1j * lam * x)
        lamc = self.lam[:, None]
        f_top = plane_wave_local_factor(self.orders[None, :], lamc, k2, downward=True)  # (N_S, P)
        f_bot = plane_wave_local_factor(self.orders[None, :], lamc, k2, downward=False)
        q = (self.wt / (FOUR_PI * gamma(self.lam, k2)))[:, None]
        return e_top @ (q * s2p[:, None] * f_top) + e_bot @ (q * s2m[:, None] * f_bot)

    # --- R beta: reflected coupling (a3 -> a4 -> a5) --------------------------------------------
    def reflection(self, beta, rows=None):
        p_plus, q_minus = self.aggregate(beta)
        sig = self.layer_densities(None, p_plus, q_minus)
        return self.disaggregate(sig[:, 1], sig[:, 2], rows)

    # --- (a6) the preconditioned operator ---------------------------------------------------------
    def apply(self, x, rows=None, parts=("T", "R")):
        """y = x - S (T + R) x (Sec. 3.2 preconditioned form; Eq. "schur" up to sign)."""
        x = np.asarray(x, dtype=complex).reshape(self.N, self.P)
        alpha = np.zeros((self.N if rows is None else len(rows), self.P), dtype=complex)
        if "T" in parts:
            alpha += self.translation(x, rows)
        if "R" in parts:
            alpha += self.reflection(x, rows)
        xr = x if rows is None else x[list(rows)]
        return xr - self.scatter(alpha, rows)

    # --- (a8) incident local expansions ---------------------------------------------------------
    def incident_local(self, src, rows=None):
        """a_inc: the particle-free layered field in layer 2 expanded on each disc."""
        inc = self.m.incident_density(self.lam, src)
        sig = self.layer_densities(inc=inc)
        return self.disaggregate(sig[:, 1], sig[:, 2], rows)

    def rhs(self, src):
        return self.scatter(self.incident_local(src))

    def absorbed_power(self, src, beta) -> np.ndarray:
        """Time-averaged power absorbed inside each particle (zero for lossless ones).

        Near particle j the total field is sum_n (alpha_n J_n(k2 r) + beta_n H_n(k2 r)) e^{i n theta}
        with alpha = a_inc + (T + R) beta, its incoming coefficients.  Its flux
        Im int conj(u) du/dr ds through a circle around the particle (inside the annulus that holds
        no other sources) follows from the Wronskian J_n Y_n' - J_n' Y_n = 2 / (pi x):
        4 sum_n (|beta_n|^2 + Re(conj(alpha_n) beta_n)), the same normalisation in which the line
        source (i/4) H_0 emits 1/4.  The absorbed power is minus that flux; for a lossless particle
        (I + 2S unitary) it vanishes."""
        beta = np.asarray(beta, dtype=complex).reshape(self.N, self.P)
        alpha = self.incident_local(src) + self.translation(beta) + self.reflection(beta)
        return -4.0 * (np.abs(beta) ** 2 + (np.conj(alpha) * beta).real).sum(axis=1)

    # --- dense assembly and solves (Eq. "finalsys", Eq. "schur") ----------------------------------
    def dense_operator(self):
        """The (N P) x (N P) matrix of x -> x - S (T + R) x, column by column."""
        n = self.N * self.P
        out = np.zeros((n, n), dtype=complex)
        e = np.zeros(n, dtype=complex)
        for j in range(n):
            e[:] = 0.0
            e[j] = 1.0
            out[:, j] = self.apply(e).ravel()
        return out

    def operator_rows(self, rows):
        """Rows of the same matrix for the target particles `rows`, shape (len(rows) P, N P),
        written from the formulas instead of column by column (which costs N P applications):

        * T: for every source m != l the block T^{lm}[nu][n] = H_{n-nu}(k2 rho) e^{i (n-nu) phi}
          of Lemma 3.1 (rho, phi of x_l - x_m), from one table of H_s e^{i s phi} per target as in
          `translate`;
        * R: aggregate (Theorem 5.2) -> per-node layer response (Eq. "sommerfeldsys") ->
          disaggregate (Lemma 5.1), each written as a matrix.  The layer response is linear in
          (P+, Q-) node by node; its coefficients are the densities for a unit P+ and for a unit
          Q-;
        * then the rows of x - S (T + R) x.

        Equal to the rows of `dense_operator()` (pinned on small cases)."""
        rows = list(rows)
        N, P, p = self.N, self.P, self.p
        k2, d = self.m.k2, self.m.d
        nr = len(rows)
        tr = np.zeros((nr, P, N, P), dtype=complex)          # [r, nu, m, n] of (T + R)
        s_all = np.arange(-2 * p, 2 * p + 1)
        idx = self.orders[None, :] - self.orders[:, None] + 2 * p   # [nu, n] -> n - nu + 2p
        for r, l in enumerate(rows):
            m = np.array([j for j in range(N) if j != l], dtype=int)
            if m.size == 0:
                continue
            dxy = self.c[l][None, :] - self.c[m]
            rho = np.hypot(dxy[:, 0], dxy[:, 1])
            phi = np.arctan2(dxy[:, 1], dxy[:, 0])
            h = hankel(s_all[None, :], k2 * rho[:, None]) * np.exp(1j * s_all[None, :] * phi[:, None])
            tr[r][:, m, :] = np.transpose(h[:, idx], (1, 0, 2))
        tr = tr.reshape(nr * P, N * P)
        if N:
            lam = self.lam
            g2 = gamma(lam, k2)
            x, y = self.c[:, 0], self.c[:, 1]
            e_top = np.exp(g2[:, None] * y[None, :] - 1j * lam[:, None] * x[None, :])        # (N_S, N)
            e_bot = np.exp(-g2[:, None] * (y[None, :] + d) - 1j * lam[:, None] * x[None, :])
            f_top = m2s_factor(self.orders[None, :], lam[:, None], k2, above=True)           # (N_S, P)
            f_bot = m2s_factor(self.orders[None, :], lam[:, None], k2, above=False)
            agg_top = (e_top[:, :, None] * f_top[:, None, :]).reshape(lam.size, N * P)       # dP+/dbeta
            agg_bot = (e_bot[:, :, None] * f_bot[:, None, :]).reshape(lam.size, N * P)       # dQ-/dbeta
            one, zero = np.ones(lam.size, dtype=complex), np.zeros(lam.size, dtype=complex)
            sig_p = self.layer_densities(None, one, zero)
            sig_q = self.layer_densities(None, zero, one)
            s2p = sig_p[:, 1][:, None] * agg_top + sig_q[:, 1][:, None] * agg_bot           # dsigma2+/dbeta
            s2m = sig_p[:, 2][:, None] * agg_top + sig_q[:, 2][:, None] * agg_bot           # dsigma2-/dbeta
            cr = self.c[rows]
            q = self.wt / (FOUR_PI * g2)
            l_top = plane_wave_local_factor(self.orders[None, :], lam[:, None], k2, downward=True)
            l_bot = plane_wave_local_factor(self.orders[None, :], lam[:, None], k2, downward=False)
            dt = np.exp(g2[None, :] * cr[:, 1:2] + 1j * lam[None, :] * cr[:, 0:1])         # (nr, N_S)
            db = np.exp(-g2[None, :] * (cr[:, 1:2] + d) + 1j * lam[None, :] * cr[:, 0:1])
            dis_top = (dt[:, None, :] * (q[:, None] * l_top).T[None, :, :]).reshape(nr * P, lam.size)
            dis_bot = (db[:, None, :] * (q[:, None] * l_bot).T[None, :, :]).reshape(nr * P, lam.size)
            tr += dis_top @ s2p + dis_bot @ s2m
        tr = tr.reshape(nr, P, N * P)
        if self.smats is None:
            out = -self.S[None, :, None] * tr
        else:
            out = -np.einsum("rln,rnk->rlk", self.smats[rows], tr)
        for r, l in enumerate(rows):
            out[r, np.arange(P), l * P + np.arange(P)] += 1.0
        return out.reshape(nr * P, N * P)

    def solve_dense(self, src):
        """beta from (I - S(T + R)) beta = S a_inc by LU, on the system equilibrated by the order
        scale D = diag(|H_n(k2 R)|) (D A D^{-1} (D beta) = D rhs: the same solution; when k2 R is
        small the plain matrix's condition number grows with |H_p(k2 R)| while the equilibrated one
        stays near 1, and LU is only backward stable in the norm of the system it factors)."""
        a = self.dense_operator()
        d = np.tile(order_scale(self.p, self.m.k2, self.m.radius), self.N)
        x = np.linalg.solve(d[:, None] * a / d[None, :], d * self.rhs(src).ravel()) / d
        return x.reshape(self.N, self.P)

    def block_system(self, src):
        """[A B; C D] [sigma; beta] = [b; 0] of Eq. "finalsys", assembled entry by entry.

        sigma is ordered node-major (sigma_1, sigma_2^+, sigma_2^-, sigma_3) per node; beta is
        disc-major.  D = S T - I, C = S times the Sommerfeld-to-local map, B = minus the
        multipole-to-Sommerfeld right-hand-side map.
        """
        ns, P, N = self.lam.size, self.P, self.N
        k2, d = self.m.k2, self.m.d
        lam = self.lam
        g2 = gamma(lam, k2)
        A = np.zeros((4 * ns, 4 * ns), dtype=complex)
        al = self.m.a_lambda(lam)
        for v in range(ns):
            A[4 * v:4 * v + 4, 4 * v:4 * v + 4] = al[v]
        B = np.zeros((4 * ns, N * P), dtype=complex)
        C = np.zeros((N * P, 4 * ns), dtype=complex)
        f_top = m2s_factor(self.orders[None, :], lam[:, None], k2, above=True)
        f_bot = m2s_factor(self.orders[None, :], lam[:, None], k2, above=False)
        l_top = plane_wave_local_factor(self.orders[None, :], lam[:, None], k2, downward=True)
        l_bot = plane_wave_local_factor(self.orders[None, :], lam[:, None], k2, downward=False)
        q = self.wt / (FOUR_PI * g2)
        for j in range(N):
            xj, yj = self.c[j]
            et = np.exp(g2 * yj - 1j * lam * xj)
            eb = np.exp(-g2 * (yj + d) - 1j * lam * xj)
            pp = f_top * et[:, None]       # d P^+ / d beta^j_n
            qm = f_bot * eb[:, None]       # d Q^- / d beta^j_n
            cols = slice(j * P, (j + 1) * P)
            B[0::4, cols] = -(pp / g2[:, None])
            B[1::4, cols] = -(-qm / g2[:, None])
            B[2::4, cols] = -pp
            B[3::4, cols] = -(-qm)
            ct = np.exp(g2 * yj + 1j * lam * xj)
            cb = np.exp(-g2 * (yj + d) + 1j * lam * xj)
            rows = slice(j * P, (j + 1) * P)
            sj = np.diag(self.S) if self.smats is None else self.smats[j]
            C[rows, 1::4] = sj @ ((q * ct)[None, :] * l_top.T)
            C[rows, 2::4] = sj @ ((q * cb)[None, :] * l_bot.T)
        T = np.zeros((N * P, N * P), dtype=complex)
        for l in range(N):
            for m in range(N):
                if l != m:
                    T[l * P:(l + 1) * P, m * P:(m + 1) * P] = translation_matrix(
                        self.c[l], self.c[m], k2, self.p, self.p)
        if self.smats is None:
            D = np.tile(self.S, N)[:, None] * T - np.eye(N * P)
        else:
            sblk = np.zeros((N * P, N * P), dtype=complex)
            for j in range(N):
                sblk[j * P:(j + 1) * P, j * P:(j + 1) * P] = self.smats[j]
            D = sblk @ T - np.eye(N * P)
        inc = self.m.incident_density(lam, src)
        b = self.m.rhs(lam, inc=inc).ravel()
        return A, B, C, D, b

    def solve_block(self, src):
        """Solve Eq. "finalsys" by dense LU; returns (sigma (N_S, 4), beta (N, P))."""
        A, B, C, D, b = self.block_system(src)
        ns = self.lam.size
        big = np.block([[A, B], [C, D]])
        rhs = np.concatenate([b, np.zeros(self.N * self.P, dtype=complex)])
        sol = np.linalg.solve(big, rhs)
        return sol[:4 * ns].reshape(ns, 4), sol[4 * ns:].reshape(self.N, self.P)

    def solve_schur(self, src):
        """Solve Eq. "schur": [D - C A^{-1} B] beta = -C A^{-1} b by LU."""
        A, B, C, D, b = self.block_system(src)
        ainv_b = np.linalg.solve(A, B)
        ainv_rhs = np.linalg.solve(A, b)
        return np.linalg.solve(D - C @ ainv_b, -C @ ainv_rhs).reshape(self.N, self.P)

    # --- (a9) fields ----------------------------------------------------------------------------
    def densities(self, src, beta):
        """All four layer densities with the incident source and the discs' H-expansions."""
        inc = self.m.incident_density(self.lam, src)
        if self.N and beta is not None:
            p_plus, q_minus = self.aggregate(np.asarray(beta).reshape(self.N, self.P))
        else:
            p_plus = q_minus = np.zeros(self.lam.size, dtype=complex)
        return self.layer_densities(inc, p_plus, q_minus)

    def field_layer1(self, src, beta, pts, which="total"):
        """u_1 at points with y > 0 (Eq. "fullrep"): 'total', 'scattered' (u_1 - G) or 'particle'
        (u_1 minus the particle-free u_1)."""
        pts = np.atleast_2d(pts)
        k1 = self.m.k1
        g1 = gamma(self.lam, k1)
        sig = self.densities(src, beta)[:, 0]
        if which == "particle":
            sig = sig - self.densities(src, None)[:, 0]
        ex = np.exp(-g1[None, :] * pts[:, 1:2] + 1j * self.lam[None, :] * pts[:, 0:1])
        u = ex @ (self.wt * sig / g1) / FOUR_PI
        if which == "total":
            r = np.hypot(pts[:, 0] - src[0], pts[:, 1] - src[1])
            u = u + 0.25j * hankel(0, k1 * r)
        return u

    def field_layer2(self, src, beta, pts):
        """u_2 at points in -d < y < 0 outside the discs: Sommerfeld terms plus every H-expansion."""
        pts = np.atleast_2d(pts)
        k2, d = self.m.k2, self.m.d
        g2 = gamma(self.lam, k2)
        sig = self.densities(src, beta)
        e_t = np.exp(g2[None, :] * pts[:, 1:2] + 1j * self.lam[None, :] * pts[:, 0:1])
        e_b = np.exp(-g2[None, :] * (pts[:, 1:2] + d) + 1j * self.lam[None, :] * pts[:, 0:1])
        u = (e_t @ (self.wt * sig[:, 1] / g2) + e_b @ (self.wt * sig[:, 2] / g2)) / FOUR_PI
        if beta is not None:
            beta = np.asarray(beta).reshape(self.N, self.P)
            for j in range(self.N):
                dd = pts - self.c[j][None, :]
                r = np.hypot(dd[:, 0], dd[:, 1])
                th = np.arctan2(dd[:, 1], dd[:, 0])
                u = u + (hankel(self.orders[None, :], k2 * r[:, None])
                         * np.exp(1j * self.orders[None, :] * th[:, None])) @ beta[j]
        return u

    def field_layer3(self, src, beta, pts):
        pts = np.atleast_2d(pts)
        k3, d = self.m.k3, self.m.d
        g3 = gamma(self.lam, k3)
        sig = self.densities(src, beta)[:, 3]
        ex = np.exp(g3[None, :] * (pts[:, 1:2] + d) + 1j * self.lam[None, :] * pts[:, 0:1])
        return ex @ (self.wt * sig / g3) / FOUR_PI

    # --- radiated power (lossless media; a check of the whole solution, not a step of it) -------
    def outgoing_power(self, src, beta, tol=1e-13):
        """Time-averaged power leaving through y = +inf (layer 1) and y = -inf (layer 3).

        Above the source, u_1 = (1/4pi) int U exp(-gamma_1 y + i lambda x) / gamma_1 with
        U = sigma_1 + exp(gamma_1 y0 - i lambda x0) (the direct wave written in the same form, as in
        Eq. "sommer"); below y = -d, u_3 = (1/4pi) int sigma_3 exp(gamma_3 (y + d) + i lambda x) /
        gamma_3.  Parseval turns the flux Im int conj(u) du/dn dx into (1/8pi) int |U|^2 / s_1 over
        |lambda| < k_1 (s_i = sqrt(k_i^2 - lambda^2); evanescent waves carry no power), and likewise
        (1/8pi) int |sigma_3|^2 / s_3 over |lambda| < k_3.  With lambda = k cos(theta) the weight
        1/s becomes d theta; each interval is split where lambda crosses the other layers'
        wavenumbers (square-root branch points of the densities), each piece is mapped by
        theta = a + (b - a)(1 - cos phi)/2, which makes the endpoint square roots smooth in phi, and
        integrated by adaptive Gauss-Kronrod (QUADPACK): between k_1 and k_2 the layer acts as a
        leaky waveguide and the densities peak near its modes.  The densities are evaluated exactly
        on the real axis from beta.
        """
        from scipy import integrate

        k1, k2, k3 = self.m.k1, self.m.k2, self.m.k3

        def density(lam_real, layer):
            lam = np.array([lam_real], dtype=complex)
            pr = Problem(self.m, self.p, self.c, lam, np.zeros_like(lam))
            sig = pr.densities(src, beta)[0]
            if layer == 1:
                return sig[0] + np.exp(gamma(lam, k1)[0] * src[1] - 1j * lam[0] * src[0])
            return sig[3]

        def piece(k, layer, a, b):
            def f(phi):
                th = a + (b - a) * 0.5 * (1.0 - math.cos(phi))
                return abs(density(k * math.cos(th), layer)) ** 2 * (b - a) * 0.5 * math.sin(phi)
            return integrate.quad(f, 0.0, math.pi, epsabs=tol, epsrel=tol, limit=4000)[0]

        branch = [complex(kk).real for kk in getattr(self.m, "ks", (k1, k2, k3))]   # every layer's Re k

        def pieces(k, layer):
            inner = sorted(set(math.acos(kk / k) for kk in branch if kk < k))
            breaks = [0.0] + inner + [math.pi - t for t in reversed(inner)] + [math.pi]
            return sum(piece(k, layer, a, b) for a, b in zip(breaks[:-1], breaks[1:])) / (2.0 * FOUR_PI)

        if complex(k3).imag == 0.0:
            return pieces(k1, 1), pieces(complex(k3).real, 3)
        # an absorbing bottom half-space: the power crossing into it, all of which it absorbs,
        # -(1/8pi) int |sigma_L|^2 Im(gamma_L) / |gamma_L|^2 over the whole real axis (the same
        # Parseval identity; for real k_L only |lambda| < k_L contributes and this is the form above)
        kl = complex(k3)

        def f(lam_real):
            g = gamma(np.array([lam_real], dtype=complex), kl)[0]
            return -abs(density(lam_real, 3)) ** 2 * g.imag / abs(g) ** 2

        tail = max(abs(kk) for kk in branch) + 60.0
        pts = sorted(set([-tail, tail] + [s * abs(kk) for kk in branch for s in (-1.0, 1.0)]))
        down = sum(integrate.quad(f, a, b, epsabs=tol, epsrel=tol, limit=4000)[0]
                   for a, b in zip(pts[:-1], pts[1:])) / (2.0 * FOUR_PI)
        return pieces(k1, 1), down


def guided_power(pr: "Problem", src, beta, n_circle: int = 128):
    """Time-averaged power the guided modes carry to x = +inf and x = -inf (lossless media).

    For x -> +inf the Sommerfeld integrals close upward around the poles +lambda_g (the contour
    passes below them), so the field tends to (i/2) sum_g R_g(y) e^{i lambda_g x}, R_g the residue
    of the integrand: sigma_1 e^{-gamma_1 y}/gamma_1 above, (s_j^+ e^{gamma_j (y - z_{j-1})} +
    s_j^- e^{-gamma_j (y - z_j)})/gamma_j in interior layer j (for three layers
    (sigma_2^+ e^{gamma_2 y} + sigma_2^- e^{-gamma_2 (y + d)})/gamma_2), sigma_L
    e^{gamma_L (y - z_{L-1})}/gamma_L below (the discs' own H-expansions have no poles); likewise
    -lambda_g for x -> -inf.  The flux Im int conj(u) du/dx dy of a mode is
    (lambda_g / 4) int |R_g|^2 dy.  Residues come from the trapezoidal rule on a circle around the
    pole, with gamma_j continued from the contour (sqrt(lambda^2 - k_j^2) for k_j < lambda_g, where
    the principal -i sqrt(k^2 - lambda^2) has its cut); the mode integrals are exact exponentials in
    the half-spaces, Gauss-Legendre in each interior layer.  Works for a Medium or a Stack.
    Returns (power to +inf, power to -inf)."""
    m = pr.m
    poles = m.guided_poles()
    stack = isinstance(m, Stack)
    ks = list(m.ks) if stack else [m.k1, m.k2, m.k3]
    ds = list(m.ds) if stack else [m.d]
    zs = m.interfaces() if stack else [0.0, -m.d]

    def gcont(lam, k, lg):
        lam = np.asarray(lam, dtype=complex)
        return np.sqrt(lam * lam - k * k) if k < abs(lg) else gamma(lam, k)

    def dens(lam, lg):
        g = [gcont(lam, k, lg) for k in ks]
        inc = m.incident_density(lam, src, g[0])
        if pr.N and beta is not None:
            sub = Problem(m, pr.p, pr.c, lam, np.zeros_like(lam))
            p_plus, q_minus = sub.aggregate(np.asarray(beta).reshape(pr.N, pr.P))
        else:
            p_plus = q_minus = None
        if stack:
            return m.solve_layers(lam, inc, p_plus, q_minus, g, full=True)
        return m.solve_layers(lam, inc, p_plus, q_minus, g)      # (sigma_1, sigma_2^+-, sigma_3)

    xg, wg = np.polynomial.legendre.leggauss(64)
    total = [0.0, 0.0]
    for side, sgn in ((0, 1.0), (1, -1.0)):
        for pg in poles:
            lg = sgn * pg
            others = list(ks) + [q for q in poles if q != pg]
            rho = min(abs(pg - q) for q in others) / 3.0
            th = 2.0 * np.pi * np.arange(n_circle) / n_circle
            z = lg + rho * np.exp(1j * th)
            res = (rho / n_circle) * (dens(z, lg) * np.exp(1j * th)[:, None]).sum(axis=0)
            l = np.array([lg], dtype=complex)
            g = [gcont(l, k, lg)[0] for k in ks]
            c_top, c_bot = res[0] / g[0], res[-1] / g[-1]
            integral = abs(c_top) ** 2 / (2.0 * g[0].real) + abs(c_bot) ** 2 / (2.0 * g[-1].real)
            for j in range(2, len(ks)):                          # interior layer j: z_j < y < z_{j-1}
                d, top, bot = ds[j - 2], zs[j - 2], zs[j - 1]
                cp, cm = res[1 + 2 * (j - 2)] / g[j - 1], res[2 + 2 * (j - 2)] / g[j - 1]
                y = bot + d / 2 * (1.0 + xg)
                u = cp * np.exp(g[j - 1] * (y - top)) + cm * np.exp(-g[j - 1] * (y - bot))
                integral += np.sum(wg * d / 2 * np.abs(u) ** 2)
            total[side] += pg / 4.0 * integral
    return total[0], total[1]


# ----------------------------------------------------------------------------------------------
# Converged mode (discretisation studies only): the same contour, integrated adaptively
# ----------------------------------------------------------------------------------------------
def contour_pieces(branch_points, b: float, t_max: float) -> list:
    """Sec. 5.1's contour Gamma3 -> Gamma2 -> Gamma1, truncated at |Re lambda| = t_max, as straight
    pieces (lam0, direction, s0, s1): lambda(s) = lam0 + direction s, d lambda = direction ds,
    split at the branch points (real parts) so that every piece is smooth."""
    ks = sorted(set(float(np.real(k)) for k in branch_points if 0.0 < float(np.real(k)) < t_max))
    g1 = [0.0] + ks + [float(t_max)]
    back = g1[::-1]
    pieces = [(1j * b, 1.0, -a, -e) for a, e in zip(back[:-1], back[1:])]     # Gamma3, t up to 0
    pieces.append((1j * b, -1j, 0.0, 2.0 * b))                                 # Gamma2: i (b - s)
    pieces += [(-1j * b, 1.0, a, e) for a, e in zip(g1[:-1], g1[1:])]          # Gamma1
    return pieces


def converged_parts(pr: "Problem", src, targets, lam):
    """At nodes lam (any complex values): the integrands of the three contour sums of Problem, in
    the scaled unknowns b = |H_n(k2 R)| beta: K(lambda) (N P x N P) with D S R D^{-1} = int K,
    r(lambda) (N P) with D S a_inc = int r, and for the layer-1 scattered field at the targets
    u = int (f(lambda) + H(lambda) b).  Per node the reflection is rank two (Sec. 5: aggregate,
    layer response, disaggregate), so K = q [u_top (r_pp v_top + r_pq v_bot)^T + u_bot (r_qp v_top +
    r_qq v_bot)^T], with the factors of Problem.aggregate / disaggregate and the layer response for
    unit densities.  Returns (K, r, f, H) stacked over the nodes."""
    m, k2, d = pr.m, pr.m.k2, pr.m.d
    lam = np.atleast_1d(np.asarray(lam, dtype=complex))
    n_s, N, P = lam.size, pr.N, pr.P
    hs = order_scale(pr.p, k2, m.radius)
    x, y = pr.c[:, 0], pr.c[:, 1]
    g2 = gamma(lam, k2)[:, None]
    lc = lam[:, None]
    # aggregation factors (Theorem 5.2): P^+ = v_top . beta, Q^- = v_bot . beta
    v_top = (np.exp(g2 * y[None, :] - 1j * lc * x[None, :])[:, :, None]
             * m2s_factor(pr.orders[None, None, :], lc[:, :, None], k2, above=True)).reshape(n_s, N * P)
    v_bot = (np.exp(-g2 * (y[None, :] + d) - 1j * lc * x[None, :])[:, :, None]
             * m2s_factor(pr.orders[None, None, :], lc[:, :, None], k2, above=False)).reshape(n_s, N * P)
    # disaggregation factors (Lemma 5.1), with the scattering matrices applied (S alpha)
    u_top = (np.exp(g2 * y[None, :] + 1j * lc * x[None, :])[:, :, None]
             * plane_wave_local_factor(pr.orders[None, None, :], lc[:, :, None], k2, downward=True))
    u_bot = (np.exp(-g2 * (y[None, :] + d) + 1j * lc * x[None, :])[:, :, None]
             * plane_wave_local_factor(pr.orders[None, None, :], lc[:, :, None], k2, downward=False))
    u_top = np.stack([pr.scatter(u) for u in u_top]).reshape(n_s, N * P)
    u_bot = np.stack([pr.scatter(u) for u in u_bot]).reshape(n_s, N * P)
    q = 1.0 / (FOUR_PI * gamma(lam, k2))
    one, zero = np.ones(n_s, dtype=complex), np.zeros(n_s, dtype=complex)
    from_p = m.solve_layers(lam, None, one, zero)          # response to a unit P^+
    from_q = m.solve_layers(lam, None, zero, one)          # response to a unit Q^-
    inc = m.incident_density(lam, src)
    from_i = m.solve_layers(lam, inc)
    dsc = np.tile(hs, N)                                   # D on rows and columns
    left_t = (q[:, None] * u_top) * dsc[None, :]
    left_b = (q[:, None] * u_bot) * dsc[None, :]
    right_t = v_top / dsc[None, :]
    right_b = v_bot / dsc[None, :]
    K = (left_t[:, :, None] * (from_p[:, 1, None] * right_t + from_q[:, 1, None] * right_b)[:, None, :]
         + left_b[:, :, None] * (from_p[:, 2, None] * right_t + from_q[:, 2, None] * right_b)[:, None, :])
    r = left_t * from_i[:, 1, None] + left_b * from_i[:, 2, None]
    pts = np.atleast_2d(targets)
    g1 = gamma(lam, m.k1)
    ex = np.exp(-g1[:, None] * pts[None, :, 1] + 1j * lam[:, None] * pts[None, :, 0]) / (FOUR_PI * g1[:, None])
    f = ex * from_i[:, 0, None]
    H = ex[:, :, None] * (from_p[:, 0, None] * right_t + from_q[:, 0, None] * right_b)[:, None, :]
    return K, r, f, H


def converged_solution(pr: "Problem", src, targets, b: float, t_max: float, tol: float = 1e-13):
    """The solution of the same problem with every contour sum replaced by the exact integral over
    the same truncated contour (adaptive Gauss-Kronrod, scipy's quad_vec, to tol in the scaled
    entries), the translation unchanged: (beta, scattered field at the targets).  Only the contour
    quadrature differs from Problem's discrete solution, so the difference measures its error."""
    from scipy import integrate

    N, P = pr.N, pr.P
    n_t = np.atleast_2d(targets).shape[0]
    sizes = [(N * P) ** 2, N * P, n_t, n_t * N * P]

    def fun(lam):
        K, r, f, H = converged_parts(pr, src, targets, np.array([lam]))
        return np.concatenate([K.ravel(), r.ravel(), f.ravel(), H.ravel()])

    branch = getattr(pr.m, "ks", (pr.m.k1, pr.m.k2, pr.m.k3))
    total = 0.0
    for lam0, dr, s0, s1 in contour_pieces(branch, b, t_max):
        val, _ = integrate.quad_vec(lambda s: fun(lam0 + dr * s) * dr, s0, s1, epsabs=tol, epsrel=tol,
                                    norm="max", limit=20000)
        total = total + val
    o = np.cumsum([0] + sizes)
    K = total[o[0]:o[1]].reshape(N * P, N * P)
    r = total[o[1]:o[2]]
    f = total[o[2]:o[3]]
    H = total[o[3]:o[4]].reshape(n_t, N * P)
    hs = np.tile(order_scale(pr.p, pr.m.k2, pr.m.radius), N)
    T = np.zeros((N * P, N * P), dtype=complex)
    for l in range(N):
        for j in range(N):
            if j != l:
                T[l * P:(l + 1) * P, j * P:(j + 1) * P] = translation_matrix(pr.c[l], pr.c[j], pr.m.k2, pr.p, pr.p)
    ST = np.concatenate([pr.scatter(T[:, c].reshape(N, P)).reshape(-1, 1) for c in range(N * P)], axis=1)
    A = np.eye(N * P) - hs[:, None] * ST / hs[None, :] - K
    bsol = np.linalg.solve(A, r)
    return (bsol / hs).reshape(N, P), f + H @ bsol


def gmres(matvec, b, tol=1e-12, maxiter=500):
    """Unrestarted GMRES (Saad and Schultz, cited in Sec. 3.2) with modified Gram-Schmidt.

    Returns (x, iterations, relative residual history).
    """
    b = np.asarray(b, dtype=complex)
    n = b.size
    beta0 = np.linalg.norm(b)
    if beta0 == 0.0:
        return np.zeros(n, dtype=complex), 0, [0.0]
    V = np.zeros((maxiter + 1, n), dtype=complex)
    H = np.zeros((maxiter + 1, maxiter), dtype=complex)
    V[0] = b / beta0
    cs = np.zeros(maxiter, dtype=complex)
    sn = np.zeros(maxiter, dtype=complex)
    g = np.zeros(maxiter + 1, dtype=complex)
    g[0] = beta0
    hist = [1.0]
    k = 0
    for k in range(maxiter):
        w = matvec(V[k])
        for i in range(k + 1):
            H[i, k] = np.vdot(V[i], w)
            w = w - H[i, k] * V[i]
        H[k + 1, k] = np.linalg.norm(w)
        if H[k + 1, k] != 0:
            V[k + 1] = w / H[k + 1, k]
        for i in range(k):
            t = cs[i] * H[i, k] + sn[i] * H[i + 1, k]
            H[i + 1, k] = -np.conj(sn[i]) * H[i, k] + np.conj(cs[i]) * H[i + 1, k]
            H[i, k] = t
        a, c = H[k, k], H[k + 1, k]
        r = math.hypot(abs(a), abs(c))
        cs[k] = a / r if r else 1.0
        sn[k] = c / r if r else 0.0
        cs[k], sn[k] = np.conj(cs[k]), np.conj(sn[k])
        H[k, k] = cs[k] * a + sn[k] * c
        H[k + 1, k] = 0.0
        g[k + 1] = -np.conj(sn[k]) * g[k]
        g[k] = cs[k] * g[k]
        hist.append(abs(g[k + 1]) / beta0)
        if hist[-1] <= tol:
            k += 1
            break
    else:
        k = maxiter
    y = np.linalg.solve(np.triu(H[:k, :k]), g[:k])
    x = V[:k].T @ y
    return x, k, hist


# ----------------------------------------------------------------------------------------------
# The same sums on several host cores: target particles split into chunks across processes
# ----------------------------------------------------------------------------------------------
_POOL_PROBLEM = None


def _pool_init(problem):
    global _POOL_PROBLEM
    _POOL_PROBLEM = problem


def _pool_apply(task):
    x, rows = task
    return _POOL_PROBLEM.apply(x, rows=rows)


def _pool_operator_rows(rows):
    return _POOL_PROBLEM.operator_rows(rows)


class RowPool:
    """`Problem.apply` and `Problem.operator_rows` split over target particles in worker processes.

    Each worker holds a copy of the problem and evaluates the unchanged row sums for its chunk of
    target particles (the global aggregate and layer response are recomputed per chunk, as
    `Problem.apply(x, rows)` does); the results are concatenated in row order, so `apply` returns
    `problem.apply(x)` up to the rounding of the row-chunked matrix products.  Workers start with
    the spawn method and one BLAS thread each.  Use as a context manager, or call `close()`."""

    def __init__(self, problem, workers=None, chunks_per_worker=4):
        import multiprocessing as mp
        import os
        self.problem = problem
        self.workers = max(1, int(workers or os.cpu_count() or 1))
        self.chunks = max(1, self.workers * chunks_per_worker)
        saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for k in saved:
            os.environ[k] = "1"
        try:
            self.pool = mp.get_context("spawn").Pool(self.workers, initializer=_pool_init, initargs=(problem,))
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v

    def row_chunks(self, rows=None, chunks=None):
        rows = list(range(self.problem.N)) if rows is None else list(rows)
        n = max(1, min(chunks or self.chunks, len(rows)))
        return [c.tolist() for c in np.array_split(np.asarray(rows, dtype=int), n) if c.size]

    def apply(self, x, rows=None, chunks=None):
        """problem.apply(x, rows) (all rows by default), shape (len(rows), P)."""
        x = np.asarray(x, dtype=complex).reshape(self.problem.N, self.problem.P)
        parts = self.pool.map(_pool_apply, [(x, c) for c in self.row_chunks(rows, chunks)])
        return np.concatenate(parts, axis=0) if parts else np.zeros((0, self.problem.P), dtype=complex)

    def operator_rows(self, rows, chunks=None):
        """problem.operator_rows(rows) assembled chunk by chunk in the workers."""
        parts = self.pool.map(_pool_operator_rows, self.row_chunks(rows, chunks))
        return np.concatenate(parts, axis=0)

    def iter_operator_rows(self, rows=None, chunks=None):
        """Yield (chunk rows, problem.operator_rows(chunk rows)) in row order, one chunk in memory
        per worker at a time (for assembling a large matrix in place)."""
        ch = self.row_chunks(rows, chunks)
        for c, block in zip(ch, self.pool.imap(_pool_operator_rows, ch)):
            yield c, block

    def close(self):
        self.pool.close()
        self.pool.join()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
