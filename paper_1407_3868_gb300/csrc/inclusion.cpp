// Inclusions of any smooth shape (Sec. 4 of the paper): the scattering matrix of a prototype
// inclusion from Muller's second-kind boundary integral equations (Eqs. "intg1", "intg2"), and
// the per-particle rotated copies S_j = D(-theta_j) S D(theta_j), D(theta) = diag(e^{i n theta})
// (Sec. 4.1), that replace the disc's Mie diagonal in the operator x - S (T + R) x.
//
// Discretisation: Nystrom on the 2 pi-periodic parametrisation x(t), with Kress's product rule for
// the logarithmic singularities.  Every difference kernel of Eqs. "intg1", "intg2" is split as
// M(t, tau) = M1(t, tau) ln(4 sin^2((t - tau)/2)) + M2(t, tau) with M1, M2 smooth; M1 integrates
// against the weights R_j (exact for trigonometric polynomials of degree < n_pts/2), M2 with the
// trapezoidal rule.  M1 comes from the J_0, J_1 parts of H_0 = J_0 + (2i/pi) ln(z/2) J_0 + ... and
// H_1 = J_1 + (2i/pi) ln(z/2) J_1 - 2i/(pi z) + ...; the diagonal limits follow from the small-z
// expansions of H_0, H_1 (C = Euler's constant, s = |x'(t)|):
//   S^{k2} - S^{kp}: M1 = 0, M2 = -(s / 2 pi) ln(k2 / kp);   D, N differences: M1 = M2 = 0;
//   T^{k2} - T^{kp}: M1 = -(k2^2 - kp^2) s / 8 pi,
//     M2 = s [(i/8 + (1 - 2C)/8 pi)(k2^2 - kp^2) - (k2^2 ln(k2 s/2) - kp^2 ln(kp s/2)) / 4 pi].
// The outgoing coefficients follow from Graf's theorem for G = (i/4) H_0:
//   beta_l = (i/4) int [J_l(k2 |y|) e^{-i l theta_y} sigma + n_y . grad(J_l e^{-i l theta}) mu] ds_y.
#include <cmath>
#include <cstring>
#include <algorithm>
#include <string>
#include <thread>
#include <type_traits>
#include <vector>

#include "lsms_internal.h"
#include "lsms_ops.h"

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kEuler = 0.57721566490153286061;

// J_n(z) for any integer n (J_{-n} = (-1)^n J_n), z >= 0.
double bessel_jn(int n, double z) {
  const double v = std::cyl_bessel_j((double)std::abs(n), z);
  return (n < 0 && (std::abs(n) & 1)) ? -v : v;
}

// J_0, J_1, H_0, H_1 at a real argument (libstdc++ special math).
void bessel01(double z, double& j0, double& j1, cplx& h0, cplx& h1) {
  j0 = std::cyl_bessel_j(0.0, z);
  j1 = std::cyl_bessel_j(1.0, z);
  h0 = cplx(j0, std::cyl_neumann(0.0, z));
  h1 = cplx(j1, std::cyl_neumann(1.0, z));
}

// The same at a complex argument z (Re z >= 0, Im z >= 0, z != 0): the interior kernels of an
// absorbing inclusion.  J_n by Miller's backward recurrence J_{n-1} = (2n/z) J_n - J_{n+1} from
// J_{N+1} = 0 at N well above |z|, normalised with exp(-iz) = J_0 + 2 sum_{n>=1} (-i)^n J_n (the
// generating function exp((z/2)(t - 1/t)) = sum_n J_n t^n at t = -i; |exp(-iz)| = exp(Im z) >= 1,
// so the sum does not cancel).  Y_0 from Neumann's expansion
//   Y_0 = (2/pi)(ln(z/2) + C) J_0 - (4/pi) sum_{k>=1} (-1)^k J_{2k} / k,
// Y_1 = -Y_0' term by term (J_0' = -J_1, 2 J_n' = J_{n-1} - J_{n+1}):
//   Y_1 = -(2/pi) J_0 / z + (2/pi)(ln(z/2) + C) J_1 + (2/pi) sum_{k>=1} (-1)^k (J_{2k-1} - J_{2k+1}) / k.
// J is accurate to rounding relative to itself; H = J + iY, exponentially small when Im z is large,
// carries an absolute error of about 1e-16 |J| ~ 1e-16 exp(Im z), hence the cap on the loss.
void bessel01(cplx z, cplx& j0, cplx& j1, cplx& h0, cplx& h1) {
  const double az = std::abs(z);
  int top = (int)(az + 12.0 * std::cbrt(az)) + 40;
  top += top & 1;
  std::vector<cplx> J(top + 2);
  J[top + 1] = 0.0;
  J[top] = 1e-300;
  const cplx iz = 1.0 / z;
  for (int n = top; n >= 1; --n) {
    J[n - 1] = (2.0 * n) * iz * J[n] - J[n + 1];
    if (std::abs(J[n - 1]) > 1e250)
      for (int q = n - 1; q <= top + 1; ++q) J[q] *= 1e-250;
  }
  static const cplx mi[4] = {cplx(1, 0), cplx(0, -1), cplx(-1, 0), cplx(0, 1)};   // (-i)^n
  cplx s = J[0];
  for (int n = 1; n <= top; ++n) s += 2.0 * mi[n & 3] * J[n];
  const cplx scale = std::exp(cplx(0.0, -1.0) * z) / s;
  for (cplx& v : J) v *= scale;
  const cplx lg = std::log(0.5 * z) + kEuler;
  cplx s0 = 0.0, s1 = 0.0;
  for (int k = 1; 2 * k + 1 <= top; ++k) {
    const double sg = (k & 1) ? -1.0 : 1.0;
    s0 += sg * J[2 * k] / (double)k;
    s1 += sg * (J[2 * k - 1] - J[2 * k + 1]) / (double)k;
  }
  const cplx y0 = (2.0 / kPi) * (lg * J[0]) - (4.0 / kPi) * s0;
  const cplx y1 = -(2.0 / kPi) * J[0] * iz + (2.0 / kPi) * (lg * J[1]) + (2.0 / kPi) * s1;
  j0 = J[0];
  j1 = J[1];
  h0 = j0 + cplx(0.0, 1.0) * y0;
  h1 = j1 + cplx(0.0, 1.0) * y1;
}

// a x = b for the dense Muller system (n up to 8192 unknowns, nrhs = 2p + 1): right-looking blocked
// LU with partial pivoting on the augmented rows [a | b].  Each step factors a panel of NB columns
// over the full height, forward-substitutes its block row, and updates the trailing rows in
// parallel (row chunks over threads: the O(n^3) part); back substitution follows.  The solution
// overwrites b; a is released once copied (the augmented rows replace it).  False for a singular
// matrix.
bool solve_blocked(std::vector<cplx>& a, int n, std::vector<cplx>& b, int nrhs) {
  constexpr int NB = 64;
  const int nc = n + nrhs;
  std::vector<cplx> m((size_t)n * nc);
  for (int i = 0; i < n; ++i) {
    std::copy(a.begin() + (size_t)i * n, a.begin() + (size_t)(i + 1) * n, m.begin() + (size_t)i * nc);
    std::copy(b.begin() + (size_t)i * nrhs, b.begin() + (size_t)(i + 1) * nrhs, m.begin() + (size_t)i * nc + n);
  }
  std::vector<cplx>().swap(a);
  auto row = [&](int i) { return m.data() + (size_t)i * nc; };
  const unsigned hw = std::thread::hardware_concurrency();
  const int nthreads = (int)std::max(1u, std::min(hw ? hw : 4u, 16u));
  for (int k0 = 0; k0 < n; k0 += NB) {
    const int k1 = std::min(n, k0 + NB);
    for (int k = k0; k < k1; ++k) {                      // panel: columns k0 .. k1 - 1
      int piv = k;
      for (int i = k + 1; i < n; ++i)
        if (std::abs(row(i)[k]) > std::abs(row(piv)[k])) piv = i;
      if (std::abs(row(piv)[k]) == 0.0) return false;
      if (piv != k) std::swap_ranges(row(k), row(k) + nc, row(piv));
      const cplx inv = 1.0 / row(k)[k];
      for (int i = k + 1; i < n; ++i) {
        cplx* ri = row(i);
        const cplx f = ri[k] * inv;
        ri[k] = f;                                       // multiplier, kept as L
        if (f == cplx(0, 0)) continue;
        const cplx* rk = row(k);
        for (int j = k + 1; j < k1; ++j) ri[j] -= f * rk[j];
      }
    }
    for (int k = k0; k < k1; ++k)                        // block row of U (and of the rhs)
      for (int i = k + 1; i < k1; ++i) {
        const cplx f = row(i)[k];
        if (f == cplx(0, 0)) continue;
        cplx* ri = row(i);
        const cplx* rk = row(k);
        for (int j = k1; j < nc; ++j) ri[j] -= f * rk[j];
      }
    const int rows = n - k1;                             // trailing update, rows k1 .. n - 1
    if (rows <= 0) continue;
    auto update = [&](int r0, int r1) {
      for (int i = r0; i < r1; ++i) {
        cplx* ri = row(i);
        for (int k = k0; k < k1; ++k) {
          const cplx f = ri[k];
          if (f == cplx(0, 0)) continue;
          const cplx* rk = row(k);
          for (int j = k1; j < nc; ++j) ri[j] -= f * rk[j];
        }
      }
    };
    const int nt = std::min(nthreads, std::max(1, rows / 32));
    if (nt == 1) {
      update(k1, n);
    } else {
      std::vector<std::thread> pool;
      const int chunk = (rows + nt - 1) / nt;
      for (int t = 1; t < nt; ++t) {
        const int r0 = k1 + t * chunk, r1 = std::min(n, r0 + chunk);
        if (r0 < r1) pool.emplace_back(update, r0, r1);
      }
      update(k1, std::min(n, k1 + chunk));
      for (std::thread& th : pool) th.join();
    }
  }
  for (int k = n - 1; k >= 0; --k) {                     // back substitution on the rhs columns
    cplx* rk = row(k);
    for (int r = 0; r < nrhs; ++r) {
      cplx s = rk[n + r];
      for (int i = k + 1; i < n; ++i) s -= rk[i] * row(i)[n + r];
      rk[n + r] = s / rk[k];
    }
  }
  for (int i = 0; i < n; ++i) std::copy(row(i) + n, row(i) + nc, b.begin() + (size_t)i * nrhs);
  return true;
}

// the four kernels for one wavenumber (real, or complex for an absorbing interior) and one (i, j)
// pair: full and log part
template <typename K>
struct Kernels {
  cplx s, d, nn, t;
  K s1, d1, n1, t1;
};

// Kernels at x_i (normal nx, unit) and x_j (nu_j = |x'_j| n_j), ds_y = |x'_j| d tau folded in.
template <typename K>
Kernels<K> kernels(K k, const double dxy[2], double r, const double nx[2], const double nuj[2], double spj) {
  const K z = k * r;
  K j0, j1;
  cplx h0, h1;
  bessel01(z, j0, j1, h0, h1);
  const double nxd = nx[0] * dxy[0] + nx[1] * dxy[1];
  const double nuyd = nuj[0] * dxy[0] + nuj[1] * dxy[1];
  const double nxnuy = nx[0] * nuj[0] + nx[1] * nuj[1];
  const cplx iq(0.0, 0.25);
  const double c4 = 1.0 / (4.0 * kPi);
  Kernels<K> o;
  o.s = iq * h0 * spj;
  o.s1 = -c4 * j0 * spj;
  o.d = iq * k * h1 * nuyd / r;
  o.d1 = -c4 * k * j1 * nuyd / r;
  o.nn = -iq * k * h1 * nxd / r * spj;
  o.n1 = c4 * k * j1 * nxd / r * spj;
  const cplx a = k * k * h0 / (r * r) - 2.0 * k * h1 / (r * r * r);
  const K areg = k * k * j0 / (r * r) - 2.0 * k * j1 / (r * r * r);
  o.t = iq * (a * nxd * nuyd + k * h1 / r * nxnuy);
  o.t1 = -c4 * (areg * nxd * nuyd + k * j1 / r * nxnuy);
  return o;
}

}  // namespace

// S[l][n] (row-major, orders -p..p) of the inclusion bounded by `curve` ([n_pts][6]: x, y, x', y',
// x'', y'' at t_j = 2 pi j / n_pts, counterclockwise, about the enclosing disc's centre).
template <typename K>
int inclusion_matrix_t(int p, double k2, K kp, double radius, int n_pts, const double* curve,
                       std::vector<cplx>& S, std::string& err) {
  const int P = 2 * p + 1, n = n_pts;
  std::vector<double> x(n), y(n), sp(n), rho(n), th(n);
  std::vector<double> nux(n), nuy(n);                  // |x'| n (outward)
  double area = 0.0;
  for (int j = 0; j < n; ++j) {
    const double* c = curve + 6 * j;
    for (int q = 0; q < 6; ++q)
      if (!std::isfinite(c[q])) { err = "non-finite curve data"; return LSMS_ERR_ARG; }
    x[j] = c[0]; y[j] = c[1];
    sp[j] = std::hypot(c[2], c[3]);
    if (!(sp[j] > 0.0)) { err = "curve has a zero derivative"; return LSMS_ERR_ARG; }
    nux[j] = c[3]; nuy[j] = -c[2];
    rho[j] = std::hypot(x[j], y[j]);
    th[j] = std::atan2(y[j], x[j]);
    if (!(rho[j] > 1e-12 * radius)) { err = "curve passes through the enclosing disc's centre"; return LSMS_ERR_GEOMETRY; }
    if (!(rho[j] < radius)) { err = "inclusion is not inside the enclosing disc"; return LSMS_ERR_GEOMETRY; }
    area += 0.5 * (x[j] * c[3] - y[j] * c[2]);
  }
  if (!(area > 0.0)) { err = "curve must run counterclockwise"; return LSMS_ERR_ARG; }
  const double h = 2.0 * kPi / n;
  // Kress weights R_m, m = (i - j) mod n:  -(2 pi/h2) sum_{m'=1}^{h2-1} cos(m' t_m)/m' - (pi/h2^2) cos(h2 t_m)
  const int h2 = n / 2;
  std::vector<double> Rw(n);
  for (int m = 0; m < n; ++m) {
    const double tm = h * m;
    double s = 0.0;
    for (int q = 1; q < h2; ++q) s += std::cos(q * tm) / q;
    Rw[m] = -(2.0 * kPi / h2) * s - (kPi / ((double)h2 * h2)) * std::cos(h2 * tm);
  }
  // Muller matrix in the unknowns [mu; sigma]
  const int N2 = 2 * n;
  std::vector<cplx> A((size_t)N2 * N2, cplx(0, 0));
  const K dk2 = k2 * k2 - kp * kp;
  auto assemble_rows = [&](int i0, int i1) {             // rows i and n + i for i in [i0, i1)
    for (int i = i0; i < i1; ++i) {
      const double nx[2] = {nux[i] / sp[i], nuy[i] / sp[i]};
      for (int j = 0; j < n; ++j) {
        cplx ms, md, mn, mt;
        K m1s, m1d, m1n, m1t;
        double L = 0.0;
        if (i == j) {
          m1s = m1d = m1n = 0.0;
          m1t = -dk2 * sp[i] / (8.0 * kPi);
          if constexpr (std::is_same_v<K, double>)
            ms = cplx(-(sp[i] / (2.0 * kPi)) * std::log(k2 / kp), 0.0);
          else
            ms = -(sp[i] / (2.0 * kPi)) * std::log(k2 / kp);
          md = mn = cplx(0, 0);
          mt = sp[i] * (cplx((1.0 - 2.0 * kEuler) / (8.0 * kPi), 0.125) * dk2 -
                        (k2 * k2 * std::log(k2 * sp[i] / 2.0) - kp * kp * std::log(kp * sp[i] / 2.0)) /
                            (4.0 * kPi));
        } else {
          const double dxy[2] = {x[i] - x[j], y[i] - y[j]};
          const double r = std::hypot(dxy[0], dxy[1]);
          const double nuj[2] = {nux[j], nuy[j]};
          const Kernels<double> a = kernels(k2, dxy, r, nx, nuj, sp[j]);
          const Kernels<K> b = kernels(kp, dxy, r, nx, nuj, sp[j]);
          const double sn = std::sin(0.5 * h * (i - j));
          L = std::log(4.0 * sn * sn);
          m1s = a.s1 - b.s1; m1d = a.d1 - b.d1; m1n = a.n1 - b.n1; m1t = a.t1 - b.t1;
          ms = (a.s - b.s) - m1s * L;
          md = (a.d - b.d) - m1d * L;
          mn = (a.nn - b.nn) - m1n * L;
          mt = (a.t - b.t) - m1t * L;
        }
        const double rw = Rw[((i - j) % n + n) % n];
        A[(size_t)i * N2 + j] = rw * m1d + h * md + (i == j ? 1.0 : 0.0);
        A[(size_t)i * N2 + n + j] = rw * m1s + h * ms;
        A[(size_t)(n + i) * N2 + j] = rw * m1t + h * mt;
        A[(size_t)(n + i) * N2 + n + j] = rw * m1n + h * mn - (i == j ? 1.0 : 0.0);
      }
    }
  };
  {                                                      // the pairs' Bessel values dominate: rows over threads
    const unsigned hw = std::thread::hardware_concurrency();
    const int nt = std::max(1, std::min({(int)(hw ? hw : 4u), 16, n / 16}));
    const int chunk = (n + nt - 1) / nt;
    std::vector<std::thread> pool;
    for (int t = 1; t < nt; ++t) {
      const int i0 = t * chunk, i1 = std::min(n, i0 + chunk);
      if (i0 < i1) pool.emplace_back(assemble_rows, i0, i1);
    }
    assemble_rows(0, std::min(n, chunk));
    for (std::thread& th : pool) th.join();
  }
  // right-hand sides: -u_inc, -du_inc/dn for u_inc = J_m(k2 rho) e^{i m theta}, m = -p..p
  std::vector<cplx> B((size_t)N2 * P);
  for (int i = 0; i < n; ++i) {
    const double nr = (nux[i] * std::cos(th[i]) + nuy[i] * std::sin(th[i])) / sp[i];
    const double nt = (-nux[i] * std::sin(th[i]) + nuy[i] * std::cos(th[i])) / sp[i];
    const double z = k2 * rho[i];
    for (int m = -p; m <= p; ++m) {
      const cplx e = std::polar(1.0, m * th[i]);
      const double jm = bessel_jn(m, z);
      const double jmp = 0.5 * (bessel_jn(m - 1, z) - bessel_jn(m + 1, z));
      B[(size_t)i * P + m + p] = -jm * e;
      B[(size_t)(n + i) * P + m + p] = -(k2 * jmp * nr * e + cplx(0.0, m / rho[i]) * jm * nt * e);
    }
  }
  if (!solve_blocked(A, N2, B, P)) { err = "singular Muller system"; return LSMS_ERR_ARG; }
  // beta^m_l = (i/4) h sum_j [J_l e^{-i l theta} sigma |x'| + nu . grad(J_l e^{-i l theta}) mu]
  S.assign((size_t)P * P, cplx(0, 0));
  for (int j = 0; j < n; ++j) {
    const double z = k2 * rho[j];
    const double nr = nux[j] * std::cos(th[j]) + nuy[j] * std::sin(th[j]);    // |x'| n . e_rho
    const double nt = -nux[j] * std::sin(th[j]) + nuy[j] * std::cos(th[j]);   // |x'| n . e_theta
    for (int l = -p; l <= p; ++l) {
      const cplx e = std::polar(1.0, -l * th[j]);
      const double jl = bessel_jn(l, z);
      const double jlp = 0.5 * (bessel_jn(l - 1, z) - bessel_jn(l + 1, z));
      const cplx fs = jl * e * sp[j];
      const cplx fm = e * (k2 * jlp * nr - cplx(0.0, l / rho[j]) * jl * nt);
      for (int m = 0; m < P; ++m) {
        const cplx mu = B[(size_t)j * P + m], sigma = B[(size_t)(n + j) * P + m];
        S[(size_t)(l + p) * P + m] += cplx(0.0, 0.25 * h) * (fs * sigma + fm * mu);
      }
    }
  }
  for (const cplx& v : S)
    if (!std::isfinite(v.real()) || !std::isfinite(v.imag())) { err = "non-finite scattering matrix"; return LSMS_ERR_ARG; }
  return LSMS_OK;
}

static bool inclusion_args_ok(int p, double k2, double radius, int n_pts, const double* curve, const double* s_out) {
  return p >= 0 && p <= LSMS_MAX_P && std::isfinite(k2) && k2 > 0.0 && std::isfinite(radius) && radius > 0.0 &&
         n_pts >= 8 && n_pts <= 4096 && !(n_pts & 1) && curve && s_out;
}

extern "C" int lsms_inclusion_scattering_matrix(int p, double k2, double kp, double radius, int n_pts,
                                                const double* curve, double* s_out) {
  if (!inclusion_args_ok(p, k2, radius, n_pts, curve, s_out) || !std::isfinite(kp) || !(kp > 0.0))
    return ctx_fail(nullptr, LSMS_ERR_ARG,
                    "inclusion_scattering_matrix: need 0 <= p <= 15, k2, kp, radius > 0, an even n_pts in "
                    "[8, 4096], curve and output");
  std::vector<cplx> S;
  std::string err;
  const int rc = inclusion_matrix_t<double>(p, k2, kp, radius, n_pts, curve, S, err);
  if (rc) return ctx_fail(nullptr, rc, "inclusion_scattering_matrix: " + err);
  std::memcpy(s_out, S.data(), S.size() * sizeof(cplx));
  return LSMS_OK;
}

// An absorbing inclusion: complex kp (Re kp >= 0, Im kp >= 0) in the interior kernels, the same
// Muller system and product rule; Im kp = 0 is the call above.  The log part of Kress's split is
// J_0(kp r), J_1(kp r) over the whole curve, which grows like exp(Im kp r): the product rule and
// H = J + iY then lose about exp(Im kp * 2R) * 1e-16, hence Im kp * 2R <= 12 (1e-10 and better).
// |kp| * 2R <= 1e4 bounds the recurrence length (no curve of at most 4096 points resolves more).
extern "C" int lsms_inclusion_scattering_matrix_c(int p, double k2, double kp_re, double kp_im, double radius,
                                                  int n_pts, const double* curve, double* s_out) {
  if (!inclusion_args_ok(p, k2, radius, n_pts, curve, s_out) || !std::isfinite(kp_re) || !std::isfinite(kp_im) ||
      kp_re < 0.0 || kp_im < 0.0 || !(std::hypot(kp_re, kp_im) > 0.0) || kp_im * 2.0 * radius > 12.0 ||
      std::hypot(kp_re, kp_im) * 2.0 * radius > 1e4)
    return ctx_fail(nullptr, LSMS_ERR_ARG,
                    "inclusion_scattering_matrix_c: need 0 <= p <= 15, k2, radius > 0, Re kp >= 0, Im kp >= 0, "
                    "kp != 0, Im kp * 2 radius <= 12, |kp| * 2 radius <= 1e4, an even n_pts in [8, 4096], "
                    "curve and output");
  if (kp_im == 0.0) return lsms_inclusion_scattering_matrix(p, k2, kp_re, radius, n_pts, curve, s_out);
  std::vector<cplx> S;
  std::string err;
  const int rc = inclusion_matrix_t<cplx>(p, k2, cplx(kp_re, kp_im), radius, n_pts, curve, S, err);
  if (rc) return ctx_fail(nullptr, rc, "inclusion_scattering_matrix_c: " + err);
  std::memcpy(s_out, S.data(), S.size() * sizeof(cplx));
  return LSMS_OK;
}

// Perfectly conducting disc (Sec. 3.1, remark after Definition 3.1): the total field vanishes on
// the boundary, so S_n = -J_n(k2 R) / H_n(k2 R).
extern "C" int lsms_pec_scattering_diagonal(int p, double k2, double radius, double* s_diag) {
  if (p < 0 || p > LSMS_MAX_P || !std::isfinite(k2) || !(k2 > 0.0) || !std::isfinite(radius) || !(radius > 0.0) ||
      !s_diag)
    return ctx_fail(nullptr, LSMS_ERR_ARG, "pec_scattering_diagonal: need 0 <= p <= 15, k2 > 0, radius > 0");
  const double z = k2 * radius;
  for (int n = -p; n <= p; ++n) {
    const int an = std::abs(n);
    const double sg = (n < 0 && (an & 1)) ? -1.0 : 1.0;          // Z_{-n} = (-1)^n Z_n
    const double j = sg * std::cyl_bessel_j((double)an, z), y = sg * std::cyl_neumann((double)an, z);
    const cplx s = -j / cplx(j, y);
    s_diag[2 * (n + p)] = s.real();
    s_diag[2 * (n + p) + 1] = s.imag();
  }
  return LSMS_OK;
}

// Absorbing disc: complex k_p with Re k_p >= 0, Im k_p > 0 (a lossy or conducting interior).  The
// 2x2 mode system of Eq. "linear" divided by J_n(k_p R) leaves only the logarithmic derivative
// D_n = J_n'(z) / J_n(z) at z = k_p R:
//   S_n = (k_p D_n J_n(k2 R) - k2 J_n'(k2 R)) / (k2 H_n'(k2 R) - k_p D_n H_n(k2 R)),
// finite where J_n(z) itself overflows (Im z of several hundred).  With r_n = J_{n+1}(z) / J_n(z),
// D_n = n / z - r_n, and J_{n-1} + J_{n+1} = (2n / z) J_n gives r_{n-1} = 1 / (2n / z - r_n): run
// downward from r_N = 0 at N well above max(p, |z|), it converges to the ratio of the minimal
// solution J (Miller's backward recurrence in ratio form).  J_n has no zeros off the real axis, so
// no step divides by zero when Im z > 0.  S_{-n} = S_n.
static std::vector<cplx> mie_diagonal_c(int p, double k2, cplx kp, double R) {
  auto jn = [](int n, double x) {
    const double v = std::cyl_bessel_j((double)std::abs(n), x);
    return (n < 0 && (std::abs(n) & 1)) ? -v : v;
  };
  auto yn = [](int n, double x) {
    const double v = std::cyl_neumann((double)std::abs(n), x);
    return (n < 0 && (std::abs(n) & 1)) ? -v : v;
  };
  const cplx z = kp * R;
  const double az = std::abs(z);
  const int top = p + (int)std::ceil(az + 12.0 * std::cbrt(az)) + 60;
  std::vector<cplx> r(p + 1);
  cplx rn(0.0, 0.0);                                   // r_top
  for (int n = top; n >= 1; --n) {
    rn = 1.0 / (2.0 * n / z - rn);                     // r_{n-1}
    if (n - 1 <= p) r[n - 1] = rn;
  }
  std::vector<cplx> S(2 * p + 1);
  const double a = k2 * R;
  for (int n = 0; n <= p; ++n) {
    const cplx D = (double)n / z - r[n];
    const double j2 = jn(n, a), y2 = yn(n, a);
    const double j2p = 0.5 * (jn(n - 1, a) - jn(n + 1, a)), y2p = 0.5 * (yn(n - 1, a) - yn(n + 1, a));
    const cplx h(j2, y2), hp(j2p, y2p);
    S[p + n] = (kp * D * j2 - k2 * j2p) / (k2 * hp - kp * D * h);
    S[p - n] = S[p + n];
  }
  return S;
}

extern "C" int lsms_scattering_diagonal_c(int p, double k2, double kp_re, double kp_im, double radius,
                                          double* s_diag) {
  if (p < 0 || p > LSMS_MAX_P || !s_diag || !std::isfinite(k2) || !(k2 > 0.0) || !std::isfinite(kp_re) ||
      !std::isfinite(kp_im) || kp_re < 0.0 || kp_im < 0.0 || !(std::hypot(kp_re, kp_im) > 0.0) ||
      !std::isfinite(radius) || !(radius > 0.0) || std::hypot(kp_re, kp_im) * radius > 1e5)
    return ctx_fail(nullptr, LSMS_ERR_ARG,
                    "scattering_diagonal_c: need 0 <= p <= 15, k2 > 0, Re kp >= 0, Im kp >= 0, 0 < |kp| R <= 1e5, "
                    "radius > 0");
  const std::vector<cplx> S = kp_im == 0.0 ? mie_diagonal(p, k2, kp_re, radius)
                                           : mie_diagonal_c(p, k2, cplx(kp_re, kp_im), radius);
  std::memcpy(s_diag, S.data(), S.size() * sizeof(cplx));
  return LSMS_OK;
}

// ---------------------------------------------------------------------------------------------
// The context's scattering matrices
// ---------------------------------------------------------------------------------------------
extern "C" int lsms_set_scattering_matrix(lsms_ctx* c, const double* s) {
  if (!c) return LSMS_ERR_ARG;
  const int P = c->P;
  cudaStreamSynchronize(c->stream);
  batch_clear_graphs(c);
  if (!s) {
    c->dense = false;
    c->smat.clear();
  } else {
    std::vector<cplx> m((size_t)P * P);
    std::memcpy(static_cast<void*>(m.data()), s, m.size() * sizeof(cplx));
    for (const cplx& v : m)
      if (!std::isfinite(v.real()) || !std::isfinite(v.imag()))
        return ctx_fail(c, LSMS_ERR_ARG, "set_scattering_matrix: non-finite entry");
    // device tables, transposed ([n][l]) for the two output scalings: S and diag(|H_l(k2 R)|) S
    std::vector<cplx> t((size_t)2 * P * P);
    for (int l = 0; l < P; ++l)
      for (int q = 0; q < P; ++q) {
        t[(size_t)q * P + l] = m[(size_t)l * P + q];
        t[(size_t)P * P + (size_t)q * P + l] = c->hscale[l] * m[(size_t)l * P + q];
      }
    if (!c->d_smt && cudaMalloc((void**)&c->d_smt, t.size() * sizeof(cplx)) != cudaSuccess) {
      cudaGetLastError();
      c->d_smt = nullptr;
      return ctx_fail(c, LSMS_ERR_OOM, "set_scattering_matrix: cudaMalloc failed");
    }
    if (cudaMemcpy(c->d_smt, t.data(), t.size() * sizeof(cplx), cudaMemcpyHostToDevice) != cudaSuccess)
      return check_cuda(c, "set_scattering_matrix");
    c->smat = m;
    c->dense = true;
  }
  for (lsms_ctx* k : c->kids) {
    const int rc = lsms_set_scattering_matrix(k, s);
    if (rc) return ctx_fail(c, rc, std::string("set_scattering_matrix: ") + k->err);
  }
  return LSMS_OK;
}

extern "C" int lsms_set_orientations(lsms_ctx* c, int n, const double* theta) {
  if (!c) return LSMS_ERR_ARG;
  if (c->n < 0) return ctx_fail(c, LSMS_ERR_STATE, "call lsms_set_particles or lsms_set_layouts first");
  if (n != c->n) return ctx_fail(c, LSMS_ERR_ARG, "set_orientations: n must equal the number of particles");
  cudaStreamSynchronize(c->stream);
  batch_clear_graphs(c);
  if (!c->kids.empty()) {
    for (size_t l = 0; l < c->kids.size(); ++l) {
      lsms_ctx* k = c->kids[l];
      const int rc = lsms_set_orientations(k, k->n, theta ? theta + c->kid_off[l] : nullptr);
      if (rc) return ctx_fail(c, rc, "set_orientations: layout " + std::to_string(l) + ": " + k->err);
    }
    return LSMS_OK;
  }
  if (!theta || n == 0) {
    c->has_theta = false;
    return LSMS_OK;
  }
  for (int j = 0; j < n; ++j)
    if (!std::isfinite(theta[j])) return ctx_fail(c, LSMS_ERR_ARG, "set_orientations: non-finite angle");
  int rc;
  if ((rc = ensure(c, c->theta_buf, (size_t)n * sizeof(double)))) return rc;
  if (cudaMemcpy(c->theta_buf.ptr, theta, (size_t)n * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
    return check_cuda(c, "set_orientations");
  c->has_theta = true;
  return LSMS_OK;
}

extern "C" int lsms_get_scattering_matrix(const lsms_ctx* c, double* s) {
  if (!c || !s) return LSMS_ERR_ARG;
  const int P = c->P;
  std::vector<cplx> m((size_t)P * P, cplx(0, 0));
  if (c->dense)
    m = c->smat;
  else
    for (int q = 0; q < P; ++q) m[(size_t)q * P + q] = c->S[q];
  std::memcpy(s, m.data(), m.size() * sizeof(cplx));
  return LSMS_OK;
}
