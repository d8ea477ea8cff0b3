// Host-side setup of liblsms: contour nodes, disc scattering matrix, per-node layer constants,
// geometry validation.  Everything here runs once per lsms_create / lsms_set_particles, in FP64.
#include <algorithm>
#include <cmath>
#include <set>
#include <unordered_map>

#include "lsms_internal.h"
#include "lsms_ops.h"

static const double kPi = 3.14159265358979323846;

// Gauss-Legendre rule on [-1, 1] by Newton iteration on P_n, using the three-term recurrence
// (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1} and P_n' = n (x P_n - P_{n-1}) / (x^2 - 1).
// Nodes ascending.
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
    double pp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 1; k < n; ++k) {
        double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) { p1 = z; p0 = 1.0; }
      pp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / pp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) {
        // one more step with the converged value for the derivative
        p0 = 1.0; p1 = z;
        for (int k = 1; k < n; ++k) {
          double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
          p0 = p1;
          p1 = p2;
        }
        if (n == 1) { p1 = z; p0 = 1.0; }
        pp = n * (z * p1 - p0) / (z * z - 1.0);
        break;
      }
    }
    double wi = 2.0 / ((1.0 - z * z) * pp * pp);
    x[i] = -z;             // cos(...) is descending in i: store the negative side first
    x[n - 1 - i] = z;
    w[i] = wi;
    w[n - 1 - i] = wi;
  }
  if (n % 2 == 1) x[n / 2] = 0.0;
}

// Gamma1 panel breakpoints on [0, t_max]: 0, t_max, every branch point below t_max, graded
// geometrically toward each branch point (k +- b 2^j, j < L) with the largest L that keeps at most
// n_panels panels; then the longest panel is halved (first one on ties) until there are n_panels.
std::vector<double> contour_panel_breaks(int n_panels, const double* ks, int nk, double b,
                                         double t_max, double band_lo, double band_hi, bool greedy) {
  std::set<double> branch;
  for (int i = 0; i < nk; ++i)
    if (ks[i] > 0.0 && ks[i] < t_max) branch.insert(ks[i]);
  const bool has_band = band_hi > band_lo;
  if (has_band || greedy) {
    // guided-mode medium (poles of the layer response on the real axis in (band_lo, band_hi), a
    // distance b below Gamma1), or the greedy rule asked for: halve the panel with the largest
    // length / (b + distance to the nearest branch point) (distance 0 for a panel meeting the
    // band; first one on ties).
    std::set<double> s0 = branch;
    s0.insert(0.0);
    s0.insert(t_max);
    std::vector<double> pts(s0.begin(), s0.end());
    if ((int)pts.size() - 1 > n_panels) pts = {0.0, t_max};   // too few panels for every branch point
    auto score = [&](double a, double e) {
      double dist;
      if (has_band && e > band_lo && a < band_hi) {
        dist = 0.0;
      } else {
        dist = t_max;
        for (double s : branch) dist = std::min(dist, (a <= s && s <= e) ? 0.0 : std::min(std::abs(a - s), std::abs(e - s)));
      }
      return (e - a) / (b + dist);
    };
    while ((int)pts.size() - 1 < n_panels) {
      int best = 0;
      double bs = -1.0;
      for (size_t i = 0; i + 1 < pts.size(); ++i) {
        const double sc = score(pts[i], pts[i + 1]);
        if (sc > bs) { bs = sc; best = (int)i; }
      }
      pts.insert(pts.begin() + best + 1, 0.5 * (pts[best] + pts[best + 1]));
    }
    return pts;
  }
  int levels = 0;
  while (b * std::ldexp(1.0, levels) < t_max) ++levels;
  std::vector<double> pts;
  for (int lev = levels; lev >= 0; --lev) {
    std::set<double> cand = {0.0, t_max};
    for (double k : branch) {
      cand.insert(k);
      for (int j = 0; j < lev; ++j) {
        double off = b * std::ldexp(1.0, j);
        double lo = k - off, hi = k + off;
        if (lo > 0.0 && lo < t_max) cand.insert(lo);
        if (hi > 0.0 && hi < t_max) cand.insert(hi);
      }
    }
    if ((int)cand.size() - 1 <= n_panels) {
      pts.assign(cand.begin(), cand.end());
      break;
    }
  }
  if (pts.empty()) pts = {0.0, t_max};
  while ((int)pts.size() - 1 < n_panels) {
    int best = 0;
    double len = -1.0;
    for (size_t i = 0; i + 1 < pts.size(); ++i) {
      double l = pts[i + 1] - pts[i];
      if (l > len) { len = l; best = (int)i; }
    }
    pts.insert(pts.begin() + best + 1, 0.5 * (pts[best] + pts[best + 1]));
  }
  return pts;
}

int build_contour(const lsms_contour& c, const std::vector<double>& ks, std::vector<cplx>& lam,
                  std::vector<cplx>& wt, std::string& err) {
  const int q = c.panel_order > 0 ? c.panel_order : 16;
  const double b = c.b > 0.0 ? c.b : 0.2;
  const double t_max = c.t_max > 0.0 ? c.t_max : *std::max_element(ks.begin(), ks.end()) + 20.0;
  const int ns = c.n_nodes;
  if (ns <= 0 || q <= 0 || !std::isfinite(b) || !std::isfinite(t_max)) {
    err = "contour: n_nodes, panel_order, b and t_max must be positive and finite";
    return LSMS_ERR_ARG;
  }
  if (c.panel_rule != 0 && c.panel_rule != 1) {
    err = "contour: panel_rule must be 0 (graded) or 1 (greedy)";
    return LSMS_ERR_ARG;
  }
  const int n1 = q * ((ns - q) / (2 * q));
  const int n2 = ns - 2 * n1;
  if (n1 <= 0 || n2 <= 0) {
    err = "contour: n_nodes too small for the panel order";
    return LSMS_ERR_ARG;
  }
  // guided modes: evanescent in both half-spaces (lambda > max(k_top, k_bottom)) and propagating in
  // an interior layer (lambda < its k) -> poles of the layer response on the real axis
  double band_lo = std::max(ks.front(), ks.back()), band_hi = 0.0;
  for (size_t i = 1; i + 1 < ks.size(); ++i) band_hi = std::max(band_hi, ks[i]);
  std::vector<double> br =
      contour_panel_breaks(n1 / q, ks.data(), (int)ks.size(), b, t_max, band_lo, band_hi, c.panel_rule == 1);

  std::vector<double> gx, gw;
  gauss_legendre(q, gx, gw);
  std::vector<double> t1, w1;
  for (size_t i = 0; i + 1 < br.size(); ++i) {
    const double a = br[i], e = br[i + 1];
    for (int j = 0; j < q; ++j) {
      t1.push_back(0.5 * (a + e) + 0.5 * (e - a) * gx[j]);
      w1.push_back(0.5 * (e - a) * gw[j]);
    }
  }
  std::vector<double> sx, sw;
  gauss_legendre(n2, sx, sw);
  lam.assign(ns, cplx(0, 0));
  wt.assign(ns, cplx(0, 0));
  // Gamma3: mirror of Gamma1 (lambda -> -lambda), t increasing from -t_max to 0
  for (int i = 0; i < n1; ++i) {
    lam[i] = -cplx(t1[n1 - 1 - i], -b);
    wt[i] = cplx(w1[n1 - 1 - i], 0.0);
  }
  // Gamma2: lambda = i s, s from b down to -b, d lambda = i ds
  for (int i = 0; i < n2; ++i) {
    const double s = b * sx[n2 - 1 - i];
    lam[n1 + i] = cplx(0.0, s);
    wt[n1 + i] = cplx(0.0, -b * sw[n2 - 1 - i]);
  }
  // Gamma1: lambda = t - i b
  for (int i = 0; i < n1; ++i) {
    lam[n1 + n2 + i] = cplx(t1[i], -b);
    wt[n1 + n2 + i] = cplx(w1[i], 0.0);
  }
  return LSMS_OK;
}

// J_n, Y_n for integer n of any sign (J_{-n} = (-1)^n J_n, likewise Y), libstdc++ special math.
static double bes_j(int n, double x) {
  double v = std::cyl_bessel_j((double)std::abs(n), x);
  return (n < 0 && (std::abs(n) & 1)) ? -v : v;
}
static double bes_y(int n, double x) {
  double v = std::cyl_neumann((double)std::abs(n), x);
  return (n < 0 && (std::abs(n) & 1)) ? -v : v;
}

// Disc scattering matrix, Sec. 3.1: closed form of the 2x2 mode system Eq. "linear",
//   S_n = (kp J_n(k2R) J_n'(kpR) - k2 J_n'(k2R) J_n(kpR)) / (k2 H_n'(k2R) J_n(kpR) - kp J_n'(kpR) H_n(k2R)),
// with Z_n' = (Z_{n-1} - Z_{n+1})/2.
std::vector<cplx> mie_diagonal(int p, double k2, double kp, double R) {
  std::vector<cplx> S(2 * p + 1);
  const double a = k2 * R, bq = kp * R;
  for (int n = 0; n <= p; ++n) {
    const double j2 = bes_j(n, a), y2 = bes_y(n, a);
    const double j2p = 0.5 * (bes_j(n - 1, a) - bes_j(n + 1, a));
    const double y2p = 0.5 * (bes_y(n - 1, a) - bes_y(n + 1, a));
    const double jp = bes_j(n, bq);
    const double jpp = 0.5 * (bes_j(n - 1, bq) - bes_j(n + 1, bq));
    const cplx h(j2, y2), hp(j2p, y2p);
    const cplx num = kp * j2 * jpp - k2 * j2p * jp;
    const cplx den = k2 * hp * jp - kp * jpp * h;
    S[p + n] = num / den;
    S[p - n] = S[p + n];
  }
  return S;
}

std::vector<double> hankel_scale(int p, double k2, double R) {
  std::vector<double> h(2 * p + 1);
  for (int n = -p; n <= p; ++n) h[n + p] = std::hypot(bes_j(n, k2 * R), bes_y(n, k2 * R));
  return h;
}

// sqrt(lambda^2 - k^2) with Re >= 0, as -i sqrt(k^2 - lambda^2) (principal root).
cplx gamma_of(cplx lam, double k) { return cplx(0.0, -1.0) * std::sqrt(cplx(k * k, 0.0) - lam * lam); }
// absorbing layers (Im k > 0): Im(k^2 - lambda^2) >= 0 on the contour, so the principal root still
// gives Re gamma >= 0
cplx gamma_of(cplx lam, cplx k) { return cplx(0.0, -1.0) * std::sqrt(k * k - lam * lam); }

static cplx ipow(int n) {   // i^n for any integer n
  static const cplx t[4] = {cplx(1, 0), cplx(0, 1), cplx(-1, 0), cplx(0, -1)};
  return t[((n % 4) + 4) % 4];
}

// Gaussian elimination with partial pivoting: a (n x n, row-major) x = b (n x nrhs, row-major),
// solution in b.  False for a singular matrix.
bool solve_small(std::vector<cplx>& a, int n, std::vector<cplx>& b, int nrhs) {
  for (int k = 0; k < n; ++k) {
    int piv = k;
    for (int i = k + 1; i < n; ++i)
      if (std::abs(a[(size_t)i * n + k]) > std::abs(a[(size_t)piv * n + k])) piv = i;
    if (std::abs(a[(size_t)piv * n + k]) == 0.0) return false;
    if (piv != k) {
      for (int j = 0; j < n; ++j) std::swap(a[(size_t)k * n + j], a[(size_t)piv * n + j]);
      for (int j = 0; j < nrhs; ++j) std::swap(b[(size_t)k * nrhs + j], b[(size_t)piv * nrhs + j]);
    }
    for (int i = k + 1; i < n; ++i) {
      const cplx f = a[(size_t)i * n + k] / a[(size_t)k * n + k];
      if (f == cplx(0, 0)) continue;
      for (int j = k; j < n; ++j) a[(size_t)i * n + j] -= f * a[(size_t)k * n + j];
      for (int j = 0; j < nrhs; ++j) b[(size_t)i * nrhs + j] -= f * b[(size_t)k * nrhs + j];
    }
  }
  for (int k = n - 1; k >= 0; --k)
    for (int j = 0; j < nrhs; ++j) {
      cplx s = b[(size_t)k * nrhs + j];
      for (int i = k + 1; i < n; ++i) s -= a[(size_t)k * n + i] * b[(size_t)i * nrhs + j];
      b[(size_t)k * nrhs + j] = s / a[(size_t)k * n + k];
    }
  return true;
}

// Per-node constants.  The layer response (Sec. 2 Eq. "sommerfeldsys", generalised to any number of
// layers): interior layer j carries s_j^+ exp(g_j (y - z_{j-1})) + s_j^- exp(-g_j (y - z_j)) (over
// g_j, times exp(i lambda x)), layer 1 sigma_1 exp(-g_1 y), the bottom layer sigma_L exp(g_L (y -
// z_{L-1})); [u] = [du/dy] = 0 at the L - 1 interfaces.  The system is solved for a unit incident
// density I (line source in layer 1), a unit upgoing particle density P at the top of the disc layer
// and a unit downgoing one Q at its bottom; the tables are the linear maps (P, Q) -> (s_m^+, s_m^-),
// I -> (s_m^+, s_m^-) and (I, P, Q) -> sigma_1.
// The interface system of one node (see above) for unit I, P, Q: r[u][s] is unknown u (0: sigma_1,
// 1: s_m^+, 2: s_m^-, 3: sigma_L) for source s (0: I, 1: P, 2: Q); g receives gamma_j(lambda) of
// every layer.  NaN when the system is singular.
void layer_response(const lsms_ctx* c, cplx lam, std::vector<cplx>& g, cplx r[4][3]) {
  const int L = (int)c->ks.size(), m = c->layer, n = 2 * L - 2;
  auto col = [&](int j, int sign) {             // unknown of layer j (1-based)
    if (j == 1) return 0;
    if (j == L) return n - 1;
    return 1 + 2 * (j - 2) + (sign > 0 ? 0 : 1);
  };
  g.resize(L);
  std::vector<cplx> E(L + 1), a((size_t)n * n, cplx(0, 0)), b((size_t)n * 3, cplx(0, 0));
  for (int j = 1; j <= L; ++j) g[j - 1] = c->kc[j - 1].imag() == 0.0 ? gamma_of(lam, c->ks[j - 1]) : gamma_of(lam, c->kc[j - 1]);
  for (int j = 2; j < L; ++j) E[j] = std::exp(-g[j - 1] * c->ds[j - 2]);
  for (int i = 1; i < L; ++i) {                 // interface i: layer i above, i + 1 below
    const int rv = 2 * (i - 1), rd = rv + 1;
    const cplx gi = g[i - 1], gb = g[i];
    if (i == 1) {
      a[(size_t)rv * n + col(1, 1)] += 1.0 / gi;
      a[(size_t)rd * n + col(1, 1)] += -1.0;
    } else {
      a[(size_t)rv * n + col(i, 1)] += E[i] / gi;
      a[(size_t)rv * n + col(i, -1)] += 1.0 / gi;
      a[(size_t)rd * n + col(i, 1)] += E[i];
      a[(size_t)rd * n + col(i, -1)] += -1.0;
    }
    if (i + 1 == L) {
      a[(size_t)rv * n + col(L, 1)] -= 1.0 / gb;
      a[(size_t)rd * n + col(L, 1)] -= 1.0;
    } else {
      a[(size_t)rv * n + col(i + 1, 1)] -= 1.0 / gb;
      a[(size_t)rv * n + col(i + 1, -1)] -= E[i + 1] / gb;
      a[(size_t)rd * n + col(i + 1, 1)] -= 1.0;
      a[(size_t)rd * n + col(i + 1, -1)] += E[i + 1];
    }
    if (i == 1) {                               // incident wave, above interface 1
      b[(size_t)rv * 3 + 0] -= 1.0 / gi;
      b[(size_t)rd * 3 + 0] -= 1.0;
    }
    if (i == m - 1) {                           // discs' upgoing density, below this interface
      b[(size_t)rv * 3 + 1] += 1.0 / gb;
      b[(size_t)rd * 3 + 1] += -1.0;
    }
    if (i == m) {                               // discs' downgoing density, above this interface
      b[(size_t)rv * 3 + 2] -= 1.0 / gi;
      b[(size_t)rd * 3 + 2] -= 1.0;
    }
  }
  if (!solve_small(a, n, b, 3)) b.assign((size_t)n * 3, cplx(NAN, NAN));
  const int rows[4] = {0, col(m, 1), col(m, -1), n - 1};
  for (int u = 0; u < 4; ++u)
    for (int s = 0; s < 3; ++s) r[u][s] = b[(size_t)rows[u] * 3 + s];
}

void build_node_tables(lsms_ctx* c) {
  NodeTables& t = c->nodes;
  const int ns = c->ns, p = c->p, P = c->P;
  const int L = (int)c->ks.size(), m = c->layer;
  t.g1.resize(ns); t.g2.resize(ns); t.g3.resize(ns);
  t.refl.resize(4 * ns); t.inc.resize(2 * ns); t.field.resize(4 * ns);
  t.fagg.assign(2 * (size_t)ns * P, cplx(0, 0));
  t.udis.assign(2 * (size_t)ns * P, cplx(0, 0));
  std::vector<cplx> g;
  cplx r[4][3];
  for (int v = 0; v < ns; ++v) {
    const cplx lam = t.lam[v], w = t.wt[v];
    layer_response(c, lam, g, r);
    const cplx g1 = g[0], g2 = g[m - 1];
    t.g1[v] = g1; t.g2[v] = g2; t.g3[v] = g[L - 1];
    t.refl[4 * v + 0] = r[1][1];
    t.refl[4 * v + 1] = r[1][2];
    t.refl[4 * v + 2] = r[2][1];
    t.refl[4 * v + 3] = r[2][2];
    t.inc[2 * v + 0] = r[1][0];
    t.inc[2 * v + 1] = r[2][0];
    t.field[4 * v + 0] = r[0][0];
    t.field[4 * v + 1] = r[0][1];
    t.field[4 * v + 2] = r[0][2];
    t.field[4 * v + 3] = w / (4.0 * kPi * g1);
    const cplx wm = (lam - g2) / c->k2, wp = (lam + g2) / c->k2;
    const cplx q = w / (4.0 * kPi * g2);
    // powers w^n, n = -p..p, by repeated multiplication (w-^{-n} = w+^n since w- w+ = 1)
    std::vector<cplx> pm(P), pp(P);
    pm[p] = pp[p] = cplx(1, 0);
    for (int k = 1; k <= p; ++k) {
      pm[p + k] = pm[p + k - 1] * wm;
      pm[p - k] = pm[p - k + 1] * wp;
      pp[p + k] = pp[p + k - 1] * wp;
      pp[p - k] = pp[p - k + 1] * wm;
    }
    for (int k = -p; k <= p; ++k) {
      const cplx cn = 4.0 * ipow(-(k + 1)) ;   // 4 (-i)^{n+1} = 4 i^{-(n+1)}
      t.fagg[(size_t)v * P + k + p] = cn * pm[p + k];
      t.fagg[(size_t)(ns + v) * P + k + p] = cn * pp[p + k];
      t.udis[(size_t)v * P + k + p] = q * ipow(k) * pm[p + k];
      t.udis[(size_t)(ns + v) * P + k + p] = q * ipow(k) * pp[p + k];
    }
  }
}

// Discs must lie strictly inside the disc layer (centres given in absolute coordinates; the layer's
// top interface is `depth` below y = 0) and be separated by at least 10% of their diameter (the
// well-separation assumption of Sec. 1).
int validate_geometry(const lsms_ctx* c, int n, const double* xy, std::string& err) {
  const double R = c->R, gap = 0.2 * R, dmin = 2.0 * R + gap;
  for (int j = 0; j < n; ++j) {
    const double x = xy[2 * j], y = xy[2 * j + 1];
    if (!std::isfinite(x) || !std::isfinite(y)) {
      err = "set_particles: non-finite centre " + std::to_string(j);
      return LSMS_ERR_ARG;
    }
    if (!(y + c->depth + R < 0.0) || !(y + c->depth - R > -c->d)) {
      err = "set_particles: disc " + std::to_string(j) + " is not strictly inside the disc layer";
      return LSMS_ERR_GEOMETRY;
    }
  }
  std::unordered_map<long long, std::vector<int>> grid;
  auto key = [](long long i, long long k) { return (i << 32) ^ (k & 0xffffffffLL); };
  for (int j = 0; j < n; ++j) {
    const long long ix = (long long)std::floor(xy[2 * j] / dmin);
    const long long iy = (long long)std::floor(xy[2 * j + 1] / dmin);
    for (long long a = ix - 1; a <= ix + 1; ++a)
      for (long long b = iy - 1; b <= iy + 1; ++b) {
        auto it = grid.find(key(a, b));
        if (it == grid.end()) continue;
        for (int q : it->second) {
          const double dx = xy[2 * j] - xy[2 * q], dy = xy[2 * j + 1] - xy[2 * q + 1];
          if (dx * dx + dy * dy < dmin * dmin) {
            err = "set_particles: discs " + std::to_string(q) + " and " + std::to_string(j) +
                  " are closer than 2R + 0.2R";
            return LSMS_ERR_GEOMETRY;
          }
        }
      }
    grid[key(ix, iy)].push_back(j);
  }
  return LSMS_OK;
}
