// FP64 complex helpers and the pair Hankel sequence shared by the FP64 kernels (kernels_f64.cu,
// fmm.cu).
#pragma once

#include <cuda_runtime.h>

namespace {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {   // c + a b
  c.x = fma(a.x, b.x, c.x);
  c.x = fma(-a.y, b.y, c.x);
  c.y = fma(a.x, b.y, c.y);
  c.y = fma(a.y, b.x, c.y);
  return c;
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cexp_(double re, double im) {
  double s, c;
  sincos(im, &s, &c);
  const double m = exp(re);
  return make_double2(m * c, m * s);
}
__device__ __forceinline__ double2 warp_sum(double2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}

// h[s + 2p] = H_s(k rho) exp(i s phi) and hsum[s + 2p] = Re h + Im h, s = -2p..2p, for the pair
// offset (dx, dy) = x_l - x_m.  H_0, H_1 from the CUDA math library; H_{q+1} = (2q/z) H_q - H_{q-1}
// forward (stable normwise because the Y part dominates for q > z); H_{-q} = (-1)^q H_q.
__device__ void hankel_sequence_f64(double dx, double dy, double k, int p, double2* h, double* hsum) {
  const double rho = hypot(dx, dy);
  const double z = k * rho;
  const double2 e1 = make_double2(dx / rho, dy / rho);
  const int c0 = 2 * p;
  double2 hm = make_double2(j0(z), y0(z));
  double2 hq = make_double2(j1(z), y1(z));
  h[c0] = hm;
  hsum[c0] = hm.x + hm.y;
  double2 eq = e1;
  const double iz = 1.0 / z;
  for (int q = 1; q <= 2 * p; ++q) {
    const double2 v = cmul(hq, eq);
    h[c0 + q] = v;
    hsum[c0 + q] = v.x + v.y;
    double2 u = cmul(hq, make_double2(eq.x, -eq.y));
    if (q & 1) u = make_double2(-u.x, -u.y);
    h[c0 - q] = u;
    hsum[c0 - q] = u.x + u.y;
    if (q < 2 * p) {
      const double f = 2.0 * q * iz;
      const double2 hn = make_double2(f * hq.x - hm.x, f * hq.y - hm.y);
      hm = hq;
      hq = hn;
      eq = cmul(eq, e1);
    }
  }
}

}  // namespace
