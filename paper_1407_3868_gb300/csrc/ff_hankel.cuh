// FP32 Hankel sequences of a disc pair for the mixed-precision translation (Sec. 3.2 Lemma 3.1):
// float-float centre differences, the phase k rho reduced modulo 2 pi in float-float, H_0 and H_1
// from Hankel's large-argument expansion (or the FP64 library functions for near pairs), higher
// orders by the forward recurrence, and the angular factors exp(i s phi).
#pragma once

#include <cuda_runtime.h>

namespace {

// ---------------------------------------------------------------------------------------------
// float-float arithmetic (Dekker / Knuth error-free transformations)
// ---------------------------------------------------------------------------------------------
struct ffl {
  float hi, lo;
};
__device__ __forceinline__ ffl two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return {s, e};
}
__device__ __forceinline__ ffl fast_two_sum(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ ffl ff_add(ffl a, ffl b) {
  ffl s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ ffl ff_sub(ffl a, ffl b) { return ff_add(a, {-b.hi, -b.lo}); }
__device__ __forceinline__ ffl ff_mul(ffl a, ffl b) {
  const float p = a.hi * b.hi;
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
  return fast_two_sum(p, e);
}
__device__ __forceinline__ ffl ff_mul_f(ffl a, float b) {
  const float p = a.hi * b;
  float e = __fmaf_rn(a.hi, b, -p);
  e = __fmaf_rn(a.lo, b, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ ffl ff_sqrt(ffl a) {   // Karp: s + (a - s^2) / (2 s)
  const float s = sqrtf(a.hi);
  const float p = s * s;
  const float e = __fmaf_rn(s, s, -p);
  const ffl r = ff_sub(a, {p, e});
  return fast_two_sum(s, r.hi / (2.0f * s));
}

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

constexpr float kTwoPiHi = 6.28318548202514648f;      // float(2 pi)
constexpr float kTwoPiLo = -1.74845553146951427e-07f;  // 2 pi - float(2 pi)
constexpr float kInvTwoPi = 0.159154943091895336f;
constexpr float kZAsym = 25.0f;

// H_0(z), H_1(z) for z >= 25 from Hankel's expansion with the phase theta = z mod 2 pi in
// [-pi, pi]:  H_nu(z) ~ sqrt(2/(pi z)) exp(i (z - nu pi/2 - pi/4)) sum_k i^k a_k(nu) z^-k,
// a_k(nu) = prod_{j<=k} (4 nu^2 - (2j-1)^2) / (k! 8^k).  The hardware sine/cosine is used on the
// reduced phase (absolute error below 4e-7 there).
__device__ __forceinline__ void hankel01_asym(float zf, float theta, float2& h0, float2& h1) {
  float s, c;
  __sincosf(theta, &s, &c);
  const float iz = 1.0f / zf, iz2 = iz * iz;
  const float amp = sqrtf(0.636619772367581343f * iz) * 0.707106781186547524f;
  // nu = 0: a1 = -1/8, a2 = 9/128, a3 = -225/3072, a4 = 11025/98304
  const float p0 = 1.0f + iz2 * (-0.0703125f + iz2 * 0.112152099609375f);
  const float q0 = iz * (-0.125f + iz2 * 0.0732421875f);
  // nu = 1: a1 = 3/8, a2 = -15/128, a3 = 315/3072, a4 = -14175/98304
  const float p1 = 1.0f + iz2 * (0.1171875f + iz2 * -0.144195556640625f);
  const float q1 = iz * (0.375f + iz2 * -0.1025390625f);
  // exp(i(z - pi/4)) = (c + s + i (s - c)) / sqrt2 ; exp(i(z - 3pi/4)) = (s - c - i (s + c)) / sqrt2
  const float2 e0 = make_float2((c + s) * amp, (s - c) * amp);
  const float2 e1 = make_float2((s - c) * amp, -(s + c) * amp);
  h0 = cmulf(e0, make_float2(p0, q0));
  h1 = cmulf(e1, make_float2(p1, q1));
}

// Near pairs (z < 25, a handful per disc): FP64 library J0, Y0, J1, Y1.  Out of line so that the
// hot loop's instruction footprint stays small.
__device__ __noinline__ void hankel01_near(double z, float2* h0, float2* h1) {
  *h0 = make_float2((float)j0(z), (float)y0(z));
  *h1 = make_float2((float)j1(z), (float)y1(z));
}

// Geometry of a disc pair from float-float centres a (target) and b (source), given as
// (x_hi, x_lo, y_hi, y_lo): squared distance r2, the argument z = k rho (float-float and rounded)
// and the unit vector e1 = (cos phi, sin phi) of a - b.
struct PairGeom {
  ffl r2, z;
  float zf;
  float2 e1;
};
__device__ __forceinline__ PairGeom pair_geometry(float4 a, float4 b, ffl k) {
  PairGeom g;
  const ffl dx = ff_sub({a.x, a.y}, {b.x, b.y});
  const ffl dy = ff_sub({a.z, a.w}, {b.z, b.w});
  g.r2 = ff_add(ff_mul(dx, dx), ff_mul(dy, dy));
  const ffl rho = ff_sqrt(g.r2);
  g.z = ff_mul(rho, k);
  g.zf = g.z.hi + g.z.lo;
  const float irho = 1.0f / rho.hi;
  g.e1 = make_float2((dx.hi + dx.lo) * irho, (dy.hi + dy.lo) * irho);
  return g;
}

// H_0, H_1 at the pair's argument: Hankel's expansion with the float-float phase reduction for
// z >= 25, the FP64 library functions below.
__device__ __forceinline__ void hankel01_f32(const PairGeom& g, float2& h0, float2& h1) {
  if (g.zf >= kZAsym) {
    const float nq = rintf(g.z.hi * kInvTwoPi);
    const ffl t = ff_sub(g.z, ff_add(ff_mul_f({kTwoPiHi, 0.0f}, nq), ff_mul_f({kTwoPiLo, 0.0f}, nq)));
    hankel01_asym(g.zf, t.hi + t.lo, h0, h1);
  } else {
    hankel01_near((double)g.z.hi + (double)g.z.lo, &h0, &h1);
  }
}

// h[s + 2p] = H_s(z) exp(i s phi), s = -2p..2p, from H_0 and H_1: the forward recurrence
// H_{q+1} = (2q / z) H_q - H_{q-1}, the angular factors e1^q, and H_{-q} e^{-i q phi} =
// (-1)^q H_q conj(e1^q).  The order p is a template parameter, so the recurrence is unrolled.
template <int PT>
__device__ __forceinline__ void hankel_recurrence_f32(float2 h0, float2 h1, float2 e1, float zf, float2* h) {
  constexpr int p = PT;
  const int c0 = 2 * p;
  h[c0] = h0;
  float2 hm = h0, hq = h1, eq = e1;
  const float iz = 1.0f / zf;
#pragma unroll
  for (int q = 1; q <= 2 * p; ++q) {
    const float2 v = cmulf(hq, eq);
    h[c0 + q] = v;
    const float2 u = cmulf(hq, make_float2(eq.x, -eq.y));
    h[c0 - q] = (q & 1) ? make_float2(-u.x, -u.y) : u;
    if (q < 2 * p) {
      const float f = 2.0f * q * iz;
      const float2 hn = make_float2(f * hq.x - hm.x, f * hq.y - hm.y);
      hm = hq;
      hq = hn;
      eq = cmulf(eq, e1);
    }
  }
}

// Pair sequence h[s + 2p] = H_s(k rho) exp(i s phi), s = -2p..2p, for centres a (target) and b
// (source).  near_r2: squared distance (float-float) below which the pair is left to the near-pair
// kernel and its sequence is zero here; near_r2.hi <= 0 computes every pair here.
template <int PT>
__device__ __forceinline__ void hankel_sequence_f32(float4 a, float4 b, ffl k, ffl near_r2, float2* h) {
  const PairGeom g = pair_geometry(a, b, k);
  if (near_r2.hi > 0.0f && (g.r2.hi < near_r2.hi || (g.r2.hi == near_r2.hi && g.r2.lo < near_r2.lo))) {
#pragma unroll
    for (int q = 0; q <= 4 * PT; ++q) h[q] = make_float2(0.f, 0.f);
    return;
  }
  float2 h0, h1;
  hankel01_f32(g, h0, h1);
  hankel_recurrence_f32<PT>(h0, h1, g.e1, g.zf, h);
}

}  // namespace
