// Mixed-precision pieces of the operator: FP32 Graf translation (Sec. 3.2 Lemma 3.1) and the
// low-precision layout tables used by the mixed contour contractions.
//
// Translation in FP32.  Per pair the phase k2 rho is formed in float-float arithmetic from
// float-float centres (about 44 significant bits, so the phase of pairs thousands of wavelengths
// apart is still exact to ~1e-10 rad), reduced modulo 2 pi, and H_0, H_1 are evaluated from
// Hankel's asymptotic expansion (Abramowitz & Stegun 9.2.5-9.2.10, four terms, error < 3e-8 for
// z >= 25).  Pairs closer than z = 25 (a few per disc) use the FP64 library J0/Y0/J1/Y1.  Higher
// orders follow from the forward recurrence in FP32.  The contraction is a register-blocked
// Toeplitz product: a lane owns VB consecutive output orders of one target disc and slides a window
// of 2 VB - 1 sequence values over the source orders, so each staged value feeds VB complex FMAs.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <numeric>
#include <unordered_map>
#include <vector>

#include "lsms_internal.h"
#include "lsms_ops.h"
#include "ff_hankel.cuh"
#include "near_pairs.cuh"

namespace {

constexpr int MW = 4;      // warps per CTA
constexpr int MT = 8;      // target discs per warp
constexpr int MCH = 32;    // sources staged per chunk
// Pair slots: 32 per warp (8 targets x 4 sources), stride MHS float2.  A slot holds the 4p + 1
// values of one pair; windows of the contraction reach at most 3 entries before and 3 after them,
// into the zero margin of the neighbouring slot or the guard.  MHS = 65 = 1 (mod 16): the 32 lanes'
// window reads (offsets 2t - 16vb words) and the generator's stores hit distinct banks.
constexpr int MHS = 65;
constexpr int GUARD = 8;
constexpr size_t TRANSLATE_F32_SMEM = (size_t)(2 * GUARD + MW * 32 * MHS) * sizeof(float2);

// part[split][r][l][nu] = sum over the split's sources m != l of T^{lm} xs^m   (FP32)
// Lane roles.  Generation: lane = 8 s4 + t computes the pair (target t, source s4) into slot lane.
// Contraction: lane = 8 vb + t owns outputs nu = VB vb .. VB vb + VB - 1 of target t; for each
// staged source it slides a window of 2 VB - 1 sequence values over NB blocks of VB source orders.
// Complex products use three real FMAs (Gauss): A += hr br, B += hi bi, C += (hr+hi)(br+bi);
// re = A - B, im = C - A - B.
// RB coefficient vectors (right-hand sides r0 .. r0 + RB - 1) share every generated sequence.
// The order p is a template parameter: P = 2p + 1, VB = ceil(P/4) outputs per lane, NB = ceil(P/VB)
// blocks of source orders, and the padded tail of the last block is dropped at compile time.
template <int PT, int RB>
__global__ void __launch_bounds__(MW * 32, RB == 1 ? 3 : 2)
k_translate_f32(const float4* __restrict__ cff, int n, float k_hi, float k_lo,
                const float2* __restrict__ xs, float2* __restrict__ part, int src_per_split,
                int nrhs, float near_hi, float near_lo) {
  constexpr int p = PT;
  constexpr int P = 2 * PT + 1;
  constexpr int VB = (P + 3) / 4;
  constexpr int NB = (P + VB - 1) / VB;
  __shared__ float2 sb[RB][MCH][VB * NB + 1];
  __shared__ float4 sc[MCH];
  extern __shared__ float2 sh[];
  const int r0 = blockIdx.z * RB;
  const int split = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = lane & 7, hi8 = lane >> 3;       // hi8 = vb (contraction) = s4 (generation)
  const int l = (blockIdx.x * MW + warp) * MT + t;
  const bool lvalid = l < n;
  const float4 ct = lvalid ? cff[l] : make_float4(0.f, 0.f, 0.f, 0.f);
  for (int i = threadIdx.x; i < 2 * GUARD + MW * 32 * MHS; i += blockDim.x) sh[i] = make_float2(0.f, 0.f);
  float2* hw = sh + GUARD + warp * 32 * MHS;
  float A[RB][VB], B[RB][VB], C[RB][VB];
#pragma unroll
  for (int rr = 0; rr < RB; ++rr)
#pragma unroll
    for (int i = 0; i < VB; ++i) A[rr][i] = B[rr][i] = C[rr][i] = 0.f;
  const int jbeg = split * src_per_split;
  const int jend = min(n, jbeg + src_per_split);
  const ffl kf = {k_hi, k_lo};
  for (int j0c = jbeg; j0c < jend; j0c += MCH) {
    const int cnt = min(MCH, jend - j0c);
    __syncthreads();
    for (int i = threadIdx.x; i < RB * MCH * VB * NB; i += blockDim.x) {
      const int rr = i / (MCH * VB * NB), rem = i - rr * (MCH * VB * NB);
      const int s = rem / (VB * NB), q = rem - s * (VB * NB);
      sb[rr][s][q] = (s < cnt && q < P && r0 + rr < nrhs)
                         ? xs[((size_t)(r0 + rr) * n + j0c + s) * P + q] : make_float2(0.f, 0.f);
    }
    if (threadIdx.x < cnt) sc[threadIdx.x] = cff[j0c + threadIdx.x];
    __syncthreads();
    for (int s0 = 0; s0 < cnt; s0 += 4) {
      {
        const int js = s0 + hi8;
        float2* h = hw + lane * MHS;
        if (js < cnt && lvalid && j0c + js != l) {
          hankel_sequence_f32<PT>(ct, sc[js], kf, {near_hi, near_lo}, h);
        } else {
          for (int q = 0; q <= 4 * p; ++q) h[q] = make_float2(0.f, 0.f);
        }
      }
      __syncwarp();
      const int nq4 = min(4, cnt - s0);
      for (int q4 = 0; q4 < nq4; ++q4) {
        const float2* hs = hw + (q4 * 8 + t) * MHS + 2 * p - VB * hi8;   // hs[n - i]: output VB vb + i
        float2 win[2 * VB - 1];
        float wsum[2 * VB - 1];
#pragma unroll
        for (int j = 0; j < VB - 1; ++j) {
          win[j] = hs[j - (VB - 1)];
          wsum[j] = win[j].x + win[j].y;
        }
#pragma unroll
        for (int nb = 0; nb < NB; ++nb) {
#pragma unroll
          for (int j = 0; j < VB; ++j) {
            win[VB - 1 + j] = hs[nb * VB + j];
            wsum[VB - 1 + j] = win[VB - 1 + j].x + win[VB - 1 + j].y;
          }
#pragma unroll
          for (int u = 0; u < VB; ++u) {
            if (nb * VB + u >= P) break;            // padded source orders (compile time)
#pragma unroll
            for (int rr = 0; rr < RB; ++rr) {
              const float2 b = sb[rr][s0 + q4][nb * VB + u];
              const float bsum = b.x + b.y;
#pragma unroll
              for (int i = 0; i < VB; ++i) {
                const float2 hv = win[VB - 1 + u - i];
                A[rr][i] = __fmaf_rn(hv.x, b.x, A[rr][i]);
                B[rr][i] = __fmaf_rn(hv.y, b.y, B[rr][i]);
                C[rr][i] = __fmaf_rn(wsum[VB - 1 + u - i], bsum, C[rr][i]);
              }
            }
          }
#pragma unroll
          for (int j = 0; j < VB - 1; ++j) {
            win[j] = win[VB + j];
            wsum[j] = wsum[VB + j];
          }
        }
      }
      __syncwarp();
    }
  }
  if (lvalid) {
#pragma unroll
    for (int rr = 0; rr < RB; ++rr) {
      if (r0 + rr >= nrhs) break;
      float2* out = part + (((size_t)split * nrhs + r0 + rr) * n + l) * P;
#pragma unroll
      for (int i = 0; i < VB; ++i) {
        const int nu = VB * hi8 + i;
        if (nu < P) out[nu] = make_float2(A[rr][i] - B[rr][i], C[rr][i] - A[rr][i] - B[rr][i]);
      }
    }
  }
}

// One right-hand side per CTA, two lanes per target disc.  A warp owns MT2 = 16 target discs; lane
// (hh, t) owns the outputs nu = VB hh .. VB hh + VB - 1 of target t, VB = p + 1 (so P = 2p + 1
// orders fill 2 VB - 1 of the 2 VB output slots).  Per step the warp generates 32 pair sequences
// (lane (hh, t): target t, source s0 + hh) into its 32 slots; then each lane contracts both
// sources.  Per source order n the lane keeps a rolling window of the VB sequence values
// h_{n - nu} it needs, loads one new value and the source coefficient, and per output forms the
// Gauss products with one packed FMA (fma.rn.f32x2: h_r b_r and h_i b_i into the accumulator pair)
// and one FMA ((h_r + h_i)(b_r + b_i)): two issue slots for three FMAs.  The P source orders are
// unrolled (VB + VB - 1 steps; at p = 14 about 900 instructions, within the instruction cache).  The
// coefficient and its sum (b_r + b_i) are staged once per chunk, so the contraction spends one FADD
// (the window value's sum) per 3 VB FMAs.  Slots hold the 4p + 1 values of a pair with stride
// HS = 4p + 3 (odd: the 16 lanes of a half read 16 distinct bank pairs; at least 4p + 2: the upper
// half's first window read, one entry before its slot, lands in a zero margin or the guard).
template <int PT>
struct H2 {
  static constexpr int p = PT;
  static constexpr int P = 2 * PT + 1;
  static constexpr int VB = PT + 1;
  static constexpr int HS = 4 * PT + 3;
  static constexpr int SLOTS = MW * 32 * HS + 2 * GUARD;
  static constexpr size_t SMEM = (size_t)SLOTS * sizeof(float2);
};
constexpr int MT2 = 16;      // target discs per warp in the two-lanes-per-target kernel

// One CTA of the two-lanes-per-target translation: target tile `tile` (64 discs), source split
// `split`, right-hand side r (GRID: the block's own indices, as in a plain launch).
template <int PT, bool GRID>
__device__ __forceinline__ void h2_tile(const float4* __restrict__ cff, int n, float k_hi, float k_lo,
                                        const float2* __restrict__ xs, float2* __restrict__ part,
                                        int src_per_split, int nrhs, float near_hi, float near_lo, int row0,
                                        int nrows, int tile_arg, int split_arg, int r_arg) {
  constexpr int p = PT;
  constexpr int P = H2<PT>::P;
  constexpr int VB = H2<PT>::VB;
  constexpr int HS = H2<PT>::HS;
  __shared__ float2 sb[MCH][P];
  __shared__ float sbs[MCH][P];
  __shared__ float4 sc[MCH];
  extern __shared__ float2 sh[];
  const int r = GRID ? (int)blockIdx.z : r_arg;
  const int split = GRID ? (int)blockIdx.y : split_arg;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = lane & 15, hh = lane >> 4;       // hh = output half (contraction) = source (generation)
  const int tile = GRID ? (int)blockIdx.x : tile_arg;
  const int l = row0 + (tile * MW + warp) * MT2 + t;           // target rows row0 .. row0 + nrows - 1
  const bool lvalid = l < row0 + nrows && l < n;
  const float4 ct = lvalid ? cff[l] : make_float4(0.f, 0.f, 0.f, 0.f);
  for (int i = threadIdx.x; i < H2<PT>::SLOTS; i += blockDim.x) sh[i] = make_float2(0.f, 0.f);
  float2* hw = sh + GUARD + warp * 32 * HS;
  float2 AB[VB];             // (sum h_r b_r, sum h_i b_i): one packed FMA per window value
  float C[VB];               // sum (h_r + h_i)(b_r + b_i)
#pragma unroll
  for (int i = 0; i < VB; ++i) {
    AB[i] = make_float2(0.f, 0.f);
    C[i] = 0.f;
  }
  const int jbeg = split * src_per_split;
  const int jend = min(n, jbeg + src_per_split);
  const ffl kf = {k_hi, k_lo};
  const float2* xr = xs + (size_t)r * n * P;
  for (int j0c = jbeg; j0c < jend; j0c += MCH) {
    const int cnt = min(MCH, jend - j0c);
    __syncthreads();
    for (int i = threadIdx.x; i < MCH * P; i += blockDim.x) {
      const int s = i / P, q = i - s * P;
      const float2 v = s < cnt ? xr[(size_t)(j0c + s) * P + q] : make_float2(0.f, 0.f);
      sb[s][q] = v;
      sbs[s][q] = v.x + v.y;
    }
    if (threadIdx.x < cnt) sc[threadIdx.x] = cff[j0c + threadIdx.x];
    __syncthreads();
    for (int s0 = 0; s0 < cnt; s0 += 2) {
      {
        const int js = s0 + hh;
        float2* h = hw + lane * HS;
        if (js < cnt && lvalid && j0c + js != l) {
          hankel_sequence_f32<PT>(ct, sc[js], kf, {near_hi, near_lo}, h);
        } else {
          for (int q = 0; q <= 4 * p; ++q) h[q] = make_float2(0.f, 0.f);
        }
      }
      __syncwarp();
      const int nq = min(2, cnt - s0);
#pragma unroll 1
      for (int q2 = 0; q2 < nq; ++q2) {
        const float2* hs = hw + (q2 * 16 + t) * HS + 2 * p - VB * hh;   // hs[n - i] = h_{n - (VB hh + i)}
        const float2* bq = sb[s0 + q2];
        const float* bsq = sbs[s0 + q2];
        float2 win[VB];
        float ws[VB];
#pragma unroll
        for (int i = 0; i < VB - 1; ++i) {        // the window before the first shift: h_{-1 - i}
          win[i] = hs[-1 - i];
          ws[i] = win[i].x + win[i].y;
        }
        auto order = [&](int nn) {                   // source order nn: shift, load, 3 VB FMAs
#pragma unroll
          for (int i = VB - 1; i > 0; --i) {
            win[i] = win[i - 1];
            ws[i] = ws[i - 1];
          }
          win[0] = hs[nn];
          ws[0] = win[0].x + win[0].y;
          const float2 b = bq[nn];
          const float bsum = bsq[nn];
#pragma unroll
          for (int i = 0; i < VB; ++i) {
            AB[i] = __ffma2_rn(win[i], b, AB[i]);
            C[i] = __fmaf_rn(ws[i], bsum, C[i]);
          }
        };
#pragma unroll
        for (int u = 0; u < VB; ++u) order(u);
#pragma unroll
        for (int u = 0; u < VB - 1; ++u) order(VB + u);
      }
      __syncwarp();
    }
  }
  if (lvalid) {
    float2* out = part + (((size_t)split * nrhs + r) * nrows + (l - row0)) * P;
#pragma unroll
    for (int i = 0; i < VB; ++i) {
      const int nu = VB * hh + i;
      if (nu < P) out[nu] = make_float2(AB[i].x - AB[i].y, C[i] - AB[i].x - AB[i].y);
    }
  }
}

template <int PT>
__global__ void __launch_bounds__(MW * 32, 3)
k_translate_f32_h2(const float4* __restrict__ cff, int n, float k_hi, float k_lo,
                   const float2* __restrict__ xs, float2* __restrict__ part, int src_per_split,
                   int nrhs, float near_hi, float near_lo, int row0, int nrows) {
  h2_tile<PT, true>(cff, n, k_hi, k_lo, xs, part, src_per_split, nrhs, near_hi, near_lo, row0, nrows, 0, 0, 0);
}

// A batch of independent layouts in one launch: CTA b runs work item items[b] = (layout, tile,
// split) of the layout table (disc offset, disc count, sources per split, partial-sum offset);
// items are ordered by their layout's cost, largest first.  Centres, coefficients and partial sums
// of all layouts are concatenated.
template <int PT>
__global__ void __launch_bounds__(MW * 32, 3)
k_translate_f32_h2_batch(const float4* __restrict__ cff, const float2* __restrict__ xs,
                         float2* __restrict__ part, const int4* __restrict__ items,
                         const longlong4* __restrict__ lays, float k_hi, float k_lo, float near_hi,
                         float near_lo) {
  const int4 it = items[blockIdx.x];
  const longlong4 L = lays[it.x];                 // (disc offset, discs, sources per split, part offset)
  const int n = (int)L.y;
  h2_tile<PT, false>(cff + L.x, n, k_hi, k_lo, xs + L.x * H2<PT>::P, part + L.w, (int)L.z, 1, near_hi, near_lo,
                     0, n, it.y, it.z, 0);
}

// One pair sequence for both directions of a pair.  Turning phi by pi gives the reversed pair's
// sequence, h_s(m <- l) = (-1)^s h_s(l <- m), so out_nu(m) = (-1)^nu sum_n h_{n-nu}(l <- m)
// ((-1)^n x_n(l)): the sequence generated for l <- m, read with the same window as for the forward
// direction, also contracts l's sign-flipped coefficients into m's outputs, whose signs are
// flipped when they are written.  A CTA of two warps takes blocks (g1, g2), g1 <= g2, of 16-disc
// groups: eight steps per block, step k pairing target t of g1 with sources t + k and t + k + 8
// (mod 16) of g2, so that every disc of either group sits in two of the step's 32 pairs.  The
// warps take turns generating a step's 32 sequences into shared memory; then warp 0 contracts them
// into the targets' outputs and warp 1 into the sources' outputs, each with the two-lanes-per-disc
// register window of k_translate_f32_h2 (lane (hh, t): VB orders of disc t) and the same code
// (the role only picks the slot and the coefficient row).  Diagonal blocks (g1 = g2) already hold
// both directions of their pairs and are contracted by warp 0 alone.  Blocks form double rows h
// (g1 = h, g2 = h .. G - 1; then g1 = G - 1 - h, g2 = G - 1 - h .. G - 1: G + 1 blocks), and a CTA
// takes a run of `blocks_per_cta` blocks of one double row.  Outputs go into an FP32 accumulator
// (zeroed beforehand) by vector atomic adds: warp 0's when the target group changes, warp 1's after
// every block.
template <int PT>
struct Sym {
  static constexpr int P = 2 * PT + 1;
  static constexpr int VB = PT + 1;
  static constexpr int HS = 4 * PT + 3;                // slot stride, as in H2
  // float2 words: guard, 32 slots, warp 0's coefficients (source group), warp 1's (target group,
  // signs (-1)^nu), both groups' (re + im) sums as floats, the source group's centres (float4)
  static constexpr int WORDS = GUARD + 32 * HS + 3 * 16 * P + 32;
  static constexpr size_t SMEM = (size_t)WORDS * sizeof(float2);
};

// out_nu += sum_n hs[n - i] b_n for the lane's VB outputs nu (window and Gauss products as in
// h2_tile); hs points at the sequence value h_{-nu_0} of the lane's first output nu_0.
template <int PT>
__device__ __forceinline__ void window_contract(const float2* __restrict__ hs, const float2* __restrict__ bq,
                                                const float* __restrict__ bsq, float2 (&AB)[PT + 1],
                                                float (&C)[PT + 1]) {
  constexpr int VB = PT + 1;
  float2 win[VB];
  float ws[VB];
#pragma unroll
  for (int i = 0; i < VB - 1; ++i) {
    win[i] = hs[-1 - i];
    ws[i] = win[i].x + win[i].y;
  }
  auto order = [&](int nn) {
#pragma unroll
    for (int i = VB - 1; i > 0; --i) {
      win[i] = win[i - 1];
      ws[i] = ws[i - 1];
    }
    win[0] = hs[nn];
    ws[0] = win[0].x + win[0].y;
    const float2 b = bq[nn];
    const float bsum = bsq[nn];
#pragma unroll
    for (int i = 0; i < VB; ++i) {
      AB[i] = __ffma2_rn(win[i], b, AB[i]);
      C[i] = __fmaf_rn(ws[i], bsum, C[i]);
    }
  };
#pragma unroll
  for (int u = 0; u < VB; ++u) order(u);
#pragma unroll
  for (int u = 0; u < VB - 1; ++u) order(VB + u);
}

// Adds the lane's VB outputs of disc d (orders VB hh ..) into acc, times (-1)^nu when `flip`, and
// clears the accumulators.
template <int PT>
__device__ __forceinline__ void flush_outputs(float2* __restrict__ acc, int d, int n, int hh, bool flip,
                                              float2 (&AB)[PT + 1], float (&C)[PT + 1]) {
  constexpr int P = 2 * PT + 1, VB = PT + 1;
  if (d < n) {
#pragma unroll
    for (int i = 0; i < VB; ++i) {
      const int nu = VB * hh + i;
      if (nu < P) {
        const float sg = (flip && (nu & 1)) ? -1.0f : 1.0f;
        atomicAdd(acc + (size_t)d * P + nu,
                  make_float2(sg * (AB[i].x - AB[i].y), sg * (C[i] - AB[i].x - AB[i].y)));
      }
    }
  }
#pragma unroll
  for (int i = 0; i < VB; ++i) {
    AB[i] = make_float2(0.f, 0.f);
    C[i] = 0.f;
  }
}

// Stages the coefficients of group g (16 discs, zero past n) and their (re + im) sums, times
// (-1)^nu when `flip`.
template <int PT>
__device__ __forceinline__ void stage_group(const float2* __restrict__ xr, int g, int n, bool flip, int lane,
                                            float2* __restrict__ dst, float* __restrict__ dsum) {
  constexpr int P = 2 * PT + 1;
  const int d0 = 16 * g;
  for (int i = lane; i < 16 * P; i += 32) {
    const int s = i / P, q = i - s * P;
    float2 v = d0 + s < n ? xr[(size_t)d0 * P + i] : make_float2(0.f, 0.f);
    if (flip && (q & 1)) v = make_float2(-v.x, -v.y);
    dst[i] = v;
    dsum[i] = v.x + v.y;
  }
}

// One CTA of the symmetric translation: CTA `cta` of the layout's H per_row, right-hand side r
// (GRID: the block's own indices, as in a plain launch).
template <int PT, bool GRID>
__device__ __forceinline__ void sym_cta(const float4* __restrict__ cff, int n, float k_hi, float k_lo,
                                        const float2* __restrict__ xs, float2* __restrict__ acc,
                                        int blocks_per_cta, float near_hi, float near_lo, int cta_arg,
                                        int r_arg) {
  constexpr int p = PT;
  constexpr int P = Sym<PT>::P;
  constexpr int VB = Sym<PT>::VB;
  constexpr int HS = Sym<PT>::HS;
  extern __shared__ float2 sh[];
  const int role = threadIdx.x >> 5, lane = threadIdx.x & 31;   // role 0: forward, 1: reverse
  const int t = lane & 15, hh = lane >> 4;
  for (int i = threadIdx.x; i < Sym<PT>::WORDS; i += blockDim.x) sh[i] = make_float2(0.f, 0.f);
  __syncthreads();
  float2* slots = sh + GUARD;
  float2* sbF = slots + 32 * HS;
  float2* sbR = sbF + 16 * P;
  float* sFs = (float*)(sbR + 16 * P);
  float* sRs = sFs + 16 * P;
  float4* sc = (float4*)(sRs + 16 * P);
  const float2* coef = role ? sbR : sbF;
  const float* csum = role ? sRs : sFs;
  const int G = (n + 15) >> 4;
  const int per_row = (G + blocks_per_cta) / blocks_per_cta;       // ceil((G + 1) / blocks_per_cta)
  const int cta = GRID ? (int)blockIdx.x : cta_arg;                // cta < H per_row
  const int h = cta / per_row;
  const int b0 = (cta - h * per_row) * blocks_per_cta;
  const int b1 = min(G + 1, b0 + blocks_per_cta);
  const int r = GRID ? (int)blockIdx.y : r_arg;
  const float2* xr = xs + (size_t)r * n * P;
  float2* ar = acc + (size_t)r * n * P;
  const ffl kf = {k_hi, k_lo};
  const ffl nr = {near_hi, near_lo};
  float2 AB[VB];
  float C[VB];
#pragma unroll
  for (int i = 0; i < VB; ++i) {
    AB[i] = make_float2(0.f, 0.f);
    C[i] = 0.f;
  }
  int g1cur = -1;
  float4 ct = make_float4(0.f, 0.f, 0.f, 0.f);
  // Control flow is the same for both warps (it depends on the block index and the loop counters
  // only), so every __syncthreads below is reached by all 64 threads.
  for (int b = b0; b < b1; ++b) {
    int g1, g2;
    if (b < G - h) {
      g1 = h;
      g2 = h + b;
    } else {
      g1 = G - 1 - h;
      if (g1 == h) break;                             // the middle row of an odd G stands alone
      g2 = g1 + (b - (G - h));
    }
    if (g1 != g1cur) {
      if (g1cur >= 0 && role == 0) flush_outputs<PT>(ar, 16 * g1cur + t, n, hh, false, AB, C);
      g1cur = g1;
      if (role == 1) stage_group<PT>(xr, g1, n, true, lane, sbR, sRs);
      ct = 16 * g1 + t < n ? cff[16 * g1 + t] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (role == 0) {
      stage_group<PT>(xr, g2, n, false, lane, sbF, sFs);
      if (lane < 16) sc[lane] = 16 * g2 + lane < n ? cff[16 * g2 + lane] : make_float4(0.f, 0.f, 0.f, 0.f);
      __syncwarp();
    }
    const bool diag = g1 == g2;
    for (int k = 0; k < 8; ++k) {
      if (role == (k & 1)) {                          // the warps take turns generating
        const int s = (t + k + 8 * hh) & 15;
        const int a = 16 * g1 + t, m = 16 * g2 + s;
        float2* hq = slots + lane * HS;
        if (a < n && m < n && a != m) {
          hankel_sequence_f32<PT>(ct, sc[s], kf, nr, hq);
        } else {
          for (int q = 0; q <= 4 * p; ++q) hq[q] = make_float2(0.f, 0.f);
        }
      }
      __syncthreads();
      if (role == 0 || !diag) {
#pragma unroll 1
        for (int q2 = 0; q2 < 2; ++q2) {
          // warp 0: target t, source u = t + k + 8 q2 (slot q2 16 + t); warp 1: source t, target
          // u = t - k - 8 q2 (slot q2 16 + u, generated for u <- t)
          const int u = role ? ((t - k - 8 * q2) & 15) : ((t + k + 8 * q2) & 15);
          const int sl = q2 * 16 + (role ? u : t);
          window_contract<PT>(slots + sl * HS + 2 * p - VB * hh, coef + u * P, csum + u * P, AB, C);
        }
      }
      __syncthreads();
    }
    if (role == 1 && !diag) flush_outputs<PT>(ar, 16 * g2 + t, n, hh, true, AB, C);
  }
  if (role == 0 && g1cur >= 0) flush_outputs<PT>(ar, 16 * g1cur + t, n, hh, false, AB, C);
}

template <int PT>
__global__ void __launch_bounds__(64, 6)
k_translate_f32_sym(const float4* __restrict__ cff, int n, float k_hi, float k_lo,
                    const float2* __restrict__ xs, float2* __restrict__ acc, int blocks_per_cta,
                    float near_hi, float near_lo) {
  sym_cta<PT, true>(cff, n, k_hi, k_lo, xs, acc, blocks_per_cta, near_hi, near_lo, 0, 0);
}

// A batch of independent layouts in one launch: CTA b runs work item items[b] = (layout, CTA of
// that layout, blocks per CTA) of the layout table (disc offset, disc count); items are ordered by
// their layout's size, largest first.  Centres, coefficients and accumulators are concatenated.
template <int PT>
__global__ void __launch_bounds__(64, 6)
k_translate_f32_sym_batch(const float4* __restrict__ cff, const float2* __restrict__ xs,
                          float2* __restrict__ acc, const int4* __restrict__ items,
                          const longlong4* __restrict__ lays, float k_hi, float k_lo, float near_hi,
                          float near_lo) {
  const int4 it = items[blockIdx.x];
  const longlong4 L = lays[it.x];
  sym_cta<PT, false>(cff + L.x, (int)L.y, k_hi, k_lo, xs + L.x * Sym<PT>::P, acc + L.x * Sym<PT>::P, it.z,
                     near_hi, near_lo, it.y, 0);
}

// Near pairs (k2 rho < 25, a few per disc): Hankel's expansion does not hold there, so H_0 and H_1
// of every near pair are computed once per layout in FP64 (CUDA J0, Y0, J1, Y1) and stored in FP32
// (float4: H_0, H_1); the near-pair kernels generate the other orders by the FP32 forward recurrence
// from them.  The main FP32 kernel leaves these pairs out and k_translate_near adds them.
__global__ void k_near_h01(const double* __restrict__ cx, const double* __restrict__ cy,
                           const int* __restrict__ ptr, const int* __restrict__ idx, int n, double k,
                           float4* __restrict__ table) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n) return;
  for (int e = ptr[l]; e < ptr[l + 1]; ++e) {
    const int m = idx[e];
    const double z = k * hypot(cx[l] - cx[m], cy[l] - cy[m]);
    table[e] = make_float4((float)j0(z), (float)y0(z), (float)j1(z), (float)y1(z));
  }
}

// Batched reduction: alpha[i] = sum over the splits of element i's layout of its partial sums
// (one right-hand side; layouts by disc offset lays[l].x, ascending).
__global__ void k_reduce_parts_batch(const float2* __restrict__ part, const longlong4* __restrict__ lays, int nlay,
                                     long long total, int P, double2* __restrict__ alpha) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long d = i / P;
    int lo = 0, hi = nlay - 1;                     // last layout with offset <= d
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (lays[mid].x <= d) lo = mid;
      else hi = mid - 1;
    }
    const longlong4 L = lays[lo];
    const long long per = L.y * P, e = i - L.x * P;
    const int splits = (int)((L.y + L.z - 1) / L.z);
    double ax = 0.0, ay = 0.0;
    for (int sp = 0; sp < splits; ++sp) {
      const float2 v = part[L.w + sp * per + e];
      ax += v.x;
      ay += v.y;
    }
    alpha[i] = make_double2(ax, ay);
  }
}

template <int PT>
void launch_sym_batch(int ncta, cudaStream_t st, const float4* cff, const float2* xs, float2* acc, const int4* items,
                      const longlong4* lays, float kh, float kl, float nh, float nl) {
  k_translate_f32_sym_batch<PT><<<ncta, 64, Sym<PT>::SMEM, st>>>(cff, xs, acc, items, lays, kh, kl, nh, nl);
}

template <int PT>
void launch_h2_batch(int ncta, cudaStream_t st, const float4* cff, const float2* xs, float2* part, const int4* items,
                     const longlong4* lays, float kh, float kl, float nh, float nl) {
  static std::once_flag attr;
  std::call_once(attr, [] {
    cudaFuncSetAttribute(k_translate_f32_h2_batch<PT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)H2<PT>::SMEM);
  });
  k_translate_f32_h2_batch<PT><<<ncta, MW * 32, H2<PT>::SMEM, st>>>(cff, xs, part, items, lays, kh, kl, nh, nl);
}

// alpha[r][l][nu] = sum_split part[split][r][l][nu]   (double accumulation)
__global__ void k_reduce_parts(const float2* __restrict__ part, int nsplit, long long len,
                               double2* __restrict__ alpha) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len;
       i += (long long)gridDim.x * blockDim.x) {
    double ax = 0.0, ay = 0.0;
    for (int s = 0; s < nsplit; ++s) {
      const float2 v = part[(size_t)s * len + i];
      ax += v.x;
      ay += v.y;
    }
    alpha[i] = make_double2(ax, ay);
  }
}

__global__ void k_to_float(const double2* __restrict__ x, float2* __restrict__ y, long long len) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = make_float2((float)x[i].x, (float)x[i].y);
}

__global__ void k_centres_ff(const double* __restrict__ cx, const double* __restrict__ cy, int n,
                             float4* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const float xh = (float)cx[j], yh = (float)cy[j];
  out[j] = make_float4(xh, (float)(cx[j] - (double)xh), yh, (float)(cy[j] - (double)yh));
}

template <int PT, int RB>
void launch_pt(dim3 grid, cudaStream_t st, const float4* cff, int n, float kh, float kl,
               const float2* xs, float2* part, int sps, int nrhs, float nh, float nl) {
  static std::once_flag attr;
  std::call_once(attr, [] {
    cudaFuncSetAttribute(k_translate_f32<PT, RB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)TRANSLATE_F32_SMEM);
  });
  grid.z = (nrhs + RB - 1) / RB;
  k_translate_f32<PT, RB><<<grid, MW * 32, TRANSLATE_F32_SMEM, st>>>(cff, n, kh, kl, xs, part, sps, nrhs, nh, nl);
}

template <int PT>
void launch_h2(dim3 grid, cudaStream_t st, const float4* cff, int n, float kh, float kl,
               const float2* xs, float2* part, int sps, int nrhs, float nh, float nl, int row0, int nrows) {
  static std::once_flag attr;
  std::call_once(attr, [] {
    cudaFuncSetAttribute(k_translate_f32_h2<PT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)H2<PT>::SMEM);
  });
  grid.z = nrhs;
  k_translate_f32_h2<PT><<<grid, MW * 32, H2<PT>::SMEM, st>>>(cff, n, kh, kl, xs, part, sps, nrhs, nh, nl,
                                                             row0, nrows);
}

// Four or more right-hand sides (orders p >= 6) are contracted four at a time against each
// generated sequence (k_translate_f32<p, 4>, 32 target discs per CTA); otherwise one right-hand
// side per CTA in one of two tile shapes (`shape`, chosen by lsms_autotune): 0, two lanes per
// target (k_translate_f32_h2, 64 target discs per CTA); 1, four lanes per target
// (k_translate_f32<p, 1>, 32 target discs per CTA: twice the CTAs for small layouts).
bool translate_uses_block(int nrhs, int p) { return nrhs >= 4 && p >= 6; }
bool translate_uses_h2(int nrhs, int p, int shape = 0) { return !translate_uses_block(nrhs, p) && shape == 0; }
int translate_targets_per_cta(int nrhs, int p, int shape = 0) {
  return translate_uses_h2(nrhs, p, shape) ? MW * MT2 : MW * MT;
}

// grid.x must be ceil(n / translate_targets_per_cta(nrhs, p, shape)), or, for a range of target
// rows (nrows >= 0: rows row0 .. row0 + nrows - 1, always the two-lane kernel),
// ceil(nrows / (MW MT2)).
void launch_translate_kernel(dim3 grid, cudaStream_t st, const float4* cff, int n, int p, float kh,
                             float kl, const float2* xs, float2* part, int sps, int nrhs,
                             float nh = 0.f, float nl = 0.f, int row0 = 0, int nrows = -1, int shape = 0) {
  if (!translate_uses_block(nrhs, p) && nrows < 0 && shape == 1) {
#define LSMS_T1(PT) launch_pt<PT, 1>(grid, st, cff, n, kh, kl, xs, part, sps, nrhs, nh, nl)
    switch (p) {
      case 0: LSMS_T1(0); break;
      case 1: LSMS_T1(1); break;
      case 2: LSMS_T1(2); break;
      case 3: LSMS_T1(3); break;
      case 4: LSMS_T1(4); break;
      case 5: LSMS_T1(5); break;
      case 6: LSMS_T1(6); break;
      case 7: LSMS_T1(7); break;
      case 8: LSMS_T1(8); break;
      case 9: LSMS_T1(9); break;
      case 10: LSMS_T1(10); break;
      case 11: LSMS_T1(11); break;
      case 12: LSMS_T1(12); break;
      case 13: LSMS_T1(13); break;
      case 14: LSMS_T1(14); break;
      default: LSMS_T1(15); break;
    }
#undef LSMS_T1
    return;
  }
  if (nrows >= 0 || !translate_uses_block(nrhs, p)) {
    if (nrows < 0) nrows = n;
#define LSMS_H2(PT) launch_h2<PT>(grid, st, cff, n, kh, kl, xs, part, sps, nrhs, nh, nl, row0, nrows)
    switch (p) {
      case 0: LSMS_H2(0); break;
      case 1: LSMS_H2(1); break;
      case 2: LSMS_H2(2); break;
      case 3: LSMS_H2(3); break;
      case 4: LSMS_H2(4); break;
      case 5: LSMS_H2(5); break;
      case 6: LSMS_H2(6); break;
      case 7: LSMS_H2(7); break;
      case 8: LSMS_H2(8); break;
      case 9: LSMS_H2(9); break;
      case 10: LSMS_H2(10); break;
      case 11: LSMS_H2(11); break;
      case 12: LSMS_H2(12); break;
      case 13: LSMS_H2(13); break;
      case 14: LSMS_H2(14); break;
      default: LSMS_H2(15); break;
    }
#undef LSMS_H2
    return;
  }
#define LSMS_TB(PT) launch_pt<PT, 4>(grid, st, cff, n, kh, kl, xs, part, sps, nrhs, nh, nl)
  switch (p) {
    case 6: LSMS_TB(6); break;
    case 7: LSMS_TB(7); break;
    case 8: LSMS_TB(8); break;
    case 9: LSMS_TB(9); break;
    case 10: LSMS_TB(10); break;
    case 11: LSMS_TB(11); break;
    case 12: LSMS_TB(12); break;
    case 13: LSMS_TB(13); break;
    case 14: LSMS_TB(14); break;
    default: LSMS_TB(15); break;
  }
#undef LSMS_TB
}


// The symmetric translation (one sequence per unordered pair) of all n discs into acc (zeroed by the
// caller), runs of blocks sized so that the CTAs cover the GPU about 28 mult times (6 CTAs of two
// warps per SM).
template <int PT>
void launch_sym(cudaStream_t st, const float4* cff, int n, float kh, float kl, const float2* xs, float2* acc,
                int nrhs, float nh, float nl, double mult) {
  const int G = (n + 15) / 16, H = (G + 1) / 2;
  const double blocks = (double)H * (G + 1);
  const double ctas = std::max(1.0, mult * 152 * 6 * 28 / std::max(1, nrhs));
  const int L = std::max(1, std::min(G + 1, (int)std::ceil(blocks / ctas)));
  dim3 grid((unsigned)(H * ((G + L) / L)), nrhs);
  k_translate_f32_sym<PT><<<grid, 64, Sym<PT>::SMEM, st>>>(cff, n, kh, kl, xs, acc, L, nh, nl);
}

void launch_translate_sym(cudaStream_t st, const float4* cff, int n, int p, float kh, float kl,
                          const float2* xs, float2* acc, int nrhs, float nh, float nl, double mult) {
  if (n <= 0 || nrhs <= 0) return;
#define LSMS_SY(PT) launch_sym<PT>(st, cff, n, kh, kl, xs, acc, nrhs, nh, nl, mult)
  switch (p) {
    case 0: LSMS_SY(0); break;
    case 1: LSMS_SY(1); break;
    case 2: LSMS_SY(2); break;
    case 3: LSMS_SY(3); break;
    case 4: LSMS_SY(4); break;
    case 5: LSMS_SY(5); break;
    case 6: LSMS_SY(6); break;
    case 7: LSMS_SY(7); break;
    case 8: LSMS_SY(8); break;
    case 9: LSMS_SY(9); break;
    case 10: LSMS_SY(10); break;
    case 11: LSMS_SY(11); break;
    case 12: LSMS_SY(12); break;
    case 13: LSMS_SY(13); break;
    case 14: LSMS_SY(14); break;
    default: LSMS_SY(15); break;
  }
#undef LSMS_SY
}

}  // namespace

// CSR list of near pairs (k2 rho < 25) by target, from a cell grid, and their H_0, H_1 (FP64-built).
static int build_near_pairs(lsms_ctx* c) {
  void* old[] = {c->d_near_ptr, c->d_near_idx, c->d_near_h};
  for (void* q : old)
    if (q) cudaFree(q);
  c->d_near_ptr = nullptr;
  c->d_near_idx = nullptr;
  c->d_near_h = nullptr;
  c->near_nnz = 0;
  const int n = c->n;
  const double rn = (double)kZAsym / c->k2;
  c->near_r2 = rn * rn;
  std::vector<int> ptr(n + 1, 0), idx;
  std::unordered_map<long long, std::vector<int>> grid;
  auto key = [](long long i, long long k) { return (i << 32) ^ (k & 0xffffffffLL); };
  std::vector<double> xs(n);
  for (int j = 0; j < n; ++j) xs[j] = c->cx[j] - c->xc;
  for (int j = 0; j < n; ++j)
    grid[key((long long)std::floor(xs[j] / rn), (long long)std::floor(c->cy[j] / rn))].push_back(j);
  for (int l = 0; l < n; ++l) {
    const long long ix = (long long)std::floor(xs[l] / rn), iy = (long long)std::floor(c->cy[l] / rn);
    std::vector<int> row;
    for (long long a = ix - 1; a <= ix + 1; ++a)
      for (long long b = iy - 1; b <= iy + 1; ++b) {
        auto it = grid.find(key(a, b));
        if (it == grid.end()) continue;
        for (int m : it->second) {
          if (m == l) continue;
          const double dx = xs[l] - xs[m], dy = c->cy[l] - c->cy[m];
          if (dx * dx + dy * dy < c->near_r2) row.push_back(m);
        }
      }
    std::sort(row.begin(), row.end());
    idx.insert(idx.end(), row.begin(), row.end());
    ptr[l + 1] = (int)idx.size();
  }
  c->near_nnz = (int)idx.size();
  const size_t hb = (size_t)(c->near_nnz > 0 ? c->near_nnz : 1) * sizeof(float4);
  if (cudaMalloc((void**)&c->d_near_ptr, (n + 1) * sizeof(int)) != cudaSuccess ||
      cudaMalloc((void**)&c->d_near_idx, (idx.empty() ? 1 : idx.size()) * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&c->d_near_h, hb) != cudaSuccess) {
    cudaGetLastError();
    return ctx_fail(c, LSMS_ERR_OOM, "cudaMalloc failed for the near-pair tables");
  }
  cudaMemcpy(c->d_near_ptr, ptr.data(), (n + 1) * sizeof(int), cudaMemcpyHostToDevice);
  if (!idx.empty()) cudaMemcpy(c->d_near_idx, idx.data(), idx.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (n > 0 && c->near_nnz > 0)
    k_near_h01<<<(n + 127) / 128, 128, 0, c->stream>>>(c->d_cx, c->d_cy, c->d_near_ptr, c->d_near_idx, n, c->k2,
                                                       (float4*)c->d_near_h);
  cudaStreamSynchronize(c->stream);
  return check_cuda(c, "build_near_pairs");
}

int build_lowp_tables(lsms_ctx* c) {
  if (c->d_lp_misc) cudaFree(c->d_lp_misc);
  c->d_lp_misc = nullptr;
  if (cudaMalloc(&c->d_lp_misc, (size_t)(c->n > 0 ? c->n : 1) * sizeof(float4)) != cudaSuccess) {
    cudaGetLastError();
    return ctx_fail(c, LSMS_ERR_OOM, "cudaMalloc failed for the float-float centres");
  }
  if (c->n > 0)
    k_centres_ff<<<(c->n + 255) / 256, 256, 0, c->stream>>>(c->d_cx, c->d_cy, c->n, (float4*)c->d_lp_misc);
  cudaStreamSynchronize(c->stream);
  int rc = check_cuda(c, "build_lowp_tables");
  if (rc) return rc;
  if ((rc = build_near_pairs(c))) return rc;
  return tc_setup(c);
}

// Splits of the source range so that the grid covers the GPU several times (3 CTAs per SM for one
// right-hand side per CTA, 2 for four).
static int translate_splits(int n, int nrhs, int p, double mult = 1.0, int shape = 0) {
  const int tpc = translate_targets_per_cta(nrhs, p, shape);
  const int tiles = (n + tpc - 1) / tpc;
  const bool blk = translate_uses_block(nrhs, p);
  const int zb = blk ? (nrhs + 3) / 4 : nrhs;
  const int per_sm = blk ? 2 : 3;
  int s = (int)std::ceil(mult * (152 * per_sm * 4) / (double)(tiles * zb));
  const int max_s = (n + MCH - 1) / MCH;
  if (s > max_s) s = max_s;
  if (s < 1) s = 1;
  return s;
}

// The near pairs (k2 rho < 25) of the target rows row0 .. row0 + nrows - 1, added into alpha
// (rows of nrows): the pair-list kernel with the near-pair CSR (table row = list entry).
void launch_translate_near(lsms_ctx* c, int nrhs, const float2* xs32, double2* alpha, cudaStream_t st,
                           int row0, int nrows) {
  if (nrows < 0) nrows = c->n - row0;
  if (c->near_nnz <= 0 || nrows <= 0) return;
  launch_pair_lists(c->p, nrhs, st, nullptr, row0, std::min(nrows, c->n - row0), nrows,
                    (const float4*)c->d_lp_misc, c->d_near_ptr, c->d_near_idx, nullptr,
                    (const float4*)c->d_near_h, c->n, c->k2, xs32, alpha);
}

int translate_mixed(lsms_ctx* c, int nrhs, const double2* xs, double2* alpha, cudaStream_t st) {
  const int n = c->n, p = c->p, P = c->P;
  if (n == 0 || nrhs == 0) return LSMS_OK;
  const long long len = (long long)nrhs * n * P;
  const size_t b32 = (((size_t)len * sizeof(float2)) + 255) & ~size_t(255);
  long long g = (len + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  const bool tc = c->tc_min_rhs > 0 && nrhs >= c->tc_min_rhs && p >= 6 && p <= LSMS_MAX_P;
  const bool sym = !tc && c->f32_shape == 2 && !translate_uses_block(nrhs, p);
  int splits = 1, sps = n;
  if (!tc && !sym) {
    splits = translate_splits(n, nrhs, p, c->split_mult, c->f32_shape);
    sps = (n + splits - 1) / splits;
    sps = ((sps + MCH - 1) / MCH) * MCH;
    splits = (n + sps - 1) / sps;
  }
  int rc;
  if ((rc = ensure(c, c->ws_lp, b32 + (tc ? 0 : (size_t)splits * len * sizeof(float2))))) return rc;
  float2* xs32 = (float2*)c->ws_lp.ptr;
  k_to_float<<<(int)g, 256, 0, st>>>(xs, xs32, len);
  if (tc) {
    if ((rc = translate_mixed_tc(c, nrhs, xs, alpha, st))) return rc;
  } else if (sym) {
    float2* acc = (float2*)((unsigned char*)c->ws_lp.ptr + b32);
    const float kh = (float)c->k2, kl = (float)(c->k2 - (double)kh);
    const float nh = (float)c->near_r2, nl = (float)(c->near_r2 - (double)nh);
    cudaMemsetAsync(acc, 0, (size_t)len * sizeof(float2), st);
    launch_translate_sym(st, (const float4*)c->d_lp_misc, n, p, kh, kl, xs32, acc, nrhs, nh, nl, c->split_mult);
    k_reduce_parts<<<(int)g, 256, 0, st>>>(acc, 1, len, alpha);
  } else {
    float2* part = (float2*)((unsigned char*)c->ws_lp.ptr + b32);
    const float kh = (float)c->k2, kl = (float)(c->k2 - (double)kh);
    const int tpc = translate_targets_per_cta(nrhs, p, c->f32_shape);
    dim3 grid((n + tpc - 1) / tpc, splits, nrhs);
    const float nh = (float)c->near_r2, nl = (float)(c->near_r2 - (double)nh);
    launch_translate_kernel(grid, st, (const float4*)c->d_lp_misc, n, p, kh, kl, xs32, part, sps, nrhs, nh, nl,
                            0, -1, c->f32_shape);
    k_reduce_parts<<<(int)g, 256, 0, st>>>(part, splits, len, alpha);
  }
  launch_translate_near(c, nrhs, xs32, alpha, st);
  return check_cuda(c, "translate_mixed");
}

int translate_mixed_rows(lsms_ctx* c, int nrhs, const double2* xs, double2* alpha_rows, int row0, int nrows,
                         cudaStream_t st) {
  const int n = c->n, p = c->p, P = c->P;
  if (n == 0 || nrhs == 0 || nrows == 0) return LSMS_OK;
  const long long len = (long long)nrhs * n * P, len_rows = (long long)nrhs * nrows * P;
  const size_t b32 = (((size_t)len * sizeof(float2)) + 255) & ~size_t(255);
  const int tpc = MW * MT2;
  const int tiles = (nrows + tpc - 1) / tpc;
  int splits = (int)std::ceil(c->split_mult * (152 * 3 * 4) / (double)(tiles * nrhs));
  splits = std::max(1, std::min(splits, (n + MCH - 1) / MCH));
  int sps = (n + splits - 1) / splits;
  sps = ((sps + MCH - 1) / MCH) * MCH;
  splits = (n + sps - 1) / sps;
  int rc;
  if ((rc = ensure(c, c->ws_lp, b32 + (size_t)splits * len_rows * sizeof(float2)))) return rc;
  float2* xs32 = (float2*)c->ws_lp.ptr;
  float2* part = (float2*)((unsigned char*)c->ws_lp.ptr + b32);
  long long g = (len + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  k_to_float<<<(int)g, 256, 0, st>>>(xs, xs32, len);
  const float kh = (float)c->k2, kl = (float)(c->k2 - (double)kh);
  const float nh = (float)c->near_r2, nl = (float)(c->near_r2 - (double)nh);
  dim3 grid(tiles, splits, nrhs);
  launch_translate_kernel(grid, st, (const float4*)c->d_lp_misc, n, p, kh, kl, xs32, part, sps, nrhs, nh, nl,
                          row0, nrows);
  long long gr = (len_rows + 255) / 256;
  if (gr > 152 * 16) gr = 152 * 16;
  k_reduce_parts<<<(int)gr, 256, 0, st>>>(part, splits, len_rows, alpha_rows);
  launch_translate_near(c, nrhs, xs32, alpha_rows, st, row0, nrows);
  return check_cuda(c, "translate_mixed_rows");
}

// ---------------------------------------------------------------------------------------------
// A layout batch's mixed all-pairs translation in one launch.  The work items (layout, target tile of
// 64 discs, source split) of every layout form one grid, ordered by the layout's size, largest
// first, so that the long tiles start early; the splits are chosen so that the grid covers the GPU
// about four times.  The centres and the near-pair lists of all layouts are concatenated (pairs
// never cross layouts).
void batch_translation_free(lsms_ctx* c) {
  void* ptrs[] = {c->d_bt_items, c->d_bt_lays, c->d_bt_cff, c->d_bt_nptr, c->d_bt_nidx, c->d_bt_ntab};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  c->d_bt_items = c->d_bt_lays = c->d_bt_cff = c->d_bt_ntab = nullptr;
  c->d_bt_nptr = c->d_bt_nidx = nullptr;
  if (c->bt_ev) cudaEventDestroy(c->bt_ev);
  c->bt_ev = nullptr;
  if (c->ws_bt.ptr) cudaFree(c->ws_bt.ptr);
  c->ws_bt = DevBuf();
  c->bt_ready = false;
  c->bt_ncta = 0;
  c->bt_part = 0;
}

// Work items of the symmetric kernel: one run length for all layouts (clamped to each layout's
// double-row length), CTAs of the largest layout first.
static void sym_batch_items(lsms_ctx* c, std::vector<longlong4>& lays, std::vector<int4>& items) {
  const int nl = (int)c->kids.size();
  double blocks = 0.0;
  for (int l = 0; l < nl; ++l) {
    const int G = (c->kids[l]->n + 15) / 16;
    blocks += (double)((G + 1) / 2) * (G + 1);
    lays[l] = make_longlong4(c->kid_off[l], c->kids[l]->n, 0, 0);
  }
  const double target = 152.0 * 6 * 7 * std::max(1, c->bt_waves);
  const int Lg = std::max(1, (int)std::ceil(blocks / target));
  std::vector<int> order(nl);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return c->kids[a]->n > c->kids[b]->n; });
  for (int l : order) {
    const int G = (c->kids[l]->n + 15) / 16, H = (G + 1) / 2;
    const int L = std::min(Lg, G + 1);
    const int ctas = H * ((G + L) / L);
    for (int k = 0; k < ctas; ++k) items.push_back(make_int4(l, k, L, 0));
  }
}

int batch_translation_items(lsms_ctx* c) {
  const int nl = (int)c->kids.size();
  const int P = c->P;
  const int tpc = MW * MT2;
  long long tiles_all = 0;
  for (int l = 0; l < nl; ++l) tiles_all += (c->kids[l]->n + tpc - 1) / tpc;
  const long long target = 152LL * 3 * std::max(1, c->bt_waves);
  const int want = (int)std::max<long long>(1, (target + tiles_all - 1) / std::max<long long>(tiles_all, 1));
  std::vector<longlong4> lays(nl);
  std::vector<int> splits(nl);
  long long part = 0;
  for (int l = 0; l < nl; ++l) {
    const int n = c->kids[l]->n;
    int sp = std::max(1, std::min(want, (n + MCH - 1) / MCH));
    int sps = std::max(1, (n + sp - 1) / sp);
    sps = ((sps + MCH - 1) / MCH) * MCH;
    sp = n > 0 ? (n + sps - 1) / sps : 0;
    splits[l] = sp;
    lays[l] = make_longlong4(c->kid_off[l], n, sps, part);
    part += (long long)sp * n * P;
  }
  std::vector<int> order(nl);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return c->kids[a]->n > c->kids[b]->n; });
  std::vector<int4> items;
  if (c->bt_shape == 2) {
    sym_batch_items(c, lays, items);
    part = c->kid_off.back() * P;                    // one FP32 accumulator
  } else {
    for (int l : order) {
      const int tiles = (c->kids[l]->n + tpc - 1) / tpc;
      for (int t = 0; t < tiles; ++t)
        for (int sp = 0; sp < splits[l]; ++sp) items.push_back(make_int4(l, t, sp, 0));
    }
  }
  if (c->d_bt_items) cudaFree(c->d_bt_items);
  if (c->d_bt_lays) cudaFree(c->d_bt_lays);
  c->d_bt_items = c->d_bt_lays = nullptr;
  if (cudaMalloc(&c->d_bt_items, std::max<size_t>(1, items.size()) * sizeof(int4)) != cudaSuccess ||
      cudaMalloc(&c->d_bt_lays, nl * sizeof(longlong4)) != cudaSuccess) {
    cudaGetLastError();
    return ctx_fail(c, LSMS_ERR_OOM, "batched translation: cudaMalloc failed for the work items");
  }
  cudaMemcpy(c->d_bt_items, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice);
  cudaMemcpy(c->d_bt_lays, lays.data(), nl * sizeof(longlong4), cudaMemcpyHostToDevice);
  c->bt_ncta = (int)items.size();
  c->bt_part = part;
  return check_cuda(c, "batched translation work items");
}

int batch_translation_setup(lsms_ctx* c) {
  batch_translation_free(c);
  const int nl = (int)c->kids.size();
  if (nl == 0 || c->p > LSMS_MAX_P || c->kid_off.back() == 0) return LSMS_OK;
  const long long total = c->kid_off.back();
  // near pairs of all layouts, global disc indices
  std::vector<int> nptr(total + 1, 0), nidx;
  long long nnz = 0;
  for (int l = 0; l < nl; ++l) nnz += std::max(c->kids[l]->near_nnz, 0);
  nidx.resize((size_t)std::max<long long>(nnz, 1));
  if (cudaMalloc(&c->d_bt_cff, total * sizeof(float4)) != cudaSuccess ||
      cudaMalloc((void**)&c->d_bt_nptr, (total + 1) * sizeof(int)) != cudaSuccess ||
      cudaMalloc((void**)&c->d_bt_nidx, (size_t)std::max<long long>(nnz, 1) * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&c->d_bt_ntab, (size_t)std::max<long long>(nnz, 1) * sizeof(float4)) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->bt_ev, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    batch_translation_free(c);
    return ctx_fail(c, LSMS_ERR_OOM, "set_layouts: cudaMalloc failed for the batched translation");
  }
  long long e0 = 0;
  for (int l = 0; l < nl; ++l) {
    lsms_ctx* k = c->kids[l];
    const long long off = c->kid_off[l];
    const int n = k->n, kn = std::max(k->near_nnz, 0);
    if (n <= 0) continue;
    std::vector<int> kp(n + 1), ki((size_t)std::max(kn, 1));
    if (cudaMemcpy((float4*)c->d_bt_cff + off, k->d_lp_misc, n * sizeof(float4), cudaMemcpyDeviceToDevice) !=
            cudaSuccess ||
        cudaMemcpy(kp.data(), k->d_near_ptr, (n + 1) * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
        (kn > 0 && (cudaMemcpy(ki.data(), k->d_near_idx, kn * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
                    cudaMemcpy((float4*)c->d_bt_ntab + e0, k->d_near_h, kn * sizeof(float4),
                               cudaMemcpyDeviceToDevice) != cudaSuccess))) {
      batch_translation_free(c);
      return check_cuda(c, "set_layouts: batched translation tables");
    }
    for (int i = 0; i < n; ++i) nptr[off + i] = (int)(e0 + kp[i]);
    for (int e = 0; e < kn; ++e) nidx[e0 + e] = (int)(off + ki[e]);
    e0 += kn;
  }
  nptr[total] = (int)e0;
  cudaMemcpy(c->d_bt_nptr, nptr.data(), (total + 1) * sizeof(int), cudaMemcpyHostToDevice);
  if (nnz > 0) cudaMemcpy(c->d_bt_nidx, nidx.data(), nnz * sizeof(int), cudaMemcpyHostToDevice);
  int rc = batch_translation_items(c);
  if (rc) {
    batch_translation_free(c);
    return rc;
  }
  c->bt_ready = true;
  return check_cuda(c, "set_layouts: batched translation tables");
}

int translate_mixed_batch(lsms_ctx* c, const double2* xs, double2* alpha, cudaStream_t st) {
  if (!c->bt_ready) return ctx_fail(c, LSMS_ERR_STATE, "batched translation tables are not built");
  const int p = c->p, P = c->P;
  const long long total = c->kid_off.back(), len = total * P;
  const size_t b32 = (((size_t)len * sizeof(float2)) + 255) & ~size_t(255);
  int rc;
  if ((rc = ensure(c, c->ws_bt, b32 + (size_t)c->bt_part * sizeof(float2)))) return rc;
  float2* xs32 = (float2*)c->ws_bt.ptr;
  float2* part = (float2*)((unsigned char*)c->ws_bt.ptr + b32);
  long long g = (len + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  k_to_float<<<(int)g, 256, 0, st>>>(xs, xs32, len);
  const float kh = (float)c->k2, kl = (float)(c->k2 - (double)kh);
  const double nr = c->kids[0]->near_r2;
  const float nh = (float)nr, nl = (float)(nr - (double)nh);
  const float4* cff = (const float4*)c->d_bt_cff;
  const int4* items = (const int4*)c->d_bt_items;
  const longlong4* lays = (const longlong4*)c->d_bt_lays;
  if (c->bt_shape == 2) {
    cudaMemsetAsync(part, 0, (size_t)len * sizeof(float2), st);
    if (c->bt_ncta > 0) {
#define LSMS_SB(PT) launch_sym_batch<PT>(c->bt_ncta, st, cff, xs32, part, items, lays, kh, kl, nh, nl)
      switch (p) {
        case 0: LSMS_SB(0); break;
        case 1: LSMS_SB(1); break;
        case 2: LSMS_SB(2); break;
        case 3: LSMS_SB(3); break;
        case 4: LSMS_SB(4); break;
        case 5: LSMS_SB(5); break;
        case 6: LSMS_SB(6); break;
        case 7: LSMS_SB(7); break;
        case 8: LSMS_SB(8); break;
        case 9: LSMS_SB(9); break;
        case 10: LSMS_SB(10); break;
        case 11: LSMS_SB(11); break;
        case 12: LSMS_SB(12); break;
        case 13: LSMS_SB(13); break;
        case 14: LSMS_SB(14); break;
        default: LSMS_SB(15); break;
      }
#undef LSMS_SB
    }
    k_reduce_parts<<<(int)g, 256, 0, st>>>(part, 1, len, alpha);
  } else {
    if (c->bt_ncta > 0) {
#define LSMS_HB(PT) launch_h2_batch<PT>(c->bt_ncta, st, cff, xs32, part, items, lays, kh, kl, nh, nl)
      switch (p) {
        case 0: LSMS_HB(0); break;
        case 1: LSMS_HB(1); break;
        case 2: LSMS_HB(2); break;
        case 3: LSMS_HB(3); break;
        case 4: LSMS_HB(4); break;
        case 5: LSMS_HB(5); break;
        case 6: LSMS_HB(6); break;
        case 7: LSMS_HB(7); break;
        case 8: LSMS_HB(8); break;
        case 9: LSMS_HB(9); break;
        case 10: LSMS_HB(10); break;
        case 11: LSMS_HB(11); break;
        case 12: LSMS_HB(12); break;
        case 13: LSMS_HB(13); break;
        case 14: LSMS_HB(14); break;
        default: LSMS_HB(15); break;
      }
#undef LSMS_HB
    }
    k_reduce_parts_batch<<<(int)g, 256, 0, st>>>(part, lays, (int)c->kids.size(), len, P, alpha);
  }
  launch_pair_lists(p, 1, st, nullptr, 0, (int)total, (int)total, cff, c->d_bt_nptr, c->d_bt_nidx, nullptr,
                    (const float4*)c->d_bt_ntab, (int)total, c->k2, xs32, alpha);
  return check_cuda(c, "translate_mixed_batch");
}

// ---------------------------------------------------------------------------------------------
// Allocation-free variant of the FP32 translation (lsms_translate_mixed_noalloc).
//
// Its scratch (float-float centres and the per-split FP32 partial sums) lives in the file-scope
// device array below instead of memory obtained from cudaMalloc.  Every GPU that loads the library
// holds these 16 MiB until the process exits.  Host code cannot pass the array's name to a kernel
// (on the host it is only a stand-in symbol), so the device address is looked up once per device
// with cudaGetSymbolAddress and cached.
// ---------------------------------------------------------------------------------------------
#include <mutex>

constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device (looked up on first use).
int noalloc_scratch(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return ctx_fail(nullptr, LSMS_ERR_CUDA, "translate_mixed_noalloc: no current CUDA device");
  }
  if (dev < 0 || dev >= kMaxDevices)
    return ctx_fail(nullptr, LSMS_ERR_CUDA, "translate_mixed_noalloc: device index out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return ctx_fail(nullptr, LSMS_ERR_CUDA,
                      std::string("translate_mixed_noalloc: cudaGetSymbolAddress failed: ") +
                          cudaGetErrorString(e));
    }
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return LSMS_OK;
}

__global__ void k_centres_ff_xy(const double* __restrict__ xy, int n, float4* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double x = xy[2 * j], y = xy[2 * j + 1];
  const float xh = (float)x, yh = (float)y;
  out[j] = make_float4(xh, (float)(x - (double)xh), yh, (float)(y - (double)yh));
}

}  // namespace

extern "C" int lsms_translate_mixed_noalloc(int n, int p, double k2, int nrhs,
                                            const double* centres_xy, const double* beta,
                                            double* alpha, void* stream) {
  if (n < 0 || nrhs < 0 || p < 0 || p > LSMS_MAX_P || !std::isfinite(k2) || !(k2 > 0.0))
    return ctx_fail(nullptr, LSMS_ERR_ARG, "translate_mixed_noalloc: need n >= 0, nrhs >= 0, 0 <= p <= 15, k2 > 0");
  if (n == 0 || nrhs == 0) return LSMS_OK;
  if (!centres_xy || !beta || !alpha) return ctx_fail(nullptr, LSMS_ERR_ARG, "translate_mixed_noalloc: NULL pointer");
  const int P = 2 * p + 1;
  const long long len = (long long)nrhs * n * P;
  const size_t cbytes = (((size_t)n * sizeof(float4)) + 255) & ~size_t(255);
  const size_t b32 = (((size_t)len * sizeof(float2)) + 255) & ~size_t(255);
  const size_t per_split = (size_t)len * sizeof(float2);
  if (cbytes + b32 + per_split > kNoAllocScratchBytes)
    return ctx_fail(nullptr, LSMS_ERR_ARG,
                    "translate_mixed_noalloc: n * (16 + 16 * nrhs * (2p+1)) bytes exceed the 16 MiB scratch");
  int splits = translate_splits(n, nrhs, p);
  while (splits > 1 && cbytes + b32 + (size_t)splits * per_split > kNoAllocScratchBytes) --splits;
  int sps = (n + splits - 1) / splits;
  sps = ((sps + MCH - 1) / MCH) * MCH;
  splits = (n + sps - 1) / sps;
  void* base = nullptr;
  int rc = noalloc_scratch(&base);
  if (rc) return rc;
  float4* cff = (float4*)base;
  float2* xs32 = (float2*)((unsigned char*)base + cbytes);
  float2* part = (float2*)((unsigned char*)base + cbytes + b32);
  cudaStream_t st = (cudaStream_t)stream;
  k_centres_ff_xy<<<(n + 255) / 256, 256, 0, st>>>(centres_xy, n, cff);
  long long g = (len + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  k_to_float<<<(int)g, 256, 0, st>>>((const double2*)beta, xs32, len);
  const float kh = (float)k2, kl = (float)(k2 - (double)kh);
  const int tpc = translate_targets_per_cta(nrhs, p);
  dim3 grid((n + tpc - 1) / tpc, splits, nrhs);
  launch_translate_kernel(grid, st, cff, n, p, kh, kl, xs32, part, sps, nrhs);
  k_reduce_parts<<<(int)g, 256, 0, st>>>(part, splits, len, (double2*)alpha);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return ctx_fail(nullptr, LSMS_ERR_CUDA, std::string("translate_mixed_noalloc: ") + cudaGetErrorString(e));
  return LSMS_OK;
}
