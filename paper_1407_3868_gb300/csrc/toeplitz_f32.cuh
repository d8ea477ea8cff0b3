// FP32 contraction of one disc pair's Hankel sequence with the source's coefficients (Sec. 3.2
// Lemma 3.1: alpha_nu += sum_n H_{n-nu}(k rho) e^{i (n - nu) phi} beta_n), as the near-pair
// kernels run it: four lanes per target, lane block hb = 0..3 owning the VB consecutive outputs
// VB hb .. VB hb + VB - 1 (VB = ceil(P / 4)).  The Toeplitz matrix is read through a register window
// over the sequence that slides by VB per input block, and every complex product takes three
// real multiplications (Gauss): AB += (h.x b.x, h.y b.y) as one packed FMA, C += (h.x + h.y)(b.x + b.y);
// the output is (AB.x - AB.y, C - AB.x - AB.y).
#pragma once

#include <cuda_runtime.h>

namespace {

// Asynchronous 8-byte global -> shared copy (zero-filled when !valid: no bytes are read), and the
// wait for all of this thread's copies; a __syncwarp after the wait publishes them to the warp.
__device__ __forceinline__ void cp_async8(void* sdst, const void* gsrc, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
  const int nbytes = valid ? 8 : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(gsrc), "r"(nbytes) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// One warp stages up to 32 pair slots: slot s takes the table row erow_s (S entries, when
// table != nullptr and erow_s >= 0) into hw[s * hs_stride ..] and the source coefficients
// xr[m_s * P ..] (P entries, when m_s >= 0) into bw[s * P ..]; missing rows and sources are zero.
// erow and m are this lane's slot values (slot = lane); all 32 lanes call it.  The copies are
// only issued: cp_async_wait_all() and a __syncwarp() make them visible.
template <int S, int P>
__device__ __forceinline__ void stage_slots(float2* hw, int hs_stride, float2* bw, const float2* __restrict__ table,
                                            int erow, const float2* __restrict__ xr, int m, int lane) {
#pragma unroll 4
  for (int s = 0; s < 32; ++s) {
    const int es = __shfl_sync(0xffffffffu, erow, s);
    const int ms = __shfl_sync(0xffffffffu, m, s);
    if (table) {
#pragma unroll
      for (int c = lane; c < S; c += 32)
        cp_async8(hw + s * hs_stride + c, es >= 0 ? table + (size_t)es * S + c : table, es >= 0);
    }
    if (lane < P) cp_async8(bw + s * P + lane, ms >= 0 ? xr + (size_t)ms * P + lane : xr, ms >= 0);
  }
}

// LANES lanes per target (4 or 2); lane block hb owns the outputs VB hb .. VB hb + VB - 1.
template <int PT, int LANES> struct ToeL {
  static constexpr int P = 2 * PT + 1;
  static constexpr int VB = (P + LANES - 1) / LANES;   // outputs per lane
  static constexpr int NB = (P + VB - 1) / VB;         // input blocks
};
template <int PT> struct Toe4 : ToeL<PT, 4> {};

// hs: &h[2p - VB hb] of the pair sequence h[s + 2p], s = -2p..2p, so that hs[q - i] multiplies
// input q into output VB hb + i; reads hs[-(VB - 1)] .. hs[NB VB - 1] (the caller keeps that range
// in bounds; entries that only reach outputs >= P may hold anything finite or not).  bs: the P
// source coefficients.
template <int PT, int LANES>
__device__ __forceinline__ void toeplitz_contract(const float2* hs, const float2* bs,
                                                  float2 (&AB)[ToeL<PT, LANES>::VB],
                                                  float (&C)[ToeL<PT, LANES>::VB]) {
  constexpr int P = ToeL<PT, LANES>::P, VB = ToeL<PT, LANES>::VB, NB = ToeL<PT, LANES>::NB;
  float2 win[2 * VB - 1];
  float wsum[2 * VB - 1];
#pragma unroll
  for (int j = 0; j < VB - 1; ++j) {
    win[j] = hs[j - (VB - 1)];
    wsum[j] = win[j].x + win[j].y;
  }
#pragma unroll
  for (int nbk = 0; nbk < NB; ++nbk) {
#pragma unroll
    for (int j = 0; j < VB; ++j) {
      win[VB - 1 + j] = hs[nbk * VB + j];
      wsum[VB - 1 + j] = win[VB - 1 + j].x + win[VB - 1 + j].y;
    }
#pragma unroll
    for (int u = 0; u < VB; ++u) {
      if (nbk * VB + u >= P) break;
      const float2 bv = bs[nbk * VB + u];
      const float bsum = bv.x + bv.y;
#pragma unroll
      for (int i = 0; i < VB; ++i) {
        AB[i] = __ffma2_rn(win[VB - 1 + u - i], bv, AB[i]);
        C[i] = __fmaf_rn(wsum[VB - 1 + u - i], bsum, C[i]);
      }
    }
#pragma unroll
    for (int j = 0; j < VB - 1; ++j) {
      win[j] = win[VB + j];
      wsum[j] = wsum[VB + j];
    }
  }
}

template <int PT>
__device__ __forceinline__ void toeplitz_contract4(const float2* hs, const float2* bs,
                                                   float2 (&AB)[Toe4<PT>::VB], float (&C)[Toe4<PT>::VB]) {
  toeplitz_contract<PT, 4>(hs, bs, AB, C);
}

}  // namespace
