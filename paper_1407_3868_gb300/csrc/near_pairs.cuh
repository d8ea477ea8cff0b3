// The mixed-precision near field from pair lists (Sec. 3.2 Lemma 3.1 for the pairs that the main
// translation leaves out): for every target l, alpha^l_nu += sum over its listed sources m of
// sum_n h^{lm}_{n - nu} beta^m_n, with the pair sequences generated in FP32: H_0 and H_1 from a
// table of FP64-built values (pairs with k rho < 25, where Hankel's expansion does not hold) or
// from Hankel's expansion with the float-float phase reduction (k rho >= 25), the other orders by
// the forward recurrence.
//
// A warp serves 8 targets, 4 lanes per target for the contraction (lane block hb owns VB outputs).
// Per round it takes every target's next 2 pairs into 16 shared-memory slots: the two lanes of a
// slot run the same recurrence and store the positive and the negative orders, while the 16
// source coefficient vectors are copied in asynchronously; then each target's 4 lanes contract its
// 2 slots (toeplitz_contract4).  Small rounds keep a warp's shared memory at 12 KB, so that 16
// warps share an SM and hide each other's generation and copy latency.
#pragma once

#include <mutex>

#include "ff_hankel.cuh"
#include "toeplitz_f32.cuh"

namespace {

constexpr int PL_W = 4;         // warps per CTA
constexpr int PL_SLOTS = 16;    // pair slots per warp and round: 8 targets x 2 pairs
constexpr int PL_HS = 65;       // sequence slot stride (odd: the 8 targets' windows in distinct banks)
constexpr int PL_GUARD = 8;     // zeros before the first slot and after the last (window overhang)

template <int PT> __host__ __device__ constexpr size_t pl_warp_words() {
  return (size_t)2 * PL_GUARD + PL_SLOTS * PL_HS + PL_SLOTS * (2 * PT + 1);
}

// Half of the sequence h[s + 2p] = H_s e^{i s phi} from H_0, H_1 (see hankel_recurrence_f32):
// side 0 stores s = 0..2p, side 1 stores s = -2p..-1.
template <int PT>
__device__ __forceinline__ void hankel_recurrence_half_f32(float2 h0, float2 h1, float2 e1, float zf, int side,
                                                           float2* h) {
  constexpr int p = PT;
  const int c0 = 2 * p;
  if (side == 0) h[c0] = h0;
  float2 hm = h0, hq = h1, eq = e1;
  const float iz = 1.0f / zf;
#pragma unroll
  for (int q = 1; q <= 2 * p; ++q) {
    if (side == 0) {
      h[c0 + q] = cmulf(hq, eq);
    } else {
      const float2 u = cmulf(hq, make_float2(eq.x, -eq.y));
      h[c0 - q] = (q & 1) ? make_float2(-u.x, -u.y) : u;
    }
    if (q < 2 * p) {
      const float f = 2.0f * q * iz;
      const float2 hn = make_float2(f * hq.x - hm.x, f * hq.y - hm.y);
      hm = hq;
      hq = hn;
      eq = cmulf(eq, e1);
    }
  }
}

// Targets t = 0 .. nt-1: disc l = perm[t] (perm != nullptr) or row0 + t; its pairs are the list
// entries k = cptr[key] .. cptr[key + 1] - 1, key = t (perm) or l, with source csrc[k] and table
// row crow[k] (-1: Hankel's expansion; crow == nullptr: row k).  Adds the sum into
// alpha[r][l - row0][.] (rows of nrows_out), r = blockIdx.y.  cff: float-float centres by disc.
template <int PT>
__global__ void __launch_bounds__(PL_W * 32)
k_pair_lists_f32(const int* __restrict__ perm, int row0, int nt, int nrows_out, const float4* __restrict__ cff,
                 const int* __restrict__ cptr, const int* __restrict__ csrc, const int* __restrict__ crow,
                 const float4* __restrict__ table, int n, float k_hi, float k_lo, const float2* __restrict__ xs,
                 double2* __restrict__ alpha) {
  constexpr int p = PT, P = 2 * PT + 1;
  constexpr int VB = Toe4<PT>::VB;
  extern __shared__ float2 pl_sh[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tt = lane & 7, hb = lane >> 3;        // contraction: target tt, outputs VB hb ..
  const int gs = lane >> 1, side = lane & 1;      // generation: slot gs (pair gs >> 3 of target gs & 7)
  float2* hw = pl_sh + (size_t)warp * pl_warp_words<PT>() + PL_GUARD;   // [PL_SLOTS][PL_HS]
  float2* bw = hw + PL_SLOTS * PL_HS + PL_GUARD;                          // [PL_SLOTS][P]
  const int r = blockIdx.y;
  const int tbase = (blockIdx.x * PL_W + warp) * 8;
  const int t = tbase + tt;
  const bool tvalid = t < nt;
  const int l = !tvalid ? 0 : (perm ? perm[t] : row0 + t);
  const int tg = tbase + (gs & 7);
  const bool gvalid = tg < nt;
  const int lg = !gvalid ? 0 : (perm ? perm[tg] : row0 + tg);
  const int keyg = perm ? tg : lg;
  const float4 cg = gvalid ? cff[lg] : make_float4(0.f, 0.f, 0.f, 0.f);
  const int g0 = gvalid ? cptr[keyg] : 0, g1 = gvalid ? cptr[keyg + 1] : 0;
  const int maxlen = __reduce_max_sync(0xffffffffu, g1 - g0);
  for (int i = lane; i < (int)pl_warp_words<PT>(); i += 32) hw[i - PL_GUARD] = make_float2(0.f, 0.f);
  const float2* xr = xs + (size_t)r * n * P;
  const ffl kf = {k_hi, k_lo};
  float2 AB[VB];
  float C[VB];
#pragma unroll
  for (int i = 0; i < VB; ++i) {
    AB[i] = make_float2(0.f, 0.f);
    C[i] = 0.f;
  }
  for (int r0 = 0; r0 < maxlen; r0 += 2) {
    const int k = g0 + r0 + (gs >> 3);
    const bool have = k < g1;
    const int m = have ? csrc[k] : -1;
    const int e = !have ? -1 : (crow ? crow[k] : k);
    __syncwarp();
#pragma unroll 4
    for (int s = 0; s < PL_SLOTS; ++s) {           // source coefficients of slot s (lanes 2s, 2s + 1)
      const int ms = __shfl_sync(0xffffffffu, m, 2 * s);
      if (lane < P) cp_async8(bw + s * P + lane, ms >= 0 ? xr + (size_t)ms * P + lane : xr, ms >= 0);
    }
    float2* h = hw + gs * PL_HS;
    if (m >= 0) {
      const PairGeom g = pair_geometry(cg, cff[m], kf);
      float2 h0, h1;
      if (e >= 0) {
        const float4 v = table[e];
        h0 = make_float2(v.x, v.y);
        h1 = make_float2(v.z, v.w);
      } else {
        hankel01_f32(g, h0, h1);
      }
      hankel_recurrence_half_f32<PT>(h0, h1, g.e1, g.zf, side, h);
    } else if (side == 0) {
      for (int q = 2 * p; q <= 4 * p; ++q) h[q] = make_float2(0.f, 0.f);
    } else {
      for (int q = 0; q < 2 * p; ++q) h[q] = make_float2(0.f, 0.f);
    }
    cp_async_wait_all();
    __syncwarp();
    const int nq2 = min(2, maxlen - r0);
    for (int q2 = 0; q2 < nq2; ++q2) {
      const int slot = q2 * 8 + tt;
      toeplitz_contract4<PT>(hw + slot * PL_HS + 2 * p - VB * hb, bw + slot * P, AB, C);
    }
  }
  if (tvalid && maxlen > 0) {
    double2* o = alpha + ((size_t)r * nrows_out + (l - row0)) * P;
#pragma unroll
    for (int i = 0; i < VB; ++i) {
      const int nu = VB * hb + i;
      if (nu < P) {
        o[nu].x += (double)(AB[i].x - AB[i].y);
        o[nu].y += (double)(C[i] - AB[i].x - AB[i].y);
      }
    }
  }
}

template <int PT>
void launch_pair_lists_pt(dim3 grid, cudaStream_t st, const int* perm, int row0, int nt, int nrows_out,
                          const float4* cff, const int* cptr, const int* csrc, const int* crow,
                          const float4* table, int n, float kh, float kl, const float2* xs, double2* alpha) {
  constexpr size_t smem = PL_W * pl_warp_words<PT>() * sizeof(float2);
  static std::once_flag attr;
  std::call_once(attr, [] {
    cudaFuncSetAttribute(k_pair_lists_f32<PT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  k_pair_lists_f32<PT><<<grid, PL_W * 32, smem, st>>>(perm, row0, nt, nrows_out, cff, cptr, csrc, crow, table, n,
                                                      kh, kl, xs, alpha);
}

// Host entry: nt targets (see k_pair_lists_f32), nrhs right-hand sides, order p (0..15).
inline void launch_pair_lists(int p, int nrhs, cudaStream_t st, const int* perm, int row0, int nt, int nrows_out,
                              const float4* cff, const int* cptr, const int* csrc, const int* crow,
                              const float4* table, int n, double k, const float2* xs, double2* alpha) {
  if (nt <= 0 || nrhs <= 0) return;
  const float kh = (float)k, kl = (float)(k - (double)kh);
  dim3 grid((unsigned)((nt + PL_W * 8 - 1) / (PL_W * 8)), (unsigned)nrhs);
#define LSMS_PL(PT) \
  launch_pair_lists_pt<PT>(grid, st, perm, row0, nt, nrows_out, cff, cptr, csrc, crow, table, n, kh, kl, xs, alpha)
  switch (p) {
    case 0: LSMS_PL(0); break;
    case 1: LSMS_PL(1); break;
    case 2: LSMS_PL(2); break;
    case 3: LSMS_PL(3); break;
    case 4: LSMS_PL(4); break;
    case 5: LSMS_PL(5); break;
    case 6: LSMS_PL(6); break;
    case 7: LSMS_PL(7); break;
    case 8: LSMS_PL(8); break;
    case 9: LSMS_PL(9); break;
    case 10: LSMS_PL(10); break;
    case 11: LSMS_PL(11); break;
    case 12: LSMS_PL(12); break;
    case 13: LSMS_PL(13); break;
    case 14: LSMS_PL(14); break;
    default: LSMS_PL(15); break;
  }
#undef LSMS_PL
}

}  // namespace

namespace {

// ---------------------------------------------------------------------------------------------
// The same near field from stored sequences (the box translation's pair lists, whose geometry is
// fixed for a layout): every list entry k has its sequence h[s + 2p], s = -2p..2p, built once in
// FP64 and stored in FP32 as row k of `seq` (4p + 2 float2 per row).  A warp serves 32 / LANES
// targets, LANES lanes per target (each VB = ceil(P / LANES) consecutive outputs); rounds of one
// pair per target are double-buffered: the next round's rows and source coefficients are in
// flight (cp.async groups) while the current round is contracted.  The rows' shared-memory stride
// is odd in 8-byte words per target slot for 16 targets (two lanes), 2 mod 4 for 8 targets (four
// lanes, 16-byte copies), so that a warp's window loads fall in distinct banks.
// ---------------------------------------------------------------------------------------------
constexpr int PS_W = 4;          // warps per CTA
constexpr int PS_GUARD = 8;

template <int PT, int LANES> struct PsShape {
  static constexpr int P = 2 * PT + 1;
  static constexpr int TPW = 32 / LANES;                    // targets per warp = slots per round
  static constexpr int GRS = 4 * PT + 2;                    // float2 per stored row
  static constexpr int SRS = LANES == 4 ? 4 * PT + 2 : 4 * PT + 3;   // shared-memory row stride
  static constexpr int BUF = TPW * (SRS + P);               // one round: the rows and coefficient vectors
  static constexpr int WORDS = 2 * PS_GUARD + 2 * BUF;      // per warp, float2
  static constexpr size_t SMEM = (size_t)PS_W * WORDS * sizeof(float2);
};

__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_one() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// Targets t = 0 .. n-1 in box order (disc perm[t]); list entries k = cptr[t] .. cptr[t + 1] - 1 with
// source csrc[k] and stored row k.  Adds the sum into alpha[r][perm[t]][.], r = blockIdx.y.
template <int PT, int LANES>
__global__ void __launch_bounds__(PS_W * 32)
k_pair_seq_f32(const int* __restrict__ perm, const int* __restrict__ cptr, const int* __restrict__ csrc,
               const float2* __restrict__ seq, int n, const float2* __restrict__ xs, double2* __restrict__ alpha) {
  using S = PsShape<PT, LANES>;
  constexpr int p = PT, P = S::P, TPW = S::TPW, GRS = S::GRS, SRS = S::SRS, BUF = S::BUF;
  constexpr int VB = ToeL<PT, LANES>::VB;
  extern __shared__ __align__(16) float2 ps_sh[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tt = lane & (TPW - 1), hb = lane / TPW;
  float2* base = ps_sh + (size_t)warp * S::WORDS + PS_GUARD;   // two round buffers
  const int r = blockIdx.y;
  const int t = (blockIdx.x * PS_W + warp) * TPW + tt;
  const bool tvalid = t < n;
  const int c0 = tvalid ? cptr[t] : 0, c1 = tvalid ? cptr[t + 1] : 0;
  const int maxlen = __reduce_max_sync(0xffffffffu, c1 - c0);
  for (int i = lane; i < S::WORDS; i += 32) base[i - PS_GUARD] = make_float2(0.f, 0.f);
  __syncwarp();
  const float2* xr = xs + (size_t)r * n * P;
  // slot s of a round = target s; lane (s mod TPW) knows that target's list range
  auto issue = [&](int r0, float2* buf) {
    const int k = c0 + r0;
    const int kk = k < c1 ? k : -1;
    const int m = kk >= 0 ? csrc[kk] : -1;
    float2* hw = buf;
    float2* bw = buf + TPW * SRS;
#pragma unroll 4
    for (int s = 0; s < TPW; ++s) {
      const int ks = __shfl_sync(0xffffffffu, kk, s);
      const int ms = __shfl_sync(0xffffffffu, m, s);
      if (ks >= 0) {
        const float2* row = seq + (size_t)ks * GRS;
        if (LANES == 4) {
          if (lane < GRS / 2) cp_async16(hw + s * SRS + 2 * lane, row + 2 * lane);
        } else {
          for (int c = lane; c < GRS; c += 32) cp_async8(hw + s * SRS + c, row + c, true);
        }
        if (lane < P) cp_async8(bw + s * P + lane, xr + (size_t)ms * P + lane, true);
      } else {
        for (int c = lane; c < SRS; c += 32) hw[s * SRS + c] = make_float2(0.f, 0.f);
        if (lane < P) bw[s * P + lane] = make_float2(0.f, 0.f);
      }
    }
    cp_async_commit();
  };
  float2 AB[VB];
  float C[VB];
#pragma unroll
  for (int i = 0; i < VB; ++i) {
    AB[i] = make_float2(0.f, 0.f);
    C[i] = 0.f;
  }
  if (maxlen > 0) issue(0, base);
  for (int r0 = 0, cur = 0; r0 < maxlen; ++r0, cur ^= 1) {
    float2* buf = base + cur * BUF;
    if (r0 + 1 < maxlen) issue(r0 + 1, base + (cur ^ 1) * BUF);
    else cp_async_commit();                       // an empty group keeps the wait count uniform
    cp_async_wait_one();                          // this round's copies have landed
    __syncwarp();
    toeplitz_contract<PT, LANES>(buf + tt * SRS + 2 * p - VB * hb, buf + TPW * SRS + tt * P, AB, C);
    __syncwarp();                                 // the buffer is refilled two rounds later
  }
  if (tvalid && maxlen > 0) {
    double2* o = alpha + ((size_t)r * n + perm[t]) * P;
#pragma unroll
    for (int i = 0; i < VB; ++i) {
      const int nu = VB * hb + i;
      if (nu < P) {
        o[nu].x += (double)(AB[i].x - AB[i].y);
        o[nu].y += (double)(C[i] - AB[i].x - AB[i].y);
      }
    }
  }
}

constexpr int PS_LANES = 4;      // lanes per target of the stored-sequence near field (2: 1.5x slower)

template <int PT>
void launch_pair_seq_pt(dim3 grid, cudaStream_t st, const int* perm, const int* cptr, const int* csrc,
                        const float2* seq, int n, const float2* xs, double2* alpha) {
  using S = PsShape<PT, PS_LANES>;
  static std::once_flag attr;
  std::call_once(attr, [] {
    cudaFuncSetAttribute(k_pair_seq_f32<PT, PS_LANES>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
  });
  k_pair_seq_f32<PT, PS_LANES><<<grid, PS_W * 32, S::SMEM, st>>>(perm, cptr, csrc, seq, n, xs, alpha);
}

// Host entry (order p 0..15): n targets in box order, nrhs right-hand sides.
inline void launch_pair_seq(int p, int nrhs, cudaStream_t st, const int* perm, const int* cptr, const int* csrc,
                            const float2* seq, int n, const float2* xs, double2* alpha) {
  if (n <= 0 || nrhs <= 0) return;
  const int tpc = PS_W * (32 / PS_LANES);
  dim3 grid((unsigned)((n + tpc - 1) / tpc), (unsigned)nrhs);
#define LSMS_PS(PT) launch_pair_seq_pt<PT>(grid, st, perm, cptr, csrc, seq, n, xs, alpha)
  switch (p) {
    case 0: LSMS_PS(0); break;
    case 1: LSMS_PS(1); break;
    case 2: LSMS_PS(2); break;
    case 3: LSMS_PS(3); break;
    case 4: LSMS_PS(4); break;
    case 5: LSMS_PS(5); break;
    case 6: LSMS_PS(6); break;
    case 7: LSMS_PS(7); break;
    case 8: LSMS_PS(8); break;
    case 9: LSMS_PS(9); break;
    case 10: LSMS_PS(10); break;
    case 11: LSMS_PS(11); break;
    case 12: LSMS_PS(12); break;
    case 13: LSMS_PS(13); break;
    case 14: LSMS_PS(14); break;
    default: LSMS_PS(15); break;
  }
#undef LSMS_PS
}

}  // namespace
