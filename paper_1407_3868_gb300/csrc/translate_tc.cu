// Graf translation of a block of right-hand sides on the tensor cores (tcgen05; Sec. 3.2
// Lemma 3.1, Eq. "trans"), the mixed-precision form used when many sources are solved together.
//
// With R right-hand sides, alpha^l(r) = sum_{m != l} T^{lm} beta^m(r) is for every disc pair a
// complex (P x P) . (P x R) product with the Toeplitz block T^{lm}_{nu n} = h_{n - nu},
// h_s = H_s(k2 rho) exp(i s phi) (rho, phi: distance and angle of x_l - x_m).  It runs as real BF16
// MMAs (M = 128, N = 128, K = 16) with FP32 accumulation in tensor memory:
//
//   D (128 rows: TT targets x P orders, 128 columns: Re and Im outputs of 64 right-hand sides)
//     += A (128 x K) . B (128 x K)^T,   K = 2P padded to 64,
//
// with the K elements in pairs by source order n: A row (target i, order nu) has Re h_{n - nu} at
// K = 2n and Im h_{n - nu} at 2n + 1; B row (Re, r) has Re beta_n(r), -Im beta_n(r) there, B row
// (Im, r) Im beta_n(r), Re beta_n(r), so D(Re, r) = sum Re T Re beta - Im T Im beta and D(Im, r) =
// sum Re T Im beta + Im T Re beta.  An A row is then a contiguous run of the pair sequence's packed
// (Re, Im) words.  A tile holds
// TT = floor(128 / P) targets (5 at p = 12: 125 of 128 rows used), and each MMA instruction computes
// 64 right-hand sides' real and imaginary parts (N = 128: the instruction's fixed cost is shared by
// twice the columns of an N = 64 embedding with the complex structure in the rows).  Both operands
// are split into three BF16 planes x = hi + mid + lo and the six plane products with terms down to
// 2^-16 relative are accumulated.  The Hankel sequences are the FP32 ones of the CUDA-core path;
// near pairs (k2 rho < 25) and the self pair are left to the near-pair kernel.
//
// A persistent CTA (one per SM) owns a contiguous range of steps (right-hand-side block, group of
// TG = 2 TT target discs, source disc).  Per step: warp 0 lane 0 copies the source's B planes (48 KB,
// prepared once per application in the 128-byte-swizzled shared-memory image) with a bulk copy into
// a 3-stage ring; warps 6-7 generate the FP32 pair sequences of the next chunk of CHS sources
// (CHS TG <= 40 pairs, one per thread; fewer where the buffers would not fit), already split into three BF16 planes of packed (Re, Im)
// words, into the other of two chunk buffers, one chunk ahead of their use; warps 2-5 build the two
// A tiles of the step from the current chunk's planes (each thread one row: P words per plane,
// copied) and write them straight into tensor memory (tcgen05.st, 2-stage ring); warp 1 lane 0
// issues 24 tcgen05.mma per tile with A from tensor memory and B from shared memory into 2
// accumulators (256 columns).  Every `flush`
// source discs, warps 2-5 read the accumulators (tcgen05.ld) and add them into the FP64 output
// with atomics: the tensor cores sum in FP32 with less than round-to-nearest accuracy, so the error
// grows with the number of MMAs summed in one accumulator.  Every mbarrier wait is bounded; on a
// timeout the CTA records an error, waits for its copies in flight, frees its tensor memory and
// returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "lsms_internal.h"
#include "lsms_ops.h"
#include "ff_hankel.cuh"
#include "tc_ptx.cuh"

namespace {

constexpr int NTILE = 2;                // accumulator tiles per group
constexpr int RBLK = 64;                // right-hand sides per block
constexpr int NCOL = 2 * RBLK;          // MMA N: Re and Im columns
constexpr int B_PLANE = NCOL * 128;     // bytes: 128 rows x 64 BF16
constexpr int B_STAGE = 3 * B_PLANE;    // 49152
constexpr int NA = 2, NBS = 3;          // ring depths (A in tensor memory, B in shared memory)
constexpr int NTHR = 256;               // warp 0: copies, warp 1: MMA, warps 2-5: operands and epilogue,
                                        // warps 6-7: pair sequences of the next chunk
constexpr int NGEN = 64;                // generator threads
constexpr int MAXPAIRS = 40;            // pairs per sequence chunk at most (CHS sources x TG targets)
constexpr int BAR_BYTES = 256;
constexpr int SMEM_LIMIT = 227 * 1024;
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t ACC_COLS = NTILE * NCOL;                       // 256
constexpr uint32_t A_COLS = 3 * 32;                               // one A tile: 3 planes x 32 columns
constexpr uint32_t IDESC_T = idesc_bf16(128, NCOL);
// plane products (A plane, B plane): hi.hi, hi.mid, mid.hi, hi.lo, lo.hi, mid.mid
__host__ __device__ constexpr int plane_a(int q) { return q == 2 || q == 5 ? 1 : (q == 4 ? 2 : 0); }
__host__ __device__ constexpr int plane_b(int q) { return q == 1 || q == 5 ? 1 : (q == 3 ? 2 : 0); }

// Words per plane of a pair sequence in the chunk buffers: the smallest R >= 4p + 1 with
// 3 R + 2p + 1 = 0 mod 32.  An operand thread (row r = P i + nu of a tile) reads word w0 + n =
// 2p - nu + n of pair i, at (pair base) + 3 R i + 2p - nu + n = const + i (3 R + P) - r + n, so with
// 3 R + P = 0 mod 32 the 32 rows of a warp read 32 consecutive banks.
__host__ __device__ constexpr int tc_rws(int p) {
  int r = 4 * p + 1;
  while ((3 * r + 2 * p + 1) % 32 != 0) ++r;
  return r;
}

// Targets per tile and group, sources per sequence chunk and the chunk buffers, for order p.
template <int PT>
struct TcShape {
  static constexpr int P = 2 * PT + 1;
  static constexpr int TT = 128 / P;
  static constexpr int TG = NTILE * TT;
  static constexpr int RWS = tc_rws(PT);
  static constexpr int FIT = (SMEM_LIMIT - 1024 - NBS * B_STAGE - BAR_BYTES) / (2 * 3 * RWS * 4);
  static constexpr int PAIRS = MAXPAIRS < FIT ? MAXPAIRS : FIT;
  static constexpr int CHS = PAIRS / TG > 0 ? PAIRS / TG : 1;
  static constexpr int NPAIR = CHS * TG;                                    // pairs per chunk buffer
  static constexpr int RAW_BYTES = 2 * NPAIR * 3 * RWS * 4;                 // two chunk buffers
  static constexpr size_t SMEM = 1024 + (size_t)NBS * B_STAGE + RAW_BYTES + BAR_BYTES;
};

// B image of one (right-hand-side block, source disc): 3 planes x 128 rows x 128 bytes (K element
// 2n and 2n + 1 for order n, see the file comment; zero from 2P); row j < 64 is output Re of
// right-hand side j, row 64 + j its Im; chunk c of row r at c ^ (r mod 8).
__global__ void k_pack_b_tc(const double2* __restrict__ xs, int n, int P, int nrhs, int nrb,
                            unsigned char* __restrict__ img) {
  const long long total = (long long)nrb * n * NCOL * 8;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
       id += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(id & 7), row = (int)((id >> 3) & (NCOL - 1));
    const long long sm = id >> 10;                      // rb * n + m
    const int m = (int)(sm % n), rb = (int)(sm / n);
    const bool im_row = row >= RBLK;
    const int rr = rb * RBLK + (row & (RBLK - 1));
    uint32_t w[3][4];
#pragma unroll
    for (int e = 0; e < 8; e += 2) {
      __nv_bfloat16 h[2], md[2], lo[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int kk = 8 * c + e + u, nn = kk >> 1;
        double x = 0.0;
        if (rr < nrhs && nn < P) {
          const double2 b = xs[((size_t)rr * n + m) * P + nn];
          x = (kk & 1) ? (im_row ? b.x : -b.y) : (im_row ? b.y : b.x);
        }
        split3(x, h[u], md[u], lo[u]);
      }
      w[0][e / 2] = (uint32_t)__bfloat16_as_ushort(h[0]) | ((uint32_t)__bfloat16_as_ushort(h[1]) << 16);
      w[1][e / 2] = (uint32_t)__bfloat16_as_ushort(md[0]) | ((uint32_t)__bfloat16_as_ushort(md[1]) << 16);
      w[2][e / 2] = (uint32_t)__bfloat16_as_ushort(lo[0]) | ((uint32_t)__bfloat16_as_ushort(lo[1]) << 16);
    }
    unsigned char* base = img + (size_t)sm * B_STAGE + row * 128 + ((c ^ (row & 7)) * 16);
#pragma unroll
    for (int pl = 0; pl < 3; ++pl)
      *(uint4*)(base + pl * B_PLANE) = make_uint4(w[pl][0], w[pl][1], w[pl][2], w[pl][3]);
  }
}

// Pair sequence h[s + 2p] = H_s(k rho) e^{i s phi}, s = -2p..2p, as the generators store it: for
// every element s, plane pl of words [pl][s] holds (BF16 plane pl of Re h | that of Im h << 16),
// Re h = hi + mid + lo in BF16.  Near pairs (r2 below near_r2) are zero, as in hankel_sequence_f32.
template <int RWS>
__device__ __forceinline__ void put_planes(uint32_t* w, int s, float2 v) {
  unsigned short ur[3], ui[3];
  split3f(v.x, ur);
  split3f(v.y, ui);
#pragma unroll
  for (int pl = 0; pl < 3; ++pl) w[pl * RWS + s] = (uint32_t)ur[pl] | ((uint32_t)ui[pl] << 16);
}

template <int PT>
__device__ __forceinline__ void hankel_planes(float4 a, float4 b, ffl k, ffl near_r2, uint32_t* w) {
  constexpr int p = PT;
  constexpr int RWS = TcShape<PT>::RWS;
  const PairGeom g = pair_geometry(a, b, k);
  if (near_r2.hi > 0.0f && (g.r2.hi < near_r2.hi || (g.r2.hi == near_r2.hi && g.r2.lo < near_r2.lo))) {
    for (int q = 0; q < 3 * RWS; ++q) w[q] = 0u;
    return;
  }
  float2 h0, h1;
  hankel01_f32(g, h0, h1);
  const int c0 = 2 * p;
  put_planes<RWS>(w, c0, h0);
  float2 hm = h0, hq = h1, eq = g.e1;
  const float iz = 1.0f / g.zf;
#pragma unroll
  for (int q = 1; q <= 2 * p; ++q) {
    put_planes<RWS>(w, c0 + q, cmulf(hq, eq));
    const float2 u = cmulf(hq, make_float2(eq.x, -eq.y));
    put_planes<RWS>(w, c0 - q, (q & 1) ? make_float2(-u.x, -u.y) : u);
    if (q < 2 * p) {
      const float f = 2.0f * q * iz;
      const float2 hn = make_float2(f * hq.x - hm.x, f * hq.y - hm.y);
      hm = hq;
      hq = hn;
      eq = cmulf(eq, g.e1);
    }
  }
}

template <int PT>
__global__ void __launch_bounds__(NTHR, 1)
k_translate_tc(const float4* __restrict__ cff, int n, float k_hi, float k_lo, float near_hi,
               float near_lo, const unsigned char* __restrict__ bimg, int nrhs, long long nsteps,
               int flush, double2* __restrict__ alpha, int* __restrict__ err) {
  constexpr int p = PT, P = 2 * PT + 1;
  constexpr int TT = TcShape<PT>::TT, TG = TcShape<PT>::TG, CHS = TcShape<PT>::CHS;
  constexpr int RWS = TcShape<PT>::RWS, NPAIR = TcShape<PT>::NPAIR;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sB = smem;
  uint32_t* raw = (uint32_t*)(sB + NBS * B_STAGE);          // [2][NPAIR][3][RWS] BF16-plane words
  uint64_t* bars = (uint64_t*)((unsigned char*)raw + TcShape<PT>::RAW_BYTES);
  uint32_t* tmem_slot = (uint32_t*)(bars + 2 * NA + 2 * NBS + 3 + 4);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  volatile int* bcast = abort_flag + 1;
  volatile int* gbcast = abort_flag + 2;
  const uint32_t a_full = smem_u32(bars), a_empty = a_full + 8 * NA;
  const uint32_t b_full = a_empty + 8 * NA, b_empty = b_full + 8 * NBS;
  const uint32_t acc_full = b_empty + 8 * NBS, acc_empty = acc_full + 8, done = acc_empty + 8;
  const uint32_t raw_full = done + 8, raw_empty = raw_full + 16;   // two chunk buffers each
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ngroups = (n + TG - 1) / TG;
  // accumulation segment of a step: (right-hand-side block, group, block of `flush` sources); the
  // accumulators are drained into the FP64 output at every segment end, which bounds the number of
  // MMAs summed in FP32 in one accumulator
  const int nseg = (n + flush - 1) / flush;
  auto segkey = [&](long long s) { return (s / n) * nseg + (s % n) / flush; };
  const long long s0 = nsteps * blockIdx.x / gridDim.x;
  const long long s1 = nsteps * (blockIdx.x + 1) / gridDim.x;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NA; ++s) {
      mbar_init(a_full + 8 * s, 1);
      mbar_init(a_empty + 8 * s, 1);
    }
    for (int s = 0; s < NBS; ++s) {
      mbar_init(b_full + 8 * s, 1);
      mbar_init(b_empty + 8 * s, 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, 1);
    mbar_init(done, 1);
    for (int s = 0; s < 2; ++s) {
      mbar_init(raw_full + 8 * s, 1);
      mbar_init(raw_empty + 8 * s, 1);
    }
    *abort_flag = 0;
    *bcast = 0;
    *gbcast = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(smem_u32(tmem_slot), TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---- producer: one bulk copy of the B planes per step ----
    long long i = 0;
    for (long long s = s0; s < s1; ++s, ++i) {
      if (*abort_flag) break;
      const int bs = (int)(i % NBS);
      const long long round = i / NBS;
      if (round > 0 && !mbar_wait(b_empty + 8 * bs, (uint32_t)((round - 1) & 1))) {
        *abort_flag = 1;
        atomicExch(err, 11);
        break;
      }
      const long long key = s / n;                      // rb * ngroups + g
      const int m = (int)(s - key * n);
      const long long rb = key / ngroups;
      mbar_expect_tx(b_full + 8 * bs, B_STAGE);
      bulk_load(smem_u32(sB + bs * B_STAGE), bimg + ((size_t)rb * n + m) * B_STAGE, B_STAGE, b_full + 8 * bs);
    }
    // copies in flight: the last round of every stage must have landed before the CTA exits
    for (int bs = 0; bs < NBS; ++bs)
      if (i > bs) mbar_wait(b_full + 8 * bs, (uint32_t)(((i - 1 - bs) / NBS) & 1));
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer: A from tensor memory, B from shared memory ----
    long long i = 0, t = 0, key_prev = -1;
    int grp = 0;
    bool first = true, ok = true;
    for (long long s = s0; s < s1; ++s, ++i) {
      const long long key = segkey(s);
      if (key != key_prev) {
        if (key_prev >= 0) {
          mma_commit(acc_full);
          if (!mbar_wait(acc_empty, (uint32_t)(grp & 1))) {
            ok = false;
            break;
          }
          ++grp;
        }
        key_prev = key;
        first = true;
      }
      if (*abort_flag) {
        ok = false;
        break;
      }
      const int bs = (int)(i % NBS);
      if (!mbar_wait(b_full + 8 * bs, (uint32_t)((i / NBS) & 1))) {
        ok = false;
        break;
      }
      const uint32_t b0 = smem_u32(sB + bs * B_STAGE);
      for (int tt = 0; tt < NTILE; ++tt, ++t) {
        const int as = (int)(t % NA);
        if (!mbar_wait(a_full + 8 * as, (uint32_t)((t / NA) & 1))) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t a0 = tmem + ACC_COLS + as * A_COLS;
#pragma unroll
        for (int q = 0; q < 6; ++q)
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
            mma_bf16_ta(tmem + tt * NCOL, a0 + plane_a(q) * 32 + kk * 8,
                        sw128_desc(b0 + plane_b(q) * B_PLANE + kk * 32), IDESC_T, (!first || q || kk) ? 1u : 0u);
        mma_commit(a_empty + 8 * as);
      }
      if (!ok) break;
      mma_commit(b_empty + 8 * bs);
      first = false;
    }
    if (ok && key_prev >= 0) mma_commit(acc_full);
    if (!ok) {
      *abort_flag = 1;
      atomicExch(err, 12);
    }
    // every MMA issued by this thread has finished before the tensor memory is freed
    mma_commit(done);
    mbar_wait(done, 0);
  } else if (warp >= 2 && warp < 6) {
    // ---- operands and epilogue: 128 threads, named barrier 1.  Thread (warp, lane) owns row
    // 32 (warp mod 4) + lane of every A tile and accumulator (its tensor-memory lane quarter):
    // row = P i + nu for target i < TT of the tile and order nu; rows from TT P on are zero.  The
    // rows are built from the FP32 sequences the generator warps left in the chunk's buffer: the
    // 2P entries [Re h_{n - nu} | Im h_{n - nu}] split into three BF16 planes on the fly.
    const int b = threadIdx.x - 64;
    const int q4 = warp & 3;
    const int row = 32 * q4 + lane;
    const int ti = row / P;                       // target within the tile
    const int nu = row - ti * P;
    const bool valid = ti < TT;
    const int w0 = 2 * p - nu;                    // window start: h_{n - nu} = h[w0 + n]
    const uint32_t lane_addr = (uint32_t)(32 * q4) << 16;
    long long t = 0, s = s0, chunk = 0;
    int grp = 0;
    while (s < s1) {
      const long long key = segkey(s), gkey = s / n;      // gkey = rb * ngroups + g
      const int g = (int)(gkey % ngroups);
      const int m0 = (int)(s - gkey * n);
      const int cnt = (int)min((long long)min(CHS, flush - m0 % flush), min(s1 - s, (long long)(n - m0)));
      const int cb = (int)(chunk & 1);
      if (b == 0) {                               // the chunk's sequences are in buffer cb
        bool w = !*abort_flag && mbar_wait(raw_full + 8 * cb, (uint32_t)((chunk >> 1) & 1));
        if (!w && !*abort_flag) {
          *abort_flag = 1;
          atomicExch(err, 15);
        }
        *bcast = w ? 1 : 0;
      }
      named_bar_sync(1, 128);
      if (!*bcast) break;
      bool ok = true;
      for (int j = 0; j < cnt && ok; ++j) {
        for (int tt = 0; tt < NTILE; ++tt, ++t) {
          const int as = (int)(t % NA);
          if (b == 0) {
            bool w = !*abort_flag;
            if (w && t >= NA) w = mbar_wait(a_empty + 8 * as, (uint32_t)((t / NA - 1) & 1));
            if (!w && !*abort_flag) {
              *abort_flag = 1;
              atomicExch(err, 13);
            }
            *bcast = w ? 1 : 0;
          }
          named_bar_sync(1, 128);
          if (!*bcast) {
            ok = false;
            break;
          }
          tc_fence_after();
          // K element 2n: Re h[w0 + n], 2n + 1: Im h[w0 + n]: word n of plane pl is the generators'
          // packed word (Re, Im) of sequence element w0 + n
          uint32_t v[3][32];
          const uint32_t* hr = raw + ((size_t)cb * NPAIR + j * TG + tt * TT + (valid ? ti : 0)) * 3 * RWS + w0;
#pragma unroll
          for (int pl = 0; pl < 3; ++pl)
#pragma unroll
            for (int jw = 0; jw < 32; ++jw) v[pl][jw] = (valid && jw < P) ? hr[pl * RWS + jw] : 0u;
          const uint32_t taddr = tmem + lane_addr + ACC_COLS + as * A_COLS;
#pragma unroll
          for (int pl = 0; pl < 3; ++pl) tmem_st32(taddr + pl * 32, v[pl]);
          tmem_wait_st();
          tc_fence_before();
          named_bar_sync(1, 128);
          if (b == 0) mbar_arrive(a_full + 8 * as);
        }
      }
      if (!ok) break;
      if (b == 0) mbar_arrive(raw_empty + 8 * cb);   // every row of the chunk has been read
      ++chunk;
      s += cnt;
      if (s == s1 || segkey(s) != key) {
        // segment done: read the accumulators and add them into alpha
        if (b == 0) {
          bool w = !*abort_flag && mbar_wait(acc_full, (uint32_t)(grp & 1));
          if (!w && !*abort_flag) {
            *abort_flag = 1;
            atomicExch(err, 14);
          }
          *bcast = w ? 1 : 0;
        }
        named_bar_sync(1, 128);
        if (!*bcast) break;
        tc_fence_after();
        const int rb = (int)(gkey / ngroups);
#pragma unroll 1
        for (int tt = 0; tt < NTILE; ++tt) {
          const int l = g * TG + tt * TT + ti;
          const bool use = valid && l < n;
          double* o = (double*)(alpha + (size_t)(use ? l : 0) * P + (use ? nu : 0));
#pragma unroll 1
          for (int cb2 = 0; cb2 < NCOL; cb2 += 16) {
            uint32_t vv[16];
            tmem_ld16(tmem + lane_addr + tt * NCOL + cb2, vv);
            if (use) {
              const int part = cb2 >= RBLK ? 1 : 0;          // Re columns, then Im
#pragma unroll
              for (int e = 0; e < 16; ++e) {
                const int r = rb * RBLK + (cb2 & (RBLK - 1)) + e;
                if (r < nrhs) atomicAdd(o + (size_t)r * n * P * 2 + part, (double)__uint_as_float(vv[e]));
              }
            }
          }
        }
        tc_fence_before();
        named_bar_sync(1, 128);
        if (b == 0) mbar_arrive(acc_empty);
        ++grp;
      }
    }
  } else if (warp >= 6) {
    // ---- generators: 64 threads, named barrier 2.  They walk the same chunks as the operand warps
    // one chunk ahead, writing the pair sequences of chunk c, split into BF16 planes, into buffer
    // c mod 2 once the operand warps have released it (chunk c - 2).
    const int gt = threadIdx.x - 192;
    const ffl kf = {k_hi, k_lo}, nr = {near_hi, near_lo};
    long long s = s0, chunk = 0;
    while (s < s1) {
      const long long gkey = s / n;
      const int g = (int)(gkey % ngroups);
      const int m0 = (int)(s - gkey * n);
      const int cnt = (int)min((long long)min(CHS, flush - m0 % flush), min(s1 - s, (long long)(n - m0)));
      const int cb = (int)(chunk & 1);
      if (gt == 0) {
        bool w = !*abort_flag;
        if (w && chunk >= 2) w = mbar_wait(raw_empty + 8 * cb, (uint32_t)(((chunk >> 1) - 1) & 1));
        if (!w && !*abort_flag) {
          *abort_flag = 1;
          atomicExch(err, 16);
        }
        *gbcast = w ? 1 : 0;
      }
      named_bar_sync(2, NGEN);
      if (!*gbcast) break;
      if (gt < TG * cnt) {
        const int i = gt % TG, j = gt / TG;
        const int l = g * TG + i, m = m0 + j;
        uint32_t* h = raw + ((size_t)cb * NPAIR + gt) * 3 * RWS;
        if (l < n && l != m) {
          hankel_planes<PT>(cff[l], cff[m], kf, nr, h);
        } else {
          for (int q = 0; q < 3 * RWS; ++q) h[q] = 0u;
        }
      }
      named_bar_sync(2, NGEN);
      if (gt == 0) mbar_arrive(raw_full + 8 * cb);
      ++chunk;
      s += cnt;
    }
  }
  __syncwarp();                                   // reconverge the producer and MMA warps
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, TMEM_COLS);
  }
}

template <int PT>
void launch_tc(int grid, cudaStream_t st, const float4* cff, int n, float kh, float kl, float nh, float nl,
               const unsigned char* img, int nrhs, long long nsteps, int flush, double2* alpha, int* err) {
  static std::once_flag attr;
  std::call_once(attr, [] {
    cudaFuncSetAttribute(k_translate_tc<PT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)TcShape<PT>::SMEM);
  });
  k_translate_tc<PT><<<grid, NTHR, TcShape<PT>::SMEM, st>>>(cff, n, kh, kl, nh, nl, img, nrhs, nsteps, flush, alpha, err);
}

int tc_group_size(int p) { return NTILE * (128 / (2 * p + 1)); }

int sm_count() {
  static int sms = 0;
  static std::once_flag once;
  std::call_once(once, [] {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
      cudaGetLastError();
      sms = 152;
    }
  });
  return sms;
}

}  // namespace

// alpha = T xs for nrhs right-hand sides on the tensor cores, near pairs excluded (the caller adds
// them with k_translate_near).
int translate_mixed_tc(lsms_ctx* c, int nrhs, const double2* xs, double2* alpha, cudaStream_t st) {
  const int n = c->n, p = c->p, P = c->P;
  if (n == 0 || nrhs == 0) return LSMS_OK;
  if (p < 6 || p > LSMS_MAX_P) return ctx_fail(c, LSMS_ERR_ARG, "tensor-core translation needs 6 <= p <= 15");
  int* err = tc_err_flag(c);
  if (!err) return ctx_fail(c, LSMS_ERR_STATE, "tensor-core state missing (set_particles first)");
  const int nrb = (nrhs + RBLK - 1) / RBLK;
  int rc;
  if ((rc = ensure(c, c->ws_tcb, (size_t)nrb * n * B_STAGE))) return rc;
  unsigned char* img = (unsigned char*)c->ws_tcb.ptr;
  cudaMemsetAsync(alpha, 0, (size_t)nrhs * n * P * sizeof(double2), st);
  long long tot = (long long)nrb * n * NCOL * 8;
  long long gb = (tot + 255) / 256;
  if (gb > 152 * 32) gb = 152 * 32;
  k_pack_b_tc<<<(int)gb, 256, 0, st>>>(xs, n, P, nrhs, nrb, img);
  const long long ngroups = (n + tc_group_size(p) - 1) / tc_group_size(p);
  const long long nsteps = (long long)nrb * ngroups * n;
  const int grid = (int)std::min<long long>(sm_count(), nsteps);
  const float kh = (float)c->k2, kl = (float)(c->k2 - (double)kh);
  const float nh = (float)c->near_r2, nl = (float)(c->near_r2 - (double)nh);
  const float4* cff = (const float4*)c->d_lp_misc;
  const int flush = c->tc_flush > 0 ? std::min(c->tc_flush, n) : n;
  switch (p) {
    case 6: launch_tc<6>(grid, st, cff, n, kh, kl, nh, nl, img, nrhs, nsteps, flush, alpha, err); break;
    case 7: launch_tc<7>(grid, st, cff, n, kh, kl, nh, nl, img, nrhs, nsteps, flush, alpha, err); break;
    case 8: launch_tc<8>(grid, st, cff, n, kh, kl, nh, nl, img, nrhs, nsteps, flush, alpha, err); break;
    case 9: launch_tc<9>(grid, st, cff, n, kh, kl, nh, nl, img, nrhs, nsteps, flush, alpha, err); break;
    case 10: launch_tc<10>(grid, st, cff, n, kh, kl, nh, nl, img, nrhs, nsteps, flush, alpha, err); break;
    case 11: launch_tc<11>(grid, st, cff, n, kh, kl, nh, nl, img, nrhs, nsteps, flush, alpha, err); break;
    case 12: launch_tc<12>(grid, st, cff, n, kh, kl, nh, nl, img, nrhs, nsteps, flush, alpha, err); break;
    case 13: launch_tc<13>(grid, st, cff, n, kh, kl, nh, nl, img, nrhs, nsteps, flush, alpha, err); break;
    case 14: launch_tc<14>(grid, st, cff, n, kh, kl, nh, nl, img, nrhs, nsteps, flush, alpha, err); break;
    default: launch_tc<15>(grid, st, cff, n, kh, kl, nh, nl, img, nrhs, nsteps, flush, alpha, err); break;
  }
  return check_cuda(c, "translate_mixed_tc");
}

extern "C" int lsms_set_tc_translation(lsms_ctx* c, int min_rhs, int flush) {
  if (!c) return LSMS_ERR_ARG;
  if (min_rhs < 0 || flush < 0) return ctx_fail(c, LSMS_ERR_ARG, "min_rhs and flush must be >= 0");
  c->tc_min_rhs = min_rhs;
  if (flush > 0) c->tc_flush = flush;
  for (lsms_ctx* k : c->kids) {
    k->tc_min_rhs = min_rhs;
    if (flush > 0) k->tc_flush = flush;
  }
  return LSMS_OK;
}
