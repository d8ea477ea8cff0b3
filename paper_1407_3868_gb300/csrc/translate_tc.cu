// Graf translation of a block of right-hand sides on the tensor cores (tcgen05; Sec. 3.2
// Lemma 3.1, Eq. "trans"), the mixed-precision form used when many sources are solved together.
//
// With R right-hand sides, alpha^l(r) = sum_{m != l} T^{lm} beta^m(r) is for every disc pair a
// complex (P x P) . (P x R) product with the Toeplitz block T^{lm}_{nu n} = h_{n - nu},
// h_s = H_s(k2 rho) exp(i s phi) (rho, phi: distance and angle of x_l - x_m).  It runs as real BF16
// MMAs with FP32 accumulation in tensor memory:
//
//   D (128 rows: 2 targets x 64, 64 columns: right-hand sides) += A (128 x 64) . B (64 x 64)^T
//
// A is the real embedding of two targets' Toeplitz blocks for one source disc: row nu holds
// Re alpha_nu, row P + nu holds Im alpha_nu; column n multiplies Re beta_n, column P + n Im beta_n;
// the entries are (Tr, -Ti) and (Ti, Tr).  B holds the source's coefficients for 64 right-hand
// sides in the same K order.  Both are split into three BF16 planes x = hi + mid + lo and the six
// plane products with terms down to 2^-16 relative are accumulated, so the contraction is as
// accurate as FP32 (as in the contour contractions).  The Hankel sequences are the FP32 ones of the
// CUDA-core path; near pairs (k2 rho < 25) and the self pair are left to k_translate_near.
//
// A persistent CTA (one per SM) owns a contiguous range of steps (right-hand-side block, group of 16
// target discs, source disc) and keeps the 8 accumulators of its current group in the 512 columns of
// tensor memory.  Per step: warp 0 lane 0 copies the source's B planes (24 KB, prepared once per
// application in the swizzled shared-memory image) with a bulk copy into a 2-stage ring; warps 2-5
// generate the chunk's pair sequences and write the eight A tiles (48 KB each) into a 2-stage ring;
// warp 1 lane 0 issues 24 tcgen05.mma per tile.  When the group changes, warps 2-5 read the
// accumulators (tcgen05.ld) and add them into the FP64 output with atomics.  Every mbarrier wait is
// bounded; on a timeout the CTA records an error, waits for its copies in flight, frees its tensor
// memory and returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "lsms_internal.h"
#include "lsms_ops.h"
#include "ff_hankel.cuh"
#include "tc_ptx.cuh"

namespace {

constexpr int TG = 16;                  // target discs per group
constexpr int NTILE = TG / 2;           // accumulator tiles per group (two targets each)
constexpr int RBLK = 64;                // right-hand sides per block (MMA N)
constexpr int A_PLANE = 128 * 128;      // bytes: 128 rows x 64 BF16
constexpr int A_STAGE = 3 * A_PLANE;    // 49152
constexpr int B_PLANE = RBLK * 128;     // bytes: 64 rows x 64 BF16
constexpr int B_STAGE = 3 * B_PLANE;    // 24576
constexpr int NA = 2, NBS = 2;          // ring depths
constexpr int CHS = 4;                  // source discs per sequence chunk
constexpr int SEQ = 64;                 // float2 slots per pair sequence (>= 4p + 1)
constexpr int NTHR = 192;               // warp 0: copies, warp 1: MMA, warps 2-5: operands, epilogue
constexpr int SEQ_BYTES = CHS * TG * SEQ * 8;
constexpr int BAR_BYTES = 256;
constexpr size_t TC_SMEM = 1024 + (size_t)NA * A_STAGE + (size_t)NBS * B_STAGE + SEQ_BYTES + BAR_BYTES;
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t IDESC_T = idesc_bf16(128, RBLK);
// plane products (A plane, B plane): hi.hi, hi.mid, mid.hi, hi.lo, lo.hi, mid.mid
__host__ __device__ constexpr int plane_a(int q) { return q == 2 || q == 5 ? 1 : (q == 4 ? 2 : 0); }
__host__ __device__ constexpr int plane_b(int q) { return q == 1 || q == 5 ? 1 : (q == 3 ? 2 : 0); }

// B image of one (right-hand-side block, source disc): 3 planes x 64 rows (right-hand sides) x 128
// bytes (K: Re beta_n at n, Im beta_n at P + n, zero from 2P), chunk c of row r at c ^ (r mod 8).
__global__ void k_pack_b_tc(const double2* __restrict__ xs, int n, int P, int nrhs, int nrb,
                            unsigned char* __restrict__ img) {
  const long long total = (long long)nrb * n * RBLK * 8;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
       id += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(id & 7), r = (int)((id >> 3) & (RBLK - 1));
    const long long sm = id >> 9;                       // rb * n + m
    const int m = (int)(sm % n), rb = (int)(sm / n);
    const int rr = rb * RBLK + r;
    uint32_t w[3][4];
#pragma unroll
    for (int e = 0; e < 8; e += 2) {
      __nv_bfloat16 h[2], md[2], lo[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int kk = 8 * c + e + u;
        double x = 0.0;
        if (rr < nrhs) {
          if (kk < P) x = xs[((size_t)rr * n + m) * P + kk].x;
          else if (kk < 2 * P) x = xs[((size_t)rr * n + m) * P + kk - P].y;
        }
        split3(x, h[u], md[u], lo[u]);
      }
      w[0][e / 2] = (uint32_t)__bfloat16_as_ushort(h[0]) | ((uint32_t)__bfloat16_as_ushort(h[1]) << 16);
      w[1][e / 2] = (uint32_t)__bfloat16_as_ushort(md[0]) | ((uint32_t)__bfloat16_as_ushort(md[1]) << 16);
      w[2][e / 2] = (uint32_t)__bfloat16_as_ushort(lo[0]) | ((uint32_t)__bfloat16_as_ushort(lo[1]) << 16);
    }
    unsigned char* base = img + (size_t)sm * B_STAGE + r * 128 + ((c ^ (r & 7)) * 16);
#pragma unroll
    for (int pl = 0; pl < 3; ++pl)
      *(uint4*)(base + pl * B_PLANE) = make_uint4(w[pl][0], w[pl][1], w[pl][2], w[pl][3]);
  }
}

template <int PT>
__global__ void __launch_bounds__(NTHR, 1)
k_translate_tc(const float4* __restrict__ cff, int n, float k_hi, float k_lo, float near_hi,
               float near_lo, const unsigned char* __restrict__ bimg, int nrhs, long long nsteps,
               int flush, double2* __restrict__ alpha, int* __restrict__ err) {
  constexpr int p = PT, P = 2 * PT + 1;
  constexpr int K2 = 2 * P;                        // real K in use (<= 62)
  constexpr int NCH = (K2 + 7) / 8;                // 16-byte chunks written per A row
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sA = smem;
  unsigned char* sB = sA + NA * A_STAGE;
  float2* seq = (float2*)(sB + NBS * B_STAGE);
  uint64_t* bars = (uint64_t*)((unsigned char*)seq + SEQ_BYTES);
  uint32_t* tmem_slot = (uint32_t*)(bars + 2 * NA + 2 * NBS + 3);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  volatile int* bcast = abort_flag + 1;
  const uint32_t a_full = smem_u32(bars), a_empty = a_full + 8 * NA;
  const uint32_t b_full = a_empty + 8 * NA, b_empty = b_full + 8 * NBS;
  const uint32_t acc_full = b_empty + 8 * NBS, acc_empty = acc_full + 8, done = acc_empty + 8;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ngroups = (n + TG - 1) / TG;
  // accumulation segment of a step: (right-hand-side block, group, block of `flush` sources); the
  // accumulators are drained into the FP64 output at every segment end, which bounds the number of
  // MMAs summed in FP32 in one accumulator
  const int nseg = (n + flush - 1) / flush;
  auto segkey = [&](long long s) { return (s / n) * nseg + (s % n) / flush; };
  const long long s0 = nsteps * blockIdx.x / gridDim.x;
  const long long s1 = nsteps * (blockIdx.x + 1) / gridDim.x;

  // A ring zeroed once: rows and columns past 2P are never written and stay zero
  for (int i = threadIdx.x; i < NA * A_STAGE / 16; i += NTHR) ((uint4*)sA)[i] = make_uint4(0u, 0u, 0u, 0u);
  fence_proxy_async_smem();                       // the zeros are read by the tensor cores
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
    *abort_flag = 0;
    *bcast = 0;
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
    // ---- MMA issuer ----
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
        const uint32_t a0 = smem_u32(sA + as * A_STAGE);
#pragma unroll
        for (int q = 0; q < 6; ++q)
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
            mma_bf16(tmem + tt * RBLK, sw128_desc(a0 + plane_a(q) * A_PLANE + kk * 32),
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
  } else if (warp >= 2) {
    // ---- operands (pair sequences, A tiles) and epilogue: 128 threads, named barrier 1 ----
    const int b = threadIdx.x - 64;
    const ffl kf = {k_hi, k_lo}, nr = {near_hi, near_lo};
    long long t = 0, s = s0;
    int grp = 0;
    while (s < s1) {
      const long long key = segkey(s), gkey = s / n;      // gkey = rb * ngroups + g
      const int g = (int)(gkey % ngroups);
      const int m0 = (int)(s - gkey * n);
      const int cnt = (int)min((long long)min(CHS, flush - m0 % flush), min(s1 - s, (long long)(n - m0)));
      if (b < TG * cnt) {
        const int i = b % TG, j = b / TG;
        const int l = g * TG + i, m = m0 + j;
        float2* h = seq + (j * TG + i) * SEQ;
        if (l < n && l != m) {
          hankel_sequence_f32(cff[l], cff[m], kf, p, nr, h);
        } else {
          for (int q = 0; q <= 4 * p; ++q) h[q] = make_float2(0.f, 0.f);
        }
      }
      named_bar_sync(1, 128);
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
          const int i = 2 * tt + (b >> 6), rl = b & 63;
          if (rl < K2) {
            const bool im = rl >= P;
            const int nu = im ? rl - P : rl;
            const float2* hs = seq + (j * TG + i) * SEQ + 2 * p - nu;   // hs[n] = h_{n - nu}
            float2 wv[P];
#pragma unroll
            for (int q = 0; q < P; ++q) wv[q] = hs[q];
            unsigned char* row = sA + as * A_STAGE + b * 128;
#pragma unroll
            for (int c = 0; c < NCH; ++c) {
              float v[8];
#pragma unroll
              for (int e = 0; e < 8; ++e) {
                const int kk = 8 * c + e;
                float x = 0.f;
                if (kk < P) x = im ? wv[kk].y : wv[kk].x;
                else if (kk < K2) x = im ? wv[kk - P].x : -wv[kk - P].y;
                v[e] = x;
              }
              uint4 hi, mid, lo;
              split3x8(v, hi, mid, lo);
              const int pos = (c ^ (b & 7)) * 16;
              *(uint4*)(row + pos) = hi;
              *(uint4*)(row + A_PLANE + pos) = mid;
              *(uint4*)(row + 2 * A_PLANE + pos) = lo;
            }
          }
          fence_proxy_async_smem();
          named_bar_sync(1, 128);
          if (b == 0) mbar_arrive(a_full + 8 * as);
        }
      }
      if (!ok) break;
      s += cnt;
      if (s == s1 || segkey(s) != key) {
        // group done: read the accumulators and add them into alpha
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
        const int q4 = warp & 3;                   // tensor-memory lane quarter of this warp
        const int row = 32 * q4 + lane;
        const int rb = (int)(gkey / ngroups);
        const int rl = row & 63;
        const int nu = rl < P ? rl : rl - P;
#pragma unroll 1
        for (int tt = 0; tt < NTILE; ++tt) {
          const int l = g * TG + 2 * tt + (row >> 6);
          const bool use = l < n && rl < K2;
          double* o = (double*)(alpha + (size_t)l * P + nu) + (rl < P ? 0 : 1);
#pragma unroll 1
          for (int cb = 0; cb < RBLK; cb += 16) {
            uint32_t v[16];
            tmem_ld16(tmem + ((uint32_t)(32 * q4) << 16) + tt * RBLK + cb, v);
            if (use) {
#pragma unroll
              for (int e = 0; e < 16; ++e) {
                const int r = rb * RBLK + cb + e;
                if (r < nrhs) atomicAdd(o + (size_t)r * n * P * 2, (double)__uint_as_float(v[e]));
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
    cudaFuncSetAttribute(k_translate_tc<PT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM);
  });
  k_translate_tc<PT><<<grid, NTHR, TC_SMEM, st>>>(cff, n, kh, kl, nh, nl, img, nrhs, nsteps, flush, alpha, err);
}

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
  long long tot = (long long)nrb * n * RBLK * 8;
  long long gb = (tot + 255) / 256;
  if (gb > 152 * 32) gb = 152 * 32;
  k_pack_b_tc<<<(int)gb, 256, 0, st>>>(xs, n, P, nrhs, nrb, img);
  const long long ngroups = (n + TG - 1) / TG;
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
