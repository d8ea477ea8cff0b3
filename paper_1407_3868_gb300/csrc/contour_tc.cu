// Mixed-precision Sommerfeld contractions on the tensor cores (tcgen05 + TMA).
//
// The aggregate G = E_agg . xs (Thm 5.2 / Eq. "invfft": 2 N_S x N times N x P, complex) and the
// disaggregate alpha += E_dis . V (Lemma 5.1 / Eq. "JA2": N x 2 N_S times 2 N_S x P) are dense
// complex contractions.  Each is computed as one real GEMM: a complex row (ar0, ai0, ar1, ai1, ...)
// times the real embedding of the right operand (for output column Re: br, -bi; for Im: bi, br),
// in BF16 with FP32 accumulation in tensor memory.  Every FP64 operand x is split into three BF16
// planes x = hi + mid + lo (each the BF16 rounding of the remainder), and the six plane products
// hi.hi, hi.mid, mid.hi, hi.lo, lo.hi, mid.mid are accumulated: the dropped terms are O(2^-24 |a||b|),
// so the contraction is as accurate as FP32.
//
// Kernel: one CTA per (128-row tile, 64-column tile, K range).  Thread 0 streams the six operand
// tiles of each 64-wide K block (three planes of A, three of B) with TMA into a 3-stage ring of
// 128-byte-swizzled shared memory; thread 32 issues the 24 tcgen05.mma (6 products x 4 K steps of
// 16) per block into one 128 x 64 FP32 accumulator in tensor memory and releases each stage with
// tcgen05.commit; after the last block all four warps read the accumulator (tcgen05.ld, warp w owns
// rows 32w..32w+31) and add it atomically into the FP32 output.  Every mbarrier wait is bounded; a
// timeout sets an error flag that the host reads, and the CTA still frees its tensor memory.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "lsms_internal.h"
#include "lsms_ops.h"
#include "tc_ptx.cuh"

namespace {

constexpr int BM = 128, BN = 64, BK = 64, STAGES = 3, NPL = 3;
constexpr int A_TILE = BM * BK * 2;                         // bytes of one A plane tile
constexpr int B_TILE = BN * BK * 2;                         // bytes of one B plane tile
constexpr int STAGE_BYTES = NPL * (A_TILE + B_TILE);        // 73728
constexpr int GEMM_SMEM = STAGES * STAGE_BYTES + 1024 + 256;
constexpr uint32_t TMEM_COLS = 64;

// Instruction descriptor: M = 128, N = 64.
constexpr uint32_t IDESC = idesc_bf16(BM, BN);

// Plane products: (A plane, B plane) pairs of hi (0), mid (1), lo (2).
__constant__ int kPairA[6] = {0, 0, 1, 0, 2, 1};
__constant__ int kPairB[6] = {0, 1, 0, 2, 0, 1};

// C[row][col] += sum_k A[row][k] B^T[col][k] over this CTA's K blocks, for the 6 plane products.
// ta: A planes, 3-D tensor {Kpad, M, 3}; tb: B planes {Kpad, Ncols, 3}; both BF16, box {64, rows, 1}.
__global__ void __launch_bounds__(128, 1)
k_gemm_bf16x6(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, int M,
              int Ncols, int kblocks, int kchunk, float* __restrict__ C, int ldc,
              int* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)(smem + STAGES * STAGE_BYTES);   // full[S], empty[S], done
  uint32_t* tmem_slot = (uint32_t*)(bars + 2 * STAGES + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int kb0 = blockIdx.z * kchunk;
  const int nkb = min(kchunk, kblocks - kb0);
  if (nkb <= 0) return;
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES), done = smem_u32(bars + 2 * STAGES);
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  if (warp == 0) {
    tmem_alloc(smem_u32(tmem_slot), TMEM_COLS);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t sbase = smem_u32(smem);

  if (threadIdx.x == 0) {
    // producer: TMA of 3 A planes and 3 B planes per K block
    bool ok = true;
    for (int i = 0; i < nkb; ++i) {
      const int s = i % STAGES, round = i / STAGES;
      if (round > 0 && !mbar_wait(empty0 + 8 * s, (round - 1) & 1)) {
        ok = false;
        break;
      }
      const uint32_t st = sbase + s * STAGE_BYTES;
      mbar_expect_tx(full0 + 8 * s, STAGE_BYTES);
      const int k = (kb0 + i) * BK;
      for (int pl = 0; pl < NPL; ++pl) tma_load_3d(st + pl * A_TILE, &ta, full0 + 8 * s, k, m0, pl);
      for (int pl = 0; pl < NPL; ++pl)
        tma_load_3d(st + NPL * A_TILE + pl * B_TILE, &tb, full0 + 8 * s, k, n0, pl);
    }
    if (!ok) atomicExch(err, 1);
  } else if (threadIdx.x == 32) {
    // MMA issuer
    bool ok = true;
    for (int i = 0; i < nkb; ++i) {
      const int s = i % STAGES, round = i / STAGES;
      if (!mbar_wait(full0 + 8 * s, round & 1)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t st = sbase + s * STAGE_BYTES;
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        const uint32_t a = st + kPairA[q] * A_TILE;
        const uint32_t b = st + NPL * A_TILE + kPairB[q] * B_TILE;
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk)
          mma_bf16(tmem, sw128_desc(a + kk * 32), sw128_desc(b + kk * 32), IDESC, (i | q | kk) != 0);
      }
      mma_commit(empty0 + 8 * s);
    }
    mma_commit(done);
    if (!ok) atomicExch(err, 2);
  }
  __syncwarp();
  // epilogue: all warps
  bool dok = mbar_wait(done, 0);
  dok = __all_sync(0xffffffffu, dok);
  tc_fence_after();
  if (dok) {
    const int row = m0 + warp * 32 + lane;
    uint32_t v[16];
#pragma unroll
    for (int cb = 0; cb < BN; cb += 16) {
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + cb, v);
      if (row < M) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int col = n0 + cb + j;
          if (col < Ncols) atomicAdd(&C[(size_t)row * ldc + col], __uint_as_float(v[j]));
        }
      }
    }
  } else if (lane == 0) {
    atomicExch(err, 3);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, TMEM_COLS);
  }
}


// A planes from a complex row-major matrix src[rows][K]: plane[pl][row][2k + e] = part e of
// src[row][k]; row pitch kpad (zero padding beyond 2K is left untouched).
__global__ void k_split_a(const double2* __restrict__ src, int rows, int K, int kpad,
                          __nv_bfloat16* __restrict__ planes) {
  const long long total = (long long)rows * K;
  const size_t plane = (size_t)rows * kpad;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int row = (int)(i / K), k = (int)(i - (long long)row * K);
    const double2 v = src[i];
    __nv_bfloat16 h, m, l;
    const size_t o = (size_t)row * kpad + 2 * k;
    split3(v.x, h, m, l);
    planes[o] = h; planes[plane + o] = m; planes[2 * plane + o] = l;
    split3(v.y, h, m, l);
    planes[o + 1] = h; planes[plane + o + 1] = m; planes[2 * plane + o + 1] = l;
  }
}

// B^T planes of the real embedding of a complex right operand src[r][Kc][P]:
// column c = r 2P + h P + n (h = 0: real part of the output, 1: imaginary part), row 2k + e:
//   h = 0: e = 0 -> Re src, e = 1 -> -Im src;   h = 1: e = 0 -> Im src, e = 1 -> Re src.
__device__ __forceinline__ void put_b(__nv_bfloat16* planes, size_t plane, int kpad, int c, int kr,
                                      double v) {
  __nv_bfloat16 h, m, l;
  split3(v, h, m, l);
  const size_t o = (size_t)c * kpad + kr;
  planes[o] = h;
  planes[plane + o] = m;
  planes[2 * plane + o] = l;
}

__global__ void k_split_b(const double2* __restrict__ src, int nrhs, int Kc, int P, int ncols_pad,
                          int kpad, __nv_bfloat16* __restrict__ planes) {
  const long long total = (long long)nrhs * Kc * P;
  const size_t plane = (size_t)ncols_pad * kpad;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int n = (int)(i % P);
    const long long rk = i / P;
    const int k = (int)(rk % Kc), r = (int)(rk / Kc);
    const double2 v = src[i];
    const int cre = r * 2 * P + n, cim = cre + P;
    put_b(planes, plane, kpad, cre, 2 * k, v.x);
    put_b(planes, plane, kpad, cre, 2 * k + 1, -v.y);
    put_b(planes, plane, kpad, cim, 2 * k, v.y);
    put_b(planes, plane, kpad, cim, 2 * k + 1, v.x);
  }
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 warp_sum(double2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}

// Per node (one warp per (r, nu)): P+, Q- from the aggregate's FP32 output (order dots with c_n w^n,
// Thm 5.2), the closed-form layer response (Eq. "sommerfeldsys"), V = U sigma, written directly as
// the disaggregate's B^T planes (rows 2 nu' + e, nu' = nu top, ns + nu bottom).
__global__ void k_node_stage_tc(int ns, int P, int nrhs, const float* __restrict__ Cagg, int ldc,
                                const double2* __restrict__ fagg, const double2* __restrict__ refl,
                                const double2* __restrict__ udis, int ncols_pad, int kpad,
                                __nv_bfloat16* __restrict__ planes) {
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (gw >= ns * nrhs) return;
  const int r = gw / ns, v = gw - r * ns;
  double2 a = make_double2(0.0, 0.0), b = make_double2(0.0, 0.0);
  if (lane < P) {
    const int cre = r * 2 * P + lane, cim = cre + P;
    const double2 gt = make_double2(Cagg[(size_t)v * ldc + cre], Cagg[(size_t)v * ldc + cim]);
    const double2 gb = make_double2(Cagg[(size_t)(ns + v) * ldc + cre], Cagg[(size_t)(ns + v) * ldc + cim]);
    a = cmul(fagg[(size_t)v * P + lane], gt);
    b = cmul(fagg[(size_t)(ns + v) * P + lane], gb);
  }
  const double2 Pp = warp_sum(a), Qm = warp_sum(b);
  const double2 sp = make_double2(cmul(refl[4 * v], Pp).x + cmul(refl[4 * v + 1], Qm).x,
                                  cmul(refl[4 * v], Pp).y + cmul(refl[4 * v + 1], Qm).y);
  const double2 sm = make_double2(cmul(refl[4 * v + 2], Pp).x + cmul(refl[4 * v + 3], Qm).x,
                                  cmul(refl[4 * v + 2], Pp).y + cmul(refl[4 * v + 3], Qm).y);
  if (lane < P) {
    const size_t plane = (size_t)ncols_pad * kpad;
    const int cre = r * 2 * P + lane, cim = cre + P;
    const double2 vt = cmul(udis[(size_t)v * P + lane], sp);
    const double2 vb = cmul(udis[(size_t)(ns + v) * P + lane], sm);
    const int kt = 2 * v, kb = 2 * (ns + v);
    put_b(planes, plane, kpad, cre, kt, vt.x);
    put_b(planes, plane, kpad, cre, kt + 1, -vt.y);
    put_b(planes, plane, kpad, cim, kt, vt.y);
    put_b(planes, plane, kpad, cim, kt + 1, vt.x);
    put_b(planes, plane, kpad, cre, kb, vb.x);
    put_b(planes, plane, kpad, cre, kb + 1, -vb.y);
    put_b(planes, plane, kpad, cim, kb, vb.y);
    put_b(planes, plane, kpad, cim, kb + 1, vb.x);
  }
}

// G[r][row][n] = C[row][r 2P + n] + i C[row][r 2P + P + n]  (aggregate output as complex doubles)
__global__ void k_c_to_complex(const float* __restrict__ C, int ldc, int rows, int P, int nrhs,
                               double2* __restrict__ G) {
  const long long total = (long long)nrhs * rows * P;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int n = (int)(i % P);
    const long long rr = i / P;
    const int row = (int)(rr % rows), r = (int)(rr / rows);
    G[i] = make_double2(C[(size_t)row * ldc + r * 2 * P + n], C[(size_t)row * ldc + r * 2 * P + P + n]);
  }
}

// alpha[r][i][m] += C[i][r 2P + m] + i C[i][r 2P + P + m]
__global__ void k_c_add_alpha(const float* __restrict__ C, int ldc, int rows, int P, int nrhs,
                              double2* __restrict__ alpha) {
  const long long total = (long long)nrhs * rows * P;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int m = (int)(i % P);
    const long long rr = i / P;
    const int row = (int)(rr % rows), r = (int)(rr / rows);
    alpha[i].x += C[(size_t)row * ldc + r * 2 * P + m];
    alpha[i].y += C[(size_t)row * ldc + r * 2 * P + P + m];
  }
}

inline int grid_for(long long total, int block) {
  long long g = (total + block - 1) / block;
  if (g > 152LL * 32) g = 152LL * 32;
  if (g < 1) g = 1;
  return (int)g;
}
inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::mutex g_encode_mu;

int get_encoder(lsms_ctx* c) {
  std::lock_guard<std::mutex> lock(g_encode_mu);
  if (g_encode) return LSMS_OK;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !fn) {
    cudaGetLastError();
    return ctx_fail(c, LSMS_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
  }
  g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  return LSMS_OK;
}

// 3-D BF16 tensor {kpad, rows, 3 planes}, box {64, box_rows, 1}, 128-byte swizzle, zero fill.
int make_map(lsms_ctx* c, CUtensorMap* map, void* base, int kpad, int rows, int box_rows) {
  int rc;
  if ((rc = get_encoder(c))) return rc;
  cuuint64_t dims[3] = {(cuuint64_t)kpad, (cuuint64_t)rows, (cuuint64_t)NPL};
  cuuint64_t strides[2] = {(cuuint64_t)kpad * 2, (cuuint64_t)kpad * 2 * rows};
  cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)box_rows, 1};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return ctx_fail(c, LSMS_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return LSMS_OK;
}

}  // namespace

// Per-context state of the tensor-core path.
struct TcState {
  int n = 0, ns = 0, P = 0;
  int kpad_agg = 0, kpad_dis = 0;          // padded real K of the two GEMMs
  __nv_bfloat16* a_agg = nullptr;          // [3][2ns][kpad_agg]
  __nv_bfloat16* a_dis = nullptr;          // [3][n][kpad_dis]
  CUtensorMap map_a_agg, map_a_dis;
  int ncols_pad = 0;                       // capacity of the B planes / outputs in columns
  __nv_bfloat16* b_agg = nullptr;          // [3][ncols_pad][kpad_agg]
  __nv_bfloat16* b_dis = nullptr;          // [3][ncols_pad][kpad_dis]
  CUtensorMap map_b_agg, map_b_dis;
  float* c_agg = nullptr;                  // [2ns][ncols_pad]
  float* c_dis = nullptr;                  // [n][ncols_pad]
  int* d_err = nullptr;
};

void tc_free(lsms_ctx* c) {
  TcState* t = (TcState*)c->tc;
  if (!t) return;
  void* ptrs[] = {t->a_agg, t->a_dis, t->b_agg, t->b_dis, t->c_agg, t->c_dis, t->d_err};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete t;
  c->tc = nullptr;
}

// Split the layout's plane-wave tables into BF16 planes and describe them for TMA.
int tc_setup(lsms_ctx* c) {
  tc_free(c);
  if (c->n <= 0) return LSMS_OK;
  TcState* t = new TcState();
  c->tc = t;
  t->n = c->n;
  t->ns = c->ns;
  t->P = c->P;
  t->kpad_agg = round_up(2 * c->n, BK);
  t->kpad_dis = round_up(4 * c->ns, BK);
  const size_t sa = (size_t)NPL * 2 * c->ns * t->kpad_agg * 2;
  const size_t sd = (size_t)NPL * c->n * t->kpad_dis * 2;
  if (cudaMalloc((void**)&t->a_agg, sa) != cudaSuccess || cudaMalloc((void**)&t->a_dis, sd) != cudaSuccess ||
      cudaMalloc((void**)&t->d_err, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return ctx_fail(c, LSMS_ERR_OOM, "cudaMalloc failed for the BF16 plane tables");
  }
  cudaMemsetAsync(t->a_agg, 0, sa, c->stream);
  cudaMemsetAsync(t->a_dis, 0, sd, c->stream);
  cudaMemsetAsync(t->d_err, 0, sizeof(int), c->stream);
  k_split_a<<<grid_for((long long)2 * c->ns * c->n, 256), 256, 0, c->stream>>>(c->d_eagg, 2 * c->ns, c->n, t->kpad_agg, t->a_agg);
  k_split_a<<<grid_for((long long)c->n * 2 * c->ns, 256), 256, 0, c->stream>>>(c->d_edis, c->n, 2 * c->ns, t->kpad_dis, t->a_dis);
  cudaStreamSynchronize(c->stream);
  int rc;
  if ((rc = check_cuda(c, "tc_setup"))) return rc;
  if ((rc = make_map(c, &t->map_a_agg, t->a_agg, t->kpad_agg, 2 * c->ns, BM))) return rc;
  if ((rc = make_map(c, &t->map_a_dis, t->a_dis, t->kpad_dis, c->n, BM))) return rc;
  static std::once_flag attr;
  std::call_once(attr, [] {
    cudaFuncSetAttribute(k_gemm_bf16x6, cudaFuncAttributeMaxDynamicSharedMemorySize, GEMM_SMEM);
  });
  return LSMS_OK;
}

// Grow the per-application buffers to hold ncols output columns.
static int tc_reserve(lsms_ctx* c, int ncols, cudaStream_t st) {
  TcState* t = (TcState*)c->tc;
  if (!t) return ctx_fail(c, LSMS_ERR_STATE, "tensor-core tables missing");
  const int need = round_up(ncols, BN);
  if (need <= t->ncols_pad) return LSMS_OK;
  void* ptrs[] = {t->b_agg, t->b_dis, t->c_agg, t->c_dis};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  t->b_agg = t->b_dis = nullptr;
  t->c_agg = t->c_dis = nullptr;
  t->ncols_pad = 0;
  const size_t sb1 = (size_t)NPL * need * t->kpad_agg * 2, sb2 = (size_t)NPL * need * t->kpad_dis * 2;
  if (cudaMalloc((void**)&t->b_agg, sb1) != cudaSuccess || cudaMalloc((void**)&t->b_dis, sb2) != cudaSuccess ||
      cudaMalloc((void**)&t->c_agg, (size_t)2 * t->ns * need * 4) != cudaSuccess ||
      cudaMalloc((void**)&t->c_dis, (size_t)t->n * need * 4) != cudaSuccess) {
    cudaGetLastError();
    return ctx_fail(c, LSMS_ERR_OOM, "cudaMalloc failed for the BF16 operand planes");
  }
  cudaMemsetAsync(t->b_agg, 0, sb1, st);     // padding rows and columns stay zero
  cudaMemsetAsync(t->b_dis, 0, sb2, st);
  t->ncols_pad = need;
  int rc;
  if ((rc = make_map(c, &t->map_b_agg, t->b_agg, t->kpad_agg, need, BN))) return rc;
  if ((rc = make_map(c, &t->map_b_dis, t->b_dis, t->kpad_dis, need, BN))) return rc;
  return check_cuda(c, "tc_reserve");
}

static void launch_gemm(const CUtensorMap& ta, const CUtensorMap& tb, int M, int ncols, int ncols_pad,
                        int kpad, float* C, int* err, cudaStream_t st) {
  const int mt = (M + BM - 1) / BM, nt = ncols_pad / BN, kb = kpad / BK;
  int split = 152 / (mt * nt);
  if (split < 1) split = 1;
  if (split > kb) split = kb;
  const int kchunk = (kb + split - 1) / split;
  split = (kb + kchunk - 1) / kchunk;
  dim3 grid(mt, nt, split);
  k_gemm_bf16x6<<<grid, 128, GEMM_SMEM, st>>>(ta, tb, M, ncols, kb, kchunk, C, ncols_pad, err);
}

int* tc_err_flag(lsms_ctx* c) {
  TcState* t = (TcState*)c->tc;
  return t ? t->d_err : nullptr;
}

int mixed_check(lsms_ctx* c) {
  if (is_batch(c)) return batch_mixed_check(c);
  TcState* t = (TcState*)c->tc;
  if (!t) return LSMS_OK;
  int h = 0;
  if (cudaMemcpy(&h, t->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return check_cuda(c, "mixed_check");
  if (h) {
    cudaMemset(t->d_err, 0, sizeof(int));
    return ctx_fail(c, LSMS_ERR_CUDA, "tensor-core contraction timed out waiting on a barrier (code " + std::to_string(h) + ")");
  }
  return LSMS_OK;
}

// G[r][2ns][P] = E_agg . xs   (complex doubles out)
int aggregate_mixed(lsms_ctx* c, int nrhs, const double2* xs, double2* G, cudaStream_t st) {
  int rc;
  const int P = c->P, ncols = nrhs * 2 * P;
  if ((rc = tc_reserve(c, ncols, st))) return rc;
  TcState* t = (TcState*)c->tc;
  k_split_b<<<grid_for((long long)nrhs * c->n * P, 256), 256, 0, st>>>(xs, nrhs, c->n, P, t->ncols_pad, t->kpad_agg, t->b_agg);
  cudaMemsetAsync(t->c_agg, 0, (size_t)2 * c->ns * t->ncols_pad * 4, st);
  launch_gemm(t->map_a_agg, t->map_b_agg, 2 * c->ns, ncols, t->ncols_pad, t->kpad_agg, t->c_agg, t->d_err, st);
  k_c_to_complex<<<grid_for((long long)nrhs * 2 * c->ns * P, 256), 256, 0, st>>>(t->c_agg, t->ncols_pad, 2 * c->ns, P, nrhs, G);
  return check_cuda(c, "aggregate_mixed");
}

// alpha[r][N][P] += E_dis . V, V[r][2ns][P]
int disaggregate_mixed(lsms_ctx* c, int nrhs, const double2* V, double2* alpha, cudaStream_t st) {
  int rc;
  const int P = c->P, ncols = nrhs * 2 * P;
  if ((rc = tc_reserve(c, ncols, st))) return rc;
  TcState* t = (TcState*)c->tc;
  k_split_b<<<grid_for((long long)nrhs * 2 * c->ns * P, 256), 256, 0, st>>>(V, nrhs, 2 * c->ns, P, t->ncols_pad, t->kpad_dis, t->b_dis);
  cudaMemsetAsync(t->c_dis, 0, (size_t)c->n * t->ncols_pad * 4, st);
  launch_gemm(t->map_a_dis, t->map_b_dis, c->n, ncols, t->ncols_pad, t->kpad_dis, t->c_dis, t->d_err, st);
  k_c_add_alpha<<<grid_for((long long)nrhs * c->n * P, 256), 256, 0, st>>>(t->c_dis, t->ncols_pad, c->n, P, nrhs, alpha);
  return check_cuda(c, "disaggregate_mixed");
}

// alpha += R xs: aggregate GEMM -> per-node stage writing the second GEMM's planes -> disaggregate.
// The reflected coupling up to (excluding) the final add into alpha, on stream st.
int reflection_mixed_stage(lsms_ctx* c, int nrhs, const double2* xs, cudaStream_t st) {
  int rc;
  const int P = c->P, ncols = nrhs * 2 * P, ns = c->ns;
  if ((rc = tc_reserve(c, ncols, st))) return rc;
  TcState* t = (TcState*)c->tc;
  k_split_b<<<grid_for((long long)nrhs * c->n * P, 256), 256, 0, st>>>(xs, nrhs, c->n, P, t->ncols_pad, t->kpad_agg, t->b_agg);
  cudaMemsetAsync(t->c_agg, 0, (size_t)2 * ns * t->ncols_pad * 4, st);
  cudaMemsetAsync(t->c_dis, 0, (size_t)c->n * t->ncols_pad * 4, st);
  launch_gemm(t->map_a_agg, t->map_b_agg, 2 * ns, ncols, t->ncols_pad, t->kpad_agg, t->c_agg, t->d_err, st);
  const long long threads = (long long)ns * nrhs * 32;
  k_node_stage_tc<<<(int)((threads + 255) / 256), 256, 0, st>>>(ns, P, nrhs, t->c_agg, t->ncols_pad, c->d_fagg,
                                                               c->d_refl, c->d_udis, t->ncols_pad, t->kpad_dis, t->b_dis);
  launch_gemm(t->map_a_dis, t->map_b_dis, c->n, ncols, t->ncols_pad, t->kpad_dis, t->c_dis, t->d_err, st);
  return check_cuda(c, "reflection_mixed");
}

// alpha += the disaggregated reflected coupling of the last reflection_mixed_stage.
void reflection_mixed_add(lsms_ctx* c, int nrhs, double2* alpha, cudaStream_t st) {
  TcState* t = (TcState*)c->tc;
  const int P = c->P;
  k_c_add_alpha<<<grid_for((long long)nrhs * c->n * P, 256), 256, 0, st>>>(t->c_dis, t->ncols_pad, c->n, P, nrhs, alpha);
}

int reflection_mixed(lsms_ctx* c, int nrhs, const double2* xs, double2* alpha, cudaStream_t st) {
  int rc;
  if ((rc = reflection_mixed_stage(c, nrhs, xs, st))) return rc;
  reflection_mixed_add(c, nrhs, alpha, st);
  return check_cuda(c, "reflection_mixed");
}
