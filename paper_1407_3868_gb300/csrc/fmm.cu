// Translation with the far field compressed by boxes (the FMM acceleration of Sec. 3.2; the
// multipole shifts of Sec. 5.3), for long layouts of many discs.
//
// The discs are grouped into boxes of width w along x (centres C_i = (x0 + (i + 1/2) w, -d/2) in
// the disc layer).  Pairs in the same or adjacent boxes are translated directly (Lemma 3.1, FP64,
// as the all-pairs kernel).  For boxes two or more apart:
//   M2M  B_i(q) = sum_{m in box i} sum_n J_{q-n}(k r_m) e^{-i (q-n) phi_m} beta^m_n     (Graf, H -> H)
//   M2L  A_i(nu) = sum_{|i-j| >= 2} sum_q H_{q-nu}(k |i-j| w) e^{i (q-nu) phi_ij} B_j(q) (Lemma 3.1)
//   L2L  alpha^l_nu += sum_q J_{q-nu}(k r_l) e^{i (q-nu) phi_l} A_{box(l)}(q)           (Graf, J -> J)
// with (r_m, phi_m) the polar offset of disc m from its box centre, |q|, |nu| <= Q, and
// phi_ij = 0 (i > j) or pi (i < j).  On the regular grid of box centres the M2L kernel depends only
// on the box offset i - j and the order difference q - nu, so the M2L step is one two-dimensional
// convolution (box index x order), done as a cyclic convolution with cuFFT on an n1 x n2 grid
// (n1 >= 2 nb - 1, n2 >= 6Q + 1: no wrap-around reaches the outputs).  An FFT spreads its rounding
// over all outputs in proportion to the largest kernel entry, and H_s(z) grows fast once |s| > z,
// so offsets with k |d| w < 2Q + 2 (where orders up to 2Q leave the oscillatory range) are
// translated box by box instead and left out of the FFT kernel.  The Graf shift tables
// J_s(k r_m) e^{i s phi_m}, |s| <= Q + p, and the transformed box kernel are built once per layout.
#include <cufft.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <numeric>
#include <vector>

#include "c64.cuh"
#include "ff_hankel.cuh"
#include "lsms_internal.h"
#include "lsms_ops.h"

namespace {

constexpr int FW = 4;     // target discs (warps) per CTA of the near-field kernel
constexpr int FCH = 32;   // source discs per staged chunk
constexpr int FHS = 65;   // pair sequence stride (4p + 1 <= 61)

// FP32 complex helpers (the FP64 ones come from c64.cuh) and loads of either precision
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 c) {
  c.x = fmaf(a.x, b.x, c.x);
  c.x = fmaf(-a.y, b.y, c.x);
  c.y = fmaf(a.x, b.y, c.y);
  c.y = fmaf(a.y, b.x, c.y);
  return c;
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C cconj(C a) { C r = a; r.y = -r.y; return r; }
template <typename C> __device__ __forceinline__ C czero() { C r; r.x = 0; r.y = 0; return r; }
template <typename C> __device__ __forceinline__ C from_d2(double2 v) { C r; r.x = v.x; r.y = v.y; return r; }

// smallest n >= m whose prime factors are 2, 3, 5, 7 (sizes cuFFT handles fastest)
int fft_size(int m) {
  for (int n = std::max(m, 1);; ++n) {
    int r = n;
    for (int f : {2, 3, 5, 7})
      while (r % f == 0) r /= f;
    if (r == 1) return n;
  }
}

// T_m[s + S] = J_s(k r_m) e^{i s phi_m}, s = -S..S, for every disc (thread per entry).
__global__ void k_fmm_shift_table(const double* __restrict__ cx, const double* __restrict__ cy,
                                  const int* __restrict__ dbox, int n, double x0, double w, double yc,
                                  double k, int S, double2* __restrict__ tab) {
  const long long W = 2LL * S + 1;
  const long long total = (long long)n * W;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int m = (int)(i / W);
    const int s = (int)(i - (long long)m * W) - S;
    const double dx = cx[m] - (x0 + (dbox[m] + 0.5) * w), dy = cy[m] - yc;
    const double r = hypot(dx, dy), ph = atan2(dy, dx);
    const int as = s < 0 ? -s : s;
    double j = (r > 0.0) ? jn(as, k * r) : (as == 0 ? 1.0 : 0.0);
    if (s < 0 && (as & 1)) j = -j;                   // J_{-s} = (-1)^s J_s
    double sn, cs;
    sincos(s * ph, &sn, &cs);
    tab[i] = make_double2(j * cs, j * sn);
  }
}

// Box kernel on the cyclic grid: G[d mod n1][s mod n2] = H_s(k |d| w) e^{i s phi_d} for
// dmin <= |d| <= nb - 1, |s| <= 2Q (phi_d = 0 for d > 0, pi for d < 0); zero elsewhere.  One thread
// per offset: H_0, H_1 from the CUDA library, forward recurrence (the arguments are >= 2 k w).
__global__ void k_fmm_box_kernel(int nb, int Q, double k, double w, int n1, int n2, int dmin,
                                 double2* __restrict__ grid) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int nd = 2 * (nb - 1) + 1;
  if (t >= nd) return;
  const int d = t - (nb - 1);
  const int ad = d < 0 ? -d : d;
  if (ad < dmin) return;
  const double z = k * ad * w;
  const int row = ((d % n1) + n1) % n1;
  double2* g = grid + (size_t)row * n2;
  double2 hm = make_double2(j0(z), y0(z)), hq = make_double2(j1(z), y1(z));
  const double sg = d < 0 ? -1.0 : 1.0;              // e^{i s pi} = (-1)^s for d < 0
  g[0] = hm;
  for (int s = 1; s <= 2 * Q; ++s) {
    const double f = (s & 1) ? sg : 1.0;
    g[s] = make_double2(f * hq.x, f * hq.y);                                   // H_s e^{i s phi}
    const double fn = (s & 1) ? -f : f;                                        // H_{-s} = (-1)^s H_s
    g[n2 - s] = make_double2(fn * hq.x, fn * hq.y);
    if (s < 2 * Q) {
      const double c = 2.0 * s / z;
      const double2 hn = make_double2(c * hq.x - hm.x, c * hq.y - hm.y);
      hm = hq;
      hq = hn;
    }
  }
}

__global__ void k_fmm_scale(double2* __restrict__ a, long long total, double s) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x)
    a[i] = make_double2(a[i].x * s, a[i].y * s);
}

template <typename C>
__global__ void k_fmm_mul(C* __restrict__ a, const C* __restrict__ b, long long total) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x)
    a[i] = cmul(a[i], b[i]);
}

// M2M: one CTA per box, thread t <-> box order q = t - Q; writes grid[i][(-q) mod n2].  C is the
// complex type of the tables and the grid (double2, or float2 in mixed precision).
template <typename C>
__global__ void k_fmm_m2m(const double2* __restrict__ xs, const int* __restrict__ perm,
                          const int* __restrict__ bstart, const C* __restrict__ tab, int p,
                          int Q, int S, int n2, C* __restrict__ grid, C* __restrict__ bq) {
  extern __shared__ unsigned char sraw[];
  C* sbeta = reinterpret_cast<C*>(sraw);             // [P] coefficients of the current disc
  const int i = blockIdx.x, P = 2 * p + 1;
  const int q = (int)threadIdx.x - Q;
  C acc = czero<C>();
  for (int jj = bstart[i]; jj < bstart[i + 1]; ++jj) {
    const int m = perm[jj];
    __syncthreads();
    if (threadIdx.x < P) sbeta[threadIdx.x] = from_d2<C>(xs[(size_t)m * P + threadIdx.x]);
    __syncthreads();
    if (q >= -Q && q <= Q) {
      const C* t = tab + (size_t)m * (2 * S + 1) + S + q + p;           // t[-(n + p)] <-> s = q - n
      for (int a = 0; a < P; ++a) acc = cfma(cconj(t[-a]), sbeta[a], acc);   // J_{q-n} e^{-i (q-n) phi}
    }
  }
  if (q >= -Q && q <= Q) {
    grid[(size_t)i * n2 + ((-q) % n2 + n2) % n2] = acc;
    bq[(size_t)i * (2 * Q + 1) + q + Q] = acc;
  }
}

// M2L for the offsets 2 <= |d| < dmin, box by box: grid[i][(-nu) mod n2] += sum_d sum_q
// hd[d][q - nu] B_{i-d}(q), hd[(sign, |d| - 2)][s + 2Q] = H_s(k |d| w) e^{i s phi_d}.
template <typename C>
__global__ void k_fmm_m2l_direct(const C* __restrict__ bq, const C* __restrict__ hd, int nb,
                                 int Q, int dmin, int n2, C* __restrict__ grid) {
  const int i = blockIdx.x;
  const int nu = (int)threadIdx.x - Q;
  if (nu < -Q || nu > Q) return;
  const int W = 2 * Q + 1, H = 4 * Q + 1;
  C acc = czero<C>();
  for (int ad = 2; ad < dmin; ++ad)
    for (int sg = 0; sg < 2; ++sg) {
      const int d = sg ? -ad : ad;
      const int j = i - d;
      if (j < 0 || j >= nb) continue;
      const C* h = hd + (size_t)(2 * (ad - 2) + sg) * H + 2 * Q - nu;   // h[q] <-> s = q - nu
      const C* b = bq + (size_t)j * W + Q;
      for (int q = -Q; q <= Q; ++q) acc = cfma(h[q], b[q], acc);
    }
  C* g = grid + (size_t)i * n2 + ((-nu) % n2 + n2) % n2;
  *g = cadd(*g, acc);
}

// Direct-offset kernels hd[(sign, |d| - 2)][s + 2Q], 2 <= |d| < dmin (one thread per offset).
__global__ void k_fmm_direct_table(int Q, double k, double w, int dmin, double2* __restrict__ hd) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * (dmin - 2)) return;
  const int ad = 2 + t / 2, sg = t & 1;
  const double z = k * ad * w;
  const double sgn = sg ? -1.0 : 1.0;
  double2* h = hd + (size_t)t * (4 * Q + 1) + 2 * Q;
  double2 hm = make_double2(j0(z), y0(z)), hq = make_double2(j1(z), y1(z));
  h[0] = hm;
  for (int s = 1; s <= 2 * Q; ++s) {
    const double f = (s & 1) ? sgn : 1.0;
    h[s] = make_double2(f * hq.x, f * hq.y);
    const double fn = (s & 1) ? -f : f;
    h[-s] = make_double2(fn * hq.x, fn * hq.y);
    if (s < 2 * Q) {
      const double c = 2.0 * s / z;
      const double2 hn = make_double2(c * hq.x - hm.x, c * hq.y - hm.y);
      hm = hq;
      hq = hn;
    }
  }
}

// L2L: one warp per disc, lane <-> nu; alpha = sum_q T_l[q - nu] A_box(q), A(q) = grid[b][(-q) mod n2].
template <typename C>
__global__ void k_fmm_l2l(const C* __restrict__ grid, const int* __restrict__ dbox,
                          const C* __restrict__ tab, int n, int p, int Q, int S, int n2,
                          double2* __restrict__ alpha) {
  const int l = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  const int P = 2 * p + 1;
  if (l >= n || lane >= P) return;
  const int nu = lane - p;
  const C* g = grid + (size_t)dbox[l] * n2;
  const C* t = tab + (size_t)l * (2 * S + 1) + S;
  C acc = czero<C>();
  for (int q = -Q; q <= Q; ++q) acc = cfma(t[q - nu], g[((-q) % n2 + n2) % n2], acc);
  alpha[(size_t)l * P + lane] = make_double2(acc.x, acc.y);
}

// Near field: CTA over FW consecutive targets in box order; sources from the neighbouring boxes,
// staged in chunks; alpha += (pairs in the same or adjacent boxes), as the all-pairs FP64 kernel.
__global__ void __launch_bounds__(FW * 32, 1)
k_fmm_near(const double* __restrict__ scx, const double* __restrict__ scy, const int* __restrict__ perm,
           const int* __restrict__ sbox, const int* __restrict__ bstart, int n, int nb, int p, double k,
           const double2* __restrict__ xs, double2* __restrict__ alpha) {
  extern __shared__ double2 smem[];
  double2* sb = smem;                                 // [FCH][32]
  double* sbs = (double*)(sb + FCH * 32);             // [FCH][32]
  double2* sh = (double2*)(sbs + FCH * 32);           // [FW][FCH][FHS]
  double* shs = (double*)(sh + FW * FCH * FHS);       // [FW][FCH][FHS]
  __shared__ double cxs[FCH], cys[FCH];
  __shared__ int bxs[FCH], ids[FCH];
  const int P = 2 * p + 1;
  const int r = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t0 = blockIdx.x * FW;
  const int t = t0 + warp;                            // sorted target index
  const bool tvalid = t < n;
  const int l = tvalid ? perm[t] : -1;
  const int bl = tvalid ? sbox[t] : 0;
  const double xl = tvalid ? scx[t] : 0.0, yl = tvalid ? scy[t] : 0.0;
  const int blo = sbox[t0], bhi = sbox[min(t0 + FW, n) - 1];
  const int j_beg = bstart[max(blo - 1, 0)], j_end = bstart[min(bhi + 2, nb)];
  const double2* xr = xs + (size_t)r * n * P;
  double2* hw = sh + (size_t)warp * FCH * FHS;
  double* hsw = shs + (size_t)warp * FCH * FHS;
  double A = 0.0, B = 0.0, C = 0.0;
  for (int j0c = j_beg; j0c < j_end; j0c += FCH) {
    const int cnt = min(FCH, j_end - j0c);
    __syncthreads();
    if (threadIdx.x < cnt) {
      cxs[threadIdx.x] = scx[j0c + threadIdx.x];
      cys[threadIdx.x] = scy[j0c + threadIdx.x];
      bxs[threadIdx.x] = sbox[j0c + threadIdx.x];
      ids[threadIdx.x] = perm[j0c + threadIdx.x];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < cnt * P; i += blockDim.x) {
      const int s = i / P, q = i - s * P;
      const double2 v = xr[(size_t)ids[s] * P + q];
      sb[s * 32 + q] = v;
      sbs[s * 32 + q] = v.x + v.y;
    }
    if (lane < cnt) {
      double2* h = hw + lane * FHS;
      double* hsm = hsw + lane * FHS;
      const int db = bxs[lane] - bl;
      if (tvalid && ids[lane] != l && db >= -1 && db <= 1) {
        hankel_sequence_f64(xl - cxs[lane], yl - cys[lane], k, p, h, hsm);
      } else {
        for (int q = 0; q <= 4 * p; ++q) {
          h[q] = make_double2(0.0, 0.0);
          hsm[q] = 0.0;
        }
      }
    }
    __syncthreads();
    if (tvalid && lane < P) {
      for (int s = 0; s < cnt; ++s) {
        const double2* hs = hw + s * FHS + 2 * p - lane;
        const double* hss = hsw + s * FHS + 2 * p - lane;
        const double2* bs = sb + s * 32;
        const double* bss = sbs + s * 32;
        for (int q = 0; q < P; ++q) {
          const double2 hv = hs[q], bv = bs[q];
          A = fma(hv.x, bv.x, A);
          B = fma(hv.y, bv.y, B);
          C = fma(hss[q], bss[q], C);
        }
      }
    }
  }
  if (tvalid && lane < P) {
    double2* o = alpha + (size_t)r * n * P + (size_t)l * P + lane;
    *o = make_double2(o->x + (A - B), o->y + (C - A - B));
  }
}

// ---------------------------------------------------------------------------------------------
// Mixed precision: the near field in FP32 (float-float phases, Hankel's asymptotic H_0, H_1 for
// k rho >= 25, forward recurrence) with the register-blocked Toeplitz contraction of the all-pairs
// FP32 kernel, restricted to adjacent boxes; pairs with k rho < 25 are left to the near-pair kernel
// (FP64-accurate sequences).  Inputs and outputs in box order.
// ---------------------------------------------------------------------------------------------
constexpr int BW = 1;      // warps per CTA: each warp's 8 targets (about one box) get their own
                           // source window, three to four boxes wide instead of a 32-target CTA's six
constexpr int BT = 8;      // target discs per warp
constexpr int BCH = 32;    // sources staged per chunk
constexpr int BHS = 65;    // pair slot stride (see the all-pairs FP32 kernel: conflict-free windows)
constexpr int BGUARD = 8;
constexpr size_t BOX_NEAR_SMEM = (size_t)(2 * BGUARD + BW * 32 * BHS) * sizeof(float2);

template <int PT>
__global__ void __launch_bounds__(BW * 32, 8)
k_box_near_f32(const float4* __restrict__ cff, const int* __restrict__ sbox, const int* __restrict__ bstart,
               int nb, int n, float k_hi, float k_lo, float near_hi, float near_lo,
               const float2* __restrict__ xs, float2* __restrict__ out) {
  constexpr int p = PT;
  constexpr int P = 2 * PT + 1;
  constexpr int VB = (P + 3) / 4;
  constexpr int NB = (P + VB - 1) / VB;
  __shared__ float2 sb[BCH][VB * NB + 1];
  __shared__ float4 sc[BCH];
  __shared__ int sbx[BCH];
  extern __shared__ float2 sh[];
  const int r = blockIdx.z;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = lane & 7, hi8 = lane >> 3;
  const int l0 = blockIdx.x * BW * BT;
  const int l = l0 + warp * BT + t;
  const bool lvalid = l < n;
  const float4 ct = lvalid ? cff[l] : make_float4(0.f, 0.f, 0.f, 0.f);
  const int bl = lvalid ? sbox[l] : 0;
  const int b0 = sbox[l0], b1 = sbox[min(l0 + BW * BT, n) - 1];
  const int jbeg = bstart[max(b0 - 1, 0)], jend = bstart[min(b1 + 2, nb)];
  for (int i = threadIdx.x; i < 2 * BGUARD + BW * 32 * BHS; i += blockDim.x) sh[i] = make_float2(0.f, 0.f);
  float2* hw = sh + BGUARD + warp * 32 * BHS;
  float2 AB[VB];           // (sum h_r b_r, sum h_i b_i), one packed FMA per window value
  float C[VB];
#pragma unroll
  for (int i = 0; i < VB; ++i) {
    AB[i] = make_float2(0.f, 0.f);
    C[i] = 0.f;
  }
  const ffl kf = {k_hi, k_lo};
  const float2* xr = xs + (size_t)r * n * P;
  for (int j0c = jbeg; j0c < jend; j0c += BCH) {
    const int cnt = min(BCH, jend - j0c);
    __syncthreads();
    for (int i = threadIdx.x; i < BCH * VB * NB; i += blockDim.x) {
      const int s = i / (VB * NB), q = i - s * (VB * NB);
      sb[s][q] = (s < cnt && q < P) ? xr[(size_t)(j0c + s) * P + q] : make_float2(0.f, 0.f);
    }
    if (threadIdx.x < cnt) {
      sc[threadIdx.x] = cff[j0c + threadIdx.x];
      sbx[threadIdx.x] = sbox[j0c + threadIdx.x];
    }
    __syncthreads();
    for (int s0 = 0; s0 < cnt; s0 += 4) {
      {
        const int js = s0 + hi8;
        float2* h = hw + lane * BHS;
        const int db = js < cnt ? sbx[js] - bl : 2;
        if (js < cnt && lvalid && j0c + js != l && db >= -1 && db <= 1) {
          hankel_sequence_f32<PT>(ct, sc[js], kf, {near_hi, near_lo}, h);
        } else {
          for (int q = 0; q <= 4 * p; ++q) h[q] = make_float2(0.f, 0.f);
        }
      }
      __syncwarp();
      const int nq4 = min(4, cnt - s0);
      for (int q4 = 0; q4 < nq4; ++q4) {
        const float2* hs = hw + (q4 * 8 + t) * BHS + 2 * p - VB * hi8;
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
            const float2 bv = sb[s0 + q4][nbk * VB + u];
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
      __syncwarp();
    }
  }
  if (lvalid) {
    float2* o = out + ((size_t)r * n + l) * P;
#pragma unroll
    for (int i = 0; i < VB; ++i) {
      const int nu = VB * hi8 + i;
      if (nu < P) o[nu] = make_float2(AB[i].x - AB[i].y, C[i] - AB[i].x - AB[i].y);
    }
  }
}

template <int PT>
void launch_box_near_pt(dim3 grid, cudaStream_t st, const float4* cff, const int* sbox, const int* bstart, int nb,
                        int n, float kh, float kl, float nh, float nl, const float2* xs, float2* out) {
  static std::once_flag attr;
  std::call_once(attr, [] {
    cudaFuncSetAttribute(k_box_near_f32<PT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BOX_NEAR_SMEM);
  });
  k_box_near_f32<PT><<<grid, BW * 32, BOX_NEAR_SMEM, st>>>(cff, sbox, bstart, nb, n, kh, kl, nh, nl, xs, out);
}

void launch_box_near(int p, dim3 grid, cudaStream_t st, const float4* cff, const int* sbox, const int* bstart,
                     int nb, int n, float kh, float kl, float nh, float nl, const float2* xs, float2* out) {
#define LSMS_BN(PT) launch_box_near_pt<PT>(grid, st, cff, sbox, bstart, nb, n, kh, kl, nh, nl, xs, out)
  switch (p) {
    case 0: LSMS_BN(0); break;
    case 1: LSMS_BN(1); break;
    case 2: LSMS_BN(2); break;
    case 3: LSMS_BN(3); break;
    case 4: LSMS_BN(4); break;
    case 5: LSMS_BN(5); break;
    case 6: LSMS_BN(6); break;
    case 7: LSMS_BN(7); break;
    case 8: LSMS_BN(8); break;
    case 9: LSMS_BN(9); break;
    case 10: LSMS_BN(10); break;
    case 11: LSMS_BN(11); break;
    case 12: LSMS_BN(12); break;
    case 13: LSMS_BN(13); break;
    case 14: LSMS_BN(14); break;
    default: LSMS_BN(15); break;
  }
#undef LSMS_BN
}

// FP32 copies of the coefficients in both orders: x32 (disc order), xs32 (box order).
__global__ void k_fmm_to_f32(const double2* __restrict__ x, const int* __restrict__ perm, int n, int P,
                             long long len, float2* __restrict__ x32, float2* __restrict__ xs32) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len;
       i += (long long)gridDim.x * blockDim.x) {
    const long long rt = i / P;
    const int q = (int)(i - rt * P);
    const long long r = rt / n;
    const int tt = (int)(rt - r * n);
    const double2 v = x[i];
    x32[i] = make_float2((float)v.x, (float)v.y);
    const double2 w = x[((size_t)r * n + perm[tt]) * P + q];
    xs32[i] = make_float2((float)w.x, (float)w.y);
  }
}

// alpha[r][perm[t]][nu] += part[r][t][nu]
__global__ void k_fmm_scatter_add(const float2* __restrict__ part, const int* __restrict__ perm, int n, int P,
                                  long long len, double2* __restrict__ alpha) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len;
       i += (long long)gridDim.x * blockDim.x) {
    const long long rt = i / P;
    const int q = (int)(i - rt * P);
    const long long r = rt / n;
    const int tt = (int)(rt - r * n);
    double2* o = alpha + ((size_t)r * n + perm[tt]) * P + q;
    const float2 v = part[i];
    *o = make_double2(o->x + v.x, o->y + v.y);
  }
}

__global__ void k_fmm_d2f(const double2* __restrict__ a, float2* __restrict__ b, long long total) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x)
    b[i] = make_float2((float)a[i].x, (float)a[i].y);
}

__global__ void k_fmm_ff_centres(const double* __restrict__ cx, const double* __restrict__ cy, int n,
                                 float4* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const float xh = (float)cx[j], yh = (float)cy[j];
  out[j] = make_float4(xh, (float)(cx[j] - (double)xh), yh, (float)(cy[j] - (double)yh));
}

inline int blocks_for(long long total, int block) {
  long long b = (total + block - 1) / block;
  return (int)std::min<long long>(std::max<long long>(b, 1), 152LL * 32);
}

}  // namespace

void fmm_free(lsms_ctx* c) {
  FmmState& f = c->fmm;
  void* ptrs[] = {f.d_perm, f.d_bstart, f.d_dbox, f.d_sbox, f.d_scx, f.d_scy, f.d_tab, f.d_khat, f.d_grid,
                  f.d_bq, f.d_hd, f.d_scff, f.ws.ptr, f.d_tab32, f.d_khat32, f.d_grid32, f.d_bq32, f.d_hd32};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  if (f.has_plan) cufftDestroy((cufftHandle)f.plan);
  if (f.has_plan32) cufftDestroy((cufftHandle)f.plan32);
  for (cudaEvent_t e : f.ev)
    if (e) cudaEventDestroy(e);
  const double w = f.box_width;
  const int order = f.order_req;
  f = FmmState();
  f.box_width = w;
  f.order_req = order;
}

// Box tables of the current layout (host grouping; device shift tables and transformed kernel).
int fmm_setup(lsms_ctx* c) {
  FmmState& f = c->fmm;
  fmm_free(c);
  if (!(f.box_width > 0.0) || c->n <= 0) return LSMS_OK;
  const int n = c->n, p = c->p;
  const double w = f.box_width;
  const double rb = std::hypot(0.5 * w, 0.5 * c->d);
  f.order = f.order_req > 0 ? f.order_req : (int)std::ceil(c->k2 * rb) + 32;
  f.S = f.order + p;
  // the device centres are x - xc (layout midpoint) and y in the disc layer's frame
  std::vector<double> x(n);
  for (int j = 0; j < n; ++j) x[j] = c->cx[j] - c->xc;
  f.x0 = *std::min_element(x.begin(), x.end());
  std::vector<int> dbox(n);
  int nb = 0;
  for (int j = 0; j < n; ++j) {
    dbox[j] = (int)std::floor((x[j] - f.x0) / w);
    nb = std::max(nb, dbox[j] + 1);
  }
  f.nb = nb;
  std::vector<int> perm(n);
  std::iota(perm.begin(), perm.end(), 0);
  std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) { return dbox[a] < dbox[b]; });
  std::vector<int> bstart(nb + 1, 0), sbox(n);
  for (int j = 0; j < n; ++j) ++bstart[dbox[j] + 1];
  for (int i = 0; i < nb; ++i) bstart[i + 1] += bstart[i];
  f.near_pairs = 0;
  for (int b = 0; b < nb; ++b) {
    const long long own = bstart[b + 1] - bstart[b];
    const long long nbr = bstart[std::min(b + 2, nb)] - bstart[std::max(b - 1, 0)];
    f.near_pairs += own * (nbr - 1);
  }
  std::vector<double> scx(n), scy(n);
  for (int t = 0; t < n; ++t) {
    sbox[t] = dbox[perm[t]];
    scx[t] = x[perm[t]];
    scy[t] = c->cy[perm[t]];
  }
  // offsets below dmin go box by box (k |d| w < 2Q + 2)
  f.dmin = 2;
  while (c->k2 * f.dmin * w < 2.0 * f.order + 2.0) ++f.dmin;
  f.far = nb >= 3;                 // boxes two apart exist only from three boxes on
  f.n1 = f.far ? fft_size(2 * nb - 1) : 1;
  f.n2 = fft_size(6 * f.order + 1);
  const size_t gsz = (size_t)f.n1 * f.n2;
  const size_t tsz = (size_t)n * (2 * f.S + 1);
  if (cudaMalloc((void**)&f.d_perm, n * sizeof(int)) != cudaSuccess ||
      cudaMalloc((void**)&f.d_bstart, (nb + 1) * sizeof(int)) != cudaSuccess ||
      cudaMalloc((void**)&f.d_dbox, n * sizeof(int)) != cudaSuccess ||
      cudaMalloc((void**)&f.d_sbox, n * sizeof(int)) != cudaSuccess ||
      cudaMalloc((void**)&f.d_scx, n * sizeof(double)) != cudaSuccess ||
      cudaMalloc((void**)&f.d_scy, n * sizeof(double)) != cudaSuccess ||
      cudaMalloc((void**)&f.d_tab, tsz * sizeof(double2)) != cudaSuccess ||
      cudaMalloc((void**)&f.d_khat, gsz * sizeof(double2)) != cudaSuccess ||
      cudaMalloc((void**)&f.d_grid, gsz * sizeof(double2)) != cudaSuccess ||
      cudaMalloc((void**)&f.d_bq, (size_t)nb * (2 * f.order + 1) * sizeof(double2)) != cudaSuccess ||
      cudaMalloc((void**)&f.d_scff, (size_t)n * sizeof(float4)) != cudaSuccess ||
      cudaMalloc((void**)&f.d_hd, (size_t)std::max(1, 2 * (f.dmin - 2)) * (4 * f.order + 1) * sizeof(double2)) !=
          cudaSuccess) {
    cudaGetLastError();
    fmm_free(c);
    return ctx_fail(c, LSMS_ERR_OOM, "set_fmm: cudaMalloc failed for the box tables");
  }
  cudaMemcpy(f.d_perm, perm.data(), n * sizeof(int), cudaMemcpyHostToDevice);
  cudaMemcpy(f.d_bstart, bstart.data(), (nb + 1) * sizeof(int), cudaMemcpyHostToDevice);
  cudaMemcpy(f.d_dbox, dbox.data(), n * sizeof(int), cudaMemcpyHostToDevice);
  cudaMemcpy(f.d_sbox, sbox.data(), n * sizeof(int), cudaMemcpyHostToDevice);
  cudaMemcpy(f.d_scx, scx.data(), n * sizeof(double), cudaMemcpyHostToDevice);
  cudaMemcpy(f.d_scy, scy.data(), n * sizeof(double), cudaMemcpyHostToDevice);
  cudaStream_t st = c->stream;
  k_fmm_ff_centres<<<(n + 255) / 256, 256, 0, st>>>(f.d_scx, f.d_scy, n, f.d_scff);
  if (!f.far) {                    // near field only
    cudaStreamSynchronize(st);
    f.ready = true;
    return check_cuda(c, "set_fmm");
  }
  cufftHandle plan;
  if (cufftPlan2d(&plan, f.n1, f.n2, CUFFT_Z2Z) != CUFFT_SUCCESS) {
    fmm_free(c);
    return ctx_fail(c, LSMS_ERR_CUDA, "set_fmm: cuFFT plan creation failed");
  }
  f.plan = (int)plan;
  f.has_plan = true;
  k_fmm_shift_table<<<blocks_for((long long)tsz, 256), 256, 0, st>>>(c->d_cx, c->d_cy, f.d_dbox, n, f.x0, w,
                                                                      -0.5 * c->d, c->k2, f.S, f.d_tab);
  cudaMemsetAsync(f.d_khat, 0, gsz * sizeof(double2), st);
  const int nd = 2 * (nb - 1) + 1;
  k_fmm_box_kernel<<<(nd + 127) / 128, 128, 0, st>>>(nb, f.order, c->k2, w, f.n1, f.n2, f.dmin, f.d_khat);
  if (f.dmin > 2) k_fmm_direct_table<<<(2 * (f.dmin - 2) + 63) / 64, 64, 0, st>>>(f.order, c->k2, w, f.dmin, f.d_hd);
  cufftSetStream(plan, st);
  if (cufftExecZ2Z(plan, (cufftDoubleComplex*)f.d_khat, (cufftDoubleComplex*)f.d_khat, CUFFT_FORWARD) !=
      CUFFT_SUCCESS) {
    fmm_free(c);
    return ctx_fail(c, LSMS_ERR_CUDA, "set_fmm: cuFFT failed");
  }
  k_fmm_scale<<<blocks_for((long long)gsz, 256), 256, 0, st>>>(f.d_khat, (long long)gsz, 1.0 / (double)gsz);
  // FP32 copies for the mixed-precision far field
  const size_t hsz = (size_t)std::max(1, 2 * (f.dmin - 2)) * (4 * f.order + 1);
  if (cudaMalloc((void**)&f.d_tab32, tsz * sizeof(float2)) != cudaSuccess ||
      cudaMalloc((void**)&f.d_khat32, gsz * sizeof(float2)) != cudaSuccess ||
      cudaMalloc((void**)&f.d_grid32, gsz * sizeof(float2)) != cudaSuccess ||
      cudaMalloc((void**)&f.d_bq32, (size_t)nb * (2 * f.order + 1) * sizeof(float2)) != cudaSuccess ||
      cudaMalloc((void**)&f.d_hd32, hsz * sizeof(float2)) != cudaSuccess) {
    cudaGetLastError();
    fmm_free(c);
    return ctx_fail(c, LSMS_ERR_OOM, "set_fmm: cudaMalloc failed for the FP32 box tables");
  }
  k_fmm_d2f<<<blocks_for((long long)tsz, 256), 256, 0, st>>>(f.d_tab, f.d_tab32, (long long)tsz);
  k_fmm_d2f<<<blocks_for((long long)gsz, 256), 256, 0, st>>>(f.d_khat, f.d_khat32, (long long)gsz);
  if (f.dmin > 2) k_fmm_d2f<<<blocks_for((long long)hsz, 256), 256, 0, st>>>(f.d_hd, f.d_hd32, (long long)hsz);
  cufftHandle plan32;
  if (cufftPlan2d(&plan32, f.n1, f.n2, CUFFT_C2C) != CUFFT_SUCCESS) {
    fmm_free(c);
    return ctx_fail(c, LSMS_ERR_CUDA, "set_fmm: cuFFT plan creation failed");
  }
  f.plan32 = (int)plan32;
  f.has_plan32 = true;
  cudaStreamSynchronize(st);
  f.ready = true;
  return check_cuda(c, "set_fmm");
}

// alpha = T xs for nrhs right-hand sides through the box method (FP64).  Launches: per right-hand
// side M2M, the pointwise product and L2L, plus one near-field launch (cuFFT's own kernels aside).
int fmm_translate(lsms_ctx* c, int nrhs, const double2* xs, double2* alpha, bool mixed, cudaStream_t st) {
  FmmState& f = c->fmm;
  const int n = c->n, p = c->p, P = 2 * p + 1;
  if (!f.ready) return ctx_fail(c, LSMS_ERR_STATE, "box translation tables are not built");
  const size_t gsz = (size_t)f.n1 * f.n2;
  cufftHandle plan = (cufftHandle)f.plan;
  cufftSetStream(plan, st);
  const bool timed = c->timing && !c->kids.size();
  if (timed && !f.ev[0])
    for (cudaEvent_t& e : f.ev) cudaEventCreate(&e);
  if (timed) cudaEventRecord(f.ev[0], st);
  const int qthreads = ((2 * f.order + 1 + 31) / 32) * 32;
  if (!f.far) cudaMemsetAsync(alpha, 0, (size_t)nrhs * n * P * sizeof(double2), st);
  for (int r = 0; r < nrhs && f.far; ++r) {
    const double2* x = xs + (size_t)r * n * P;
    double2* a = alpha + (size_t)r * n * P;
    if (mixed) {
      cufftHandle p32 = (cufftHandle)f.plan32;
      cufftSetStream(p32, st);
      cudaMemsetAsync(f.d_grid32, 0, gsz * sizeof(float2), st);
      k_fmm_m2m<float2><<<f.nb, qthreads, P * sizeof(float2), st>>>(x, f.d_perm, f.d_bstart, f.d_tab32, p, f.order,
                                                                    f.S, f.n2, f.d_grid32, f.d_bq32);
      if (cufftExecC2C(p32, (cufftComplex*)f.d_grid32, (cufftComplex*)f.d_grid32, CUFFT_FORWARD) != CUFFT_SUCCESS)
        return ctx_fail(c, LSMS_ERR_CUDA, "box translation: cuFFT failed");
      k_fmm_mul<float2><<<blocks_for((long long)gsz, 256), 256, 0, st>>>(f.d_grid32, f.d_khat32, (long long)gsz);
      if (cufftExecC2C(p32, (cufftComplex*)f.d_grid32, (cufftComplex*)f.d_grid32, CUFFT_INVERSE) != CUFFT_SUCCESS)
        return ctx_fail(c, LSMS_ERR_CUDA, "box translation: cuFFT failed");
      if (f.dmin > 2)
        k_fmm_m2l_direct<float2><<<f.nb, qthreads, 0, st>>>(f.d_bq32, f.d_hd32, f.nb, f.order, f.dmin, f.n2,
                                                            f.d_grid32);
      k_fmm_l2l<float2><<<(int)(((long long)n * 32 + 255) / 256), 256, 0, st>>>(f.d_grid32, f.d_dbox, f.d_tab32, n, p,
                                                                                f.order, f.S, f.n2, a);
      continue;
    }
    cudaMemsetAsync(f.d_grid, 0, gsz * sizeof(double2), st);
    k_fmm_m2m<double2><<<f.nb, qthreads, P * sizeof(double2), st>>>(x, f.d_perm, f.d_bstart, f.d_tab, p, f.order,
                                                                     f.S, f.n2, f.d_grid, f.d_bq);
    if (cufftExecZ2Z(plan, (cufftDoubleComplex*)f.d_grid, (cufftDoubleComplex*)f.d_grid, CUFFT_FORWARD) !=
        CUFFT_SUCCESS)
      return ctx_fail(c, LSMS_ERR_CUDA, "box translation: cuFFT failed");
    k_fmm_mul<double2><<<blocks_for((long long)gsz, 256), 256, 0, st>>>(f.d_grid, f.d_khat, (long long)gsz);
    if (cufftExecZ2Z(plan, (cufftDoubleComplex*)f.d_grid, (cufftDoubleComplex*)f.d_grid, CUFFT_INVERSE) !=
        CUFFT_SUCCESS)
      return ctx_fail(c, LSMS_ERR_CUDA, "box translation: cuFFT failed");
    if (f.dmin > 2)
      k_fmm_m2l_direct<double2><<<f.nb, qthreads, 0, st>>>(f.d_bq, f.d_hd, f.nb, f.order, f.dmin, f.n2, f.d_grid);
    k_fmm_l2l<double2><<<(int)(((long long)n * 32 + 255) / 256), 256, 0, st>>>(f.d_grid, f.d_dbox, f.d_tab, n, p,
                                                                                f.order, f.S, f.n2, a);
  }
  if (mixed) {
    // near field in FP32: box-order copies, the adjacent-box kernel, scatter-add, the near pairs
    const long long len = (long long)nrhs * n * P;
    const size_t b = (((size_t)len * sizeof(float2)) + 255) & ~size_t(255);
    int rc;
    if ((rc = ensure(c, f.ws, 3 * b))) return rc;
    float2* x32 = (float2*)f.ws.ptr;
    float2* xs32 = (float2*)((unsigned char*)f.ws.ptr + b);
    float2* part = (float2*)((unsigned char*)f.ws.ptr + 2 * b);
    if (timed) cudaEventRecord(f.ev[1], st);
    k_fmm_to_f32<<<blocks_for(len, 256), 256, 0, st>>>(xs, f.d_perm, n, P, len, x32, xs32);
    const float kh = (float)c->k2, kl = (float)(c->k2 - (double)kh);
    const float nh = (float)c->near_r2, nl = (float)(c->near_r2 - (double)nh);
    dim3 grid((n + BW * BT - 1) / (BW * BT), 1, nrhs);
    launch_box_near(p, grid, st, f.d_scff, f.d_sbox, f.d_bstart, f.nb, n, kh, kl, nh, nl, xs32, part);
    k_fmm_scatter_add<<<blocks_for(len, 256), 256, 0, st>>>(part, f.d_perm, n, P, len, alpha);
    launch_translate_near(c, nrhs, x32, alpha, st);
    if (timed) cudaEventRecord(f.ev[2], st);
    f.timed = timed;
    return LSMS_OK;
  }
  const size_t smem = (size_t)(FCH * 32 + FW * FCH * FHS) * (sizeof(double2) + sizeof(double));
  static std::once_flag attr;
  std::call_once(attr, [smem] {
    cudaFuncSetAttribute(k_fmm_near, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  dim3 grid((n + FW - 1) / FW, nrhs);
  if (timed) cudaEventRecord(f.ev[1], st);
  k_fmm_near<<<grid, FW * 32, smem, st>>>(f.d_scx, f.d_scy, f.d_perm, f.d_sbox, f.d_bstart, n, f.nb, p, c->k2, xs,
                                           alpha);
  if (timed) cudaEventRecord(f.ev[2], st);
  f.timed = timed;
  return LSMS_OK;
}

extern "C" int lsms_set_fmm(lsms_ctx* c, double box_width, int order) {
  if (!c) return LSMS_ERR_ARG;
  if (!std::isfinite(box_width) || order < 0 || order > 400)
    return ctx_fail(c, LSMS_ERR_ARG, "set_fmm: box_width must be finite and 0 <= order <= 400");
  if (box_width > 0.0 && !(box_width >= c->d))
    return ctx_fail(c, LSMS_ERR_ARG, "set_fmm: box_width must be at least the disc layer's thickness");
  if (order > 0 && order < c->p) return ctx_fail(c, LSMS_ERR_ARG, "set_fmm: order must be >= p");
  cudaStreamSynchronize(c->stream);
  batch_clear_graphs(c);
  c->fmm.box_width = box_width > 0.0 ? box_width : 0.0;
  c->fmm.order_req = order;
  for (lsms_ctx* k : c->kids) {
    const int rc = lsms_set_fmm(k, box_width, order);
    if (rc) return ctx_fail(c, rc, std::string("set_fmm: ") + k->err);
  }
  if (c->kids.empty() && c->n >= 0) return fmm_setup(c);
  return LSMS_OK;
}

extern "C" int lsms_set_fmm_scope(lsms_ctx* c, int scope) {
  if (!c) return LSMS_ERR_ARG;
  if (scope != LSMS_FMM_ALL && scope != LSMS_FMM_RESIDUAL)
    return ctx_fail(c, LSMS_ERR_ARG, "set_fmm_scope: LSMS_FMM_ALL or LSMS_FMM_RESIDUAL");
  cudaStreamSynchronize(c->stream);
  batch_clear_graphs(c);
  c->fmm.scope = scope;
  for (lsms_ctx* k : c->kids) k->fmm.scope = scope;
  return LSMS_OK;
}

extern "C" int lsms_fmm_stats(lsms_ctx* c, long long* near_pairs, double* far_ms, double* near_ms) {
  if (!c) return LSMS_ERR_ARG;
  FmmState& f = c->fmm;
  if (near_pairs) *near_pairs = f.ready ? f.near_pairs : 0;
  float a = 0.0f, b = 0.0f;
  if (f.timed && f.ev[2]) {
    if (cudaEventSynchronize(f.ev[2]) != cudaSuccess || cudaEventElapsedTime(&a, f.ev[0], f.ev[1]) != cudaSuccess ||
        cudaEventElapsedTime(&b, f.ev[1], f.ev[2]) != cudaSuccess)
      return check_cuda(c, "fmm_stats");
  }
  if (far_ms) *far_ms = a;
  if (near_ms) *near_ms = b;
  return LSMS_OK;
}

extern "C" int lsms_get_fmm(const lsms_ctx* c, int* n_boxes, int* order) {
  if (!c) return LSMS_ERR_ARG;
  if (n_boxes) *n_boxes = c->fmm.ready ? c->fmm.nb : 0;
  if (order) *order = c->fmm.ready ? c->fmm.order : 0;
  return LSMS_OK;
}
