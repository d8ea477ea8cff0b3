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
// cyclic convolution (box index x order) on an n1 x n2 grid (powers of two, n1 >= 2 nb - 1,
// n2 >= 4Q + 1: no wrap-around reaches the outputs), done with hand-written radix-2 FFTs: along
// the boxes by the four-step split n1 = A B (A-point transforms at stride B, twiddles, B-point
// transforms on contiguous runs, leaving the spectrum in transposed order), which the inverse
// undoes in reverse; along the orders one n2-point transform per frequency row, the product with
// the transformed kernel and the inverse, in one kernel.  Only the 2Q + 1 order columns that hold
// data are transformed along the boxes.  An FFT spreads its rounding over all outputs in
// proportion to the largest kernel entry, and H_s(z) grows fast once |s| > z, so offsets with
// k |d| w < 2Q + 2 (where orders up to 2Q leave the oscillatory range) are translated box by box
// instead and left out of the FFT kernel.  The Graf shift tables J_s(k r_m) e^{i s phi_m},
// |s| <= Q + p, and the transformed box kernel are built once per layout.
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

// Box kernel on the cyclic grid, laid out for a correlation over orders: G[d mod n1][(-s) mod n2] =
// H_s(k |d| w) e^{i s phi_d} for dmin <= |d| <= nb - 1, |s| <= 2Q (phi_d = 0 for d > 0, pi for
// d < 0); zero elsewhere.  One thread per offset: H_0, H_1 from the CUDA library, forward
// recurrence (the arguments are >= 2 k w).
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
    g[n2 - s] = make_double2(f * hq.x, f * hq.y);                              // s > 0 at column -s
    const double fn = (s & 1) ? -f : f;                                        // H_{-s} = (-1)^s H_s
    g[s] = make_double2(fn * hq.x, fn * hq.y);                                 // -s at column s
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

// M2M: one CTA per box, thread t <-> box order q = t - Q; writes bq[i][q + Q].  C is the complex
// type of the tables and the box coefficients (double2, or float2 in mixed precision).
template <typename C>
__global__ void k_fmm_m2m(const double2* __restrict__ xs, const int* __restrict__ perm,
                          const int* __restrict__ bstart, const C* __restrict__ tab, int p,
                          int Q, int S, C* __restrict__ bq) {
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
  if (q >= -Q && q <= Q) bq[(size_t)i * (2 * Q + 1) + q + Q] = acc;
}

// ---------------------------------------------------------------------------------------------
// The box-to-box convolution.  smem_fft: radix-2 Stockham (self-sorting) transforms of NF
// sequences of length L = 2^logL in shared memory, natural order in and out; element (f, pos) at
// pos NF + f (FFAST: the sequences interleaved) or f L + pos.  Stage s (Ls = 2^s, m = L / (2 Ls)):
// for t = j Ls + k < L / 2,
//   y[j 2Ls + k] = x[t] + w x[t + L/2],   y[j 2Ls + k + Ls] = x[t] - w x[t + L/2],   w = tw[k m step]
// with tw[u] = e^{-2 pi i u / (L step)} (conjugated for the inverse).  Returns the buffer that
// holds the result (x or y); every thread of the CTA takes part.
template <typename C> __device__ __forceinline__ C cplus(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C> __device__ __forceinline__ C cminus(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }

template <typename C, bool FFAST>
__device__ C* smem_fft(C* x, C* y, int logL, int logNF, const C* __restrict__ tw, int step, bool inv) {
  const int L = 1 << logL, half = L >> 1, NF = 1 << logNF;
  const int total = half << logNF;
  for (int s = 0; s < logL; ++s) {
    const int Ls = 1 << s, msh = logL - 1 - s;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
      int f, t;
      if (FFAST) {
        f = idx & (NF - 1);
        t = idx >> logNF;
      } else {
        t = idx & (half - 1);
        f = idx >> (logL - 1);
      }
      const int k = t & (Ls - 1), j = t >> s;
      C w = tw[(size_t)(k << msh) * step];
      if (inv) w.y = -w.y;
      const int o = j * 2 * Ls + k;
      const int ia = FFAST ? (t << logNF) + f : f * L + t;
      const int ib = FFAST ? ((t + half) << logNF) + f : f * L + t + half;
      const int oa = FFAST ? (o << logNF) + f : f * L + o;
      const int ob = FFAST ? ((o + Ls) << logNF) + f : f * L + o + Ls;
      const C a = x[ia], b = cmul(w, x[ib]);
      y[oa] = cplus(a, b);
      y[ob] = cminus(a, b);
    }
    __syncthreads();
    C* tmp = x;
    x = y;
    y = tmp;
  }
  return x;
}

constexpr int FFT_INV = 1;       // inverse transform (conjugate twiddles, no scaling)
constexpr int FFT_POST_TW = 2;   // forward four-step: output position k times e^{-2 pi i seg k / n1}
constexpr int FFT_PRE_TW = 4;    // inverse four-step: input position k times e^{+2 pi i seg k / n1}
constexpr int FFT_THREADS = 256;
constexpr int FFT_SMEM = 64 * 1024;   // two buffers (ping-pong) per CTA

// Transforms along the box index of the columns 0..ncols-1 of row-major arrays.  CTA (seg, column
// block of 2^logCT): the L = 2^logL rows seg * seg_stride + pos * rstride; rows >= in_rows read as
// zero, rows >= out_rows are not stored.  in and out may be the same array (each CTA reads its
// whole tile before it writes, and the tiles are disjoint).  twn[u] = e^{-2 pi i u / n1}.
template <typename C>
__global__ void __launch_bounds__(FFT_THREADS)
k_box_fft_cols(const C* in, int in_ld, int in_rows, C* out, int out_ld, int out_rows, int ncols,
               int logL, int logCT, int seg_stride, int rstride, const C* __restrict__ twn, int log_n1,
               int mode) {
  extern __shared__ __align__(16) unsigned char fft_raw[];
  const int L = 1 << logL, CT = 1 << logCT, n = L << logCT;
  C* x = reinterpret_cast<C*>(fft_raw);
  C* y = x + n;
  const int seg = blockIdx.x, c0 = blockIdx.y << logCT;
  const long long base = (long long)seg * seg_stride;
  for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
    const int pos = idx >> logCT, col = c0 + (idx & (CT - 1));
    const long long row = base + (long long)pos * rstride;
    C v = czero<C>();
    if (row < in_rows && col < ncols) v = in[row * in_ld + col];
    if (mode & FFT_PRE_TW) v = cmul(cconj(twn[(size_t)seg * pos]), v);
    x[idx] = v;
  }
  __syncthreads();
  const C* r = smem_fft<C, true>(x, y, logL, logCT, twn, 1 << (log_n1 - logL), mode & FFT_INV);
  for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
    const int pos = idx >> logCT, col = c0 + (idx & (CT - 1));
    const long long row = base + (long long)pos * rstride;
    C v = r[idx];
    if (mode & FFT_POST_TW) v = cmul(twn[(size_t)seg * pos], v);
    if (row < out_rows && col < ncols) out[row * out_ld + col] = v;
  }
}

// Transforms along the orders, 2^logNR frequency rows per CTA.  conv = 0 (kernel setup): rows of
// width n2, forward transform in place.  conv = 1: the rows hold the 2Q + 1 orders q = -Q..Q
// (row width W), placed at q mod n2 and zero elsewhere; forward transform, product with the
// transformed kernel khat (its row of the same frequency), inverse transform, the orders -Q..Q
// stored back.  tw2[u] = e^{-2 pi i u / n2}, u < n2 / 2.
template <typename C>
__global__ void __launch_bounds__(FFT_THREADS)
k_box_fft_rows(C* Y, long long nrows, int W, int Q, const C* __restrict__ khat, int logn2,
               const C* __restrict__ tw2, int logNR, int conv) {
  extern __shared__ __align__(16) unsigned char fft_raw[];
  const int n2 = 1 << logn2, n = n2 << logNR;
  C* x = reinterpret_cast<C*>(fft_raw);
  C* y = x + n;
  const long long r0 = (long long)blockIdx.x << logNR;
  for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
    const long long row = r0 + (idx >> logn2);
    const int k = idx & (n2 - 1);
    C v = czero<C>();
    if (row < nrows) {
      if (!conv) {
        v = Y[row * n2 + k];
      } else {
        const int q = k <= Q ? k : k - n2;
        if (q >= -Q) v = Y[row * W + q + Q];
      }
    }
    x[idx] = v;
  }
  __syncthreads();
  C* r = smem_fft<C, false>(x, y, logn2, logNR, tw2, 1, false);
  if (conv) {
    for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
      const long long row = r0 + (idx >> logn2);
      if (row < nrows) r[idx] = cmul(r[idx], khat[row * n2 + (idx & (n2 - 1))]);
    }
    __syncthreads();
    r = smem_fft<C, false>(r, r == x ? y : x, logn2, logNR, tw2, 1, true);
  }
  for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
    const long long row = r0 + (idx >> logn2);
    const int k = idx & (n2 - 1);
    if (row >= nrows) continue;
    if (!conv) {
      Y[row * n2 + k] = r[idx];
    } else {
      const int q = k <= Q ? k : k - n2;
      if (q >= -Q) Y[row * W + q + Q] = r[idx];
    }
  }
}

// tw[u] = e^{-2 pi i u / n}, u < count (n a power of two: -2 u / n is exact)
__global__ void k_fft_twiddles(double2* __restrict__ tw, int n, int count) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= count) return;
  double sn, cs;
  sincospi(-2.0 * (double)u / (double)n, &sn, &cs);
  tw[u] = make_double2(cs, sn);
}

// M2L for the offsets 2 <= |d| < dmin, box by box: acc[i][nu + Q] += sum_d sum_q
// hd[d][q - nu] B_{i-d}(q), hd[(sign, |d| - 2)][s + 2Q] = H_s(k |d| w) e^{i s phi_d}.
template <typename C>
__global__ void k_fmm_m2l_direct(const C* __restrict__ bq, const C* __restrict__ hd, int nb,
                                 int Q, int dmin, C* __restrict__ acc) {
  const int i = blockIdx.x;
  const int nu = (int)threadIdx.x - Q;
  if (nu < -Q || nu > Q) return;
  const int W = 2 * Q + 1, H = 4 * Q + 1;
  C a = czero<C>();
  for (int ad = 2; ad < dmin; ++ad)
    for (int sg = 0; sg < 2; ++sg) {
      const int d = sg ? -ad : ad;
      const int j = i - d;
      if (j < 0 || j >= nb) continue;
      const C* h = hd + (size_t)(2 * (ad - 2) + sg) * H + 2 * Q - nu;   // h[q] <-> s = q - nu
      const C* b = bq + (size_t)j * W + Q;
      for (int q = -Q; q <= Q; ++q) a = cfma(h[q], b[q], a);
    }
  C* g = acc + (size_t)i * W + nu + Q;
  *g = cadd(*g, a);
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

// L2L: one warp per disc, lane <-> nu; alpha = sum_q T_l[q - nu] A_box(q), A(q) = acc[b][q + Q].
template <typename C>
__global__ void k_fmm_l2l(const C* __restrict__ acc, const int* __restrict__ dbox,
                          const C* __restrict__ tab, int n, int p, int Q, int S,
                          double2* __restrict__ alpha) {
  const int l = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  const int P = 2 * p + 1;
  if (l >= n || lane >= P) return;
  const int nu = lane - p;
  const C* g = acc + (size_t)dbox[l] * (2 * Q + 1) + Q;
  const C* t = tab + (size_t)l * (2 * S + 1) + S;
  C a = czero<C>();
  for (int q = -Q; q <= Q; ++q) a = cfma(t[q - nu], g[q], a);
  alpha[(size_t)l * P + lane] = make_double2(a.x, a.y);
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

// log2 of the columns per CTA of k_box_fft_cols for L = 2^logL (at most 16, two buffers in FFT_SMEM)
template <typename C> int fft_log_tile(int logL) {
  const int elems = FFT_SMEM / (2 * (int)sizeof(C));
  int lct = 4;
  while (lct > 0 && ((1 << logL) << lct) > elems) --lct;
  return lct;
}

// One four-step pass along the boxes: step 1 (A-point transforms at stride B, segment n_b) or the
// B-point transforms on contiguous runs (segment k_a).
template <typename C>
void launch_box_cols(const FmmState& f, const C* in, int in_ld, int in_rows, C* out, int out_ld, int out_rows,
                     int ncols, bool step1, int mode, const C* twn, cudaStream_t st) {
  const int logL = step1 ? f.logA : f.logB;
  const int lct = fft_log_tile<C>(logL);
  dim3 grid(1u << (step1 ? f.logB : f.logA), (unsigned)((ncols + (1 << lct) - 1) >> lct));
  const size_t smem = 2 * ((size_t)1 << (logL + lct)) * sizeof(C);
  k_box_fft_cols<C><<<grid, FFT_THREADS, smem, st>>>(in, in_ld, in_rows, out, out_ld, out_rows, ncols, logL, lct,
                                                     step1 ? 1 : (1 << f.logB), step1 ? (1 << f.logB) : 1, twn,
                                                     f.logA + f.logB, mode);
}

template <typename C>
void launch_box_rows(const FmmState& f, C* Y, long long nrows, const C* khat, const C* tw2, int conv, cudaStream_t st) {
  const int elems = FFT_SMEM / (2 * (int)sizeof(C));
  int lnr = 0;
  while (lnr < 4 && (f.n2 << (lnr + 1)) <= elems) ++lnr;
  const long long blocks = (nrows + (1 << lnr) - 1) >> lnr;
  const size_t smem = 2 * ((size_t)f.n2 << lnr) * sizeof(C);
  k_box_fft_rows<C><<<(unsigned)blocks, FFT_THREADS, smem, st>>>(Y, nrows, 2 * f.order + 1, f.order, khat, f.logn2,
                                                                 tw2, lnr, conv);
}

void fft_attributes() {
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute(k_box_fft_cols<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, FFT_SMEM);
    cudaFuncSetAttribute(k_box_fft_cols<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, FFT_SMEM);
    cudaFuncSetAttribute(k_box_fft_rows<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, FFT_SMEM);
    cudaFuncSetAttribute(k_box_fft_rows<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, FFT_SMEM);
  });
}

// The far field of one right-hand side: M2M, the convolution (four-step transform along the boxes,
// the order rows with the kernel product, the inverse four-step transform), the direct offsets,
// L2L.  C = double2 (FP64) or float2 (mixed precision); xs and alpha are FP64.
template <typename C>
void box_far(const lsms_ctx* c, const double2* x, double2* a, const C* tab, C* bq, C* Y, C* acc, const C* khat,
             const C* hd, const C* twn, const C* tw2, cudaStream_t st) {
  const FmmState& f = c->fmm;
  const int n = c->n, p = c->p, P = 2 * p + 1, W = 2 * f.order + 1;
  const int qthreads = ((W + 31) / 32) * 32;
  k_fmm_m2m<C><<<f.nb, qthreads, P * sizeof(C), st>>>(x, f.d_perm, f.d_bstart, tab, p, f.order, f.S, bq);
  launch_box_cols<C>(f, bq, W, f.nb, Y, W, f.n1, W, true, FFT_POST_TW, twn, st);
  launch_box_cols<C>(f, Y, W, f.n1, Y, W, f.n1, W, false, 0, twn, st);
  launch_box_rows<C>(f, Y, f.n1, khat, tw2, 1, st);
  launch_box_cols<C>(f, Y, W, f.n1, Y, W, f.n1, W, false, FFT_INV, twn, st);
  launch_box_cols<C>(f, Y, W, f.n1, acc, W, f.nb, W, true, FFT_INV | FFT_PRE_TW, twn, st);
  if (f.dmin > 2) k_fmm_m2l_direct<C><<<f.nb, qthreads, 0, st>>>(bq, hd, f.nb, f.order, f.dmin, acc);
  k_fmm_l2l<C><<<(int)(((long long)n * 32 + 255) / 256), 256, 0, st>>>(acc, f.d_dbox, tab, n, p, f.order, f.S, a);
}

}  // namespace

void fmm_free(lsms_ctx* c) {
  FmmState& f = c->fmm;
  void* ptrs[] = {f.d_perm,  f.d_bstart, f.d_dbox,   f.d_sbox,   f.d_scx,  f.d_scy,   f.d_tab,   f.d_khat,
                  f.d_grid,  f.d_bq,     f.d_acc,    f.d_hd,     f.d_twn,  f.d_tw2,   f.d_scff,  f.ws.ptr,
                  f.d_tab32, f.d_khat32, f.d_grid32, f.d_bq32,   f.d_acc32, f.d_hd32, f.d_twn32, f.d_tw232};
  for (void* q : ptrs)
    if (q) cudaFree(q);
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
  int m1 = 0;
  while (f.far && (1 << m1) < 2 * nb - 1) ++m1;
  if (m1 > 18) {
    fmm_free(c);
    return ctx_fail(c, LSMS_ERR_ARG, "set_fmm: more than 131072 boxes; use wider boxes");
  }
  f.n1 = 1 << m1;
  f.logA = (m1 + 1) / 2;
  f.logB = m1 - f.logA;
  f.logn2 = 0;
  while ((1 << f.logn2) < 4 * f.order + 1) ++f.logn2;
  f.n2 = 1 << f.logn2;
  const int W = 2 * f.order + 1;
  const size_t gsz = f.far ? (size_t)f.n1 * f.n2 : 1;
  const size_t ysz = (size_t)f.n1 * W, asz = (size_t)nb * W;
  const size_t tsz = (size_t)n * (2 * f.S + 1);
  const size_t hsz = (size_t)std::max(1, 2 * (f.dmin - 2)) * (4 * f.order + 1);
  if (cudaMalloc((void**)&f.d_perm, n * sizeof(int)) != cudaSuccess ||
      cudaMalloc((void**)&f.d_bstart, (nb + 1) * sizeof(int)) != cudaSuccess ||
      cudaMalloc((void**)&f.d_dbox, n * sizeof(int)) != cudaSuccess ||
      cudaMalloc((void**)&f.d_sbox, n * sizeof(int)) != cudaSuccess ||
      cudaMalloc((void**)&f.d_scx, n * sizeof(double)) != cudaSuccess ||
      cudaMalloc((void**)&f.d_scy, n * sizeof(double)) != cudaSuccess ||
      cudaMalloc((void**)&f.d_scff, (size_t)n * sizeof(float4)) != cudaSuccess) {
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
  if (cudaMalloc((void**)&f.d_tab, tsz * sizeof(double2)) != cudaSuccess ||
      cudaMalloc((void**)&f.d_khat, gsz * sizeof(double2)) != cudaSuccess ||
      cudaMalloc((void**)&f.d_grid, ysz * sizeof(double2)) != cudaSuccess ||
      cudaMalloc((void**)&f.d_bq, asz * sizeof(double2)) != cudaSuccess ||
      cudaMalloc((void**)&f.d_acc, asz * sizeof(double2)) != cudaSuccess ||
      cudaMalloc((void**)&f.d_hd, hsz * sizeof(double2)) != cudaSuccess ||
      cudaMalloc((void**)&f.d_twn, (size_t)f.n1 * sizeof(double2)) != cudaSuccess ||
      cudaMalloc((void**)&f.d_tw2, (size_t)std::max(1, f.n2 / 2) * sizeof(double2)) != cudaSuccess ||
      cudaMalloc((void**)&f.d_tab32, tsz * sizeof(float2)) != cudaSuccess ||
      cudaMalloc((void**)&f.d_khat32, gsz * sizeof(float2)) != cudaSuccess ||
      cudaMalloc((void**)&f.d_grid32, ysz * sizeof(float2)) != cudaSuccess ||
      cudaMalloc((void**)&f.d_bq32, asz * sizeof(float2)) != cudaSuccess ||
      cudaMalloc((void**)&f.d_acc32, asz * sizeof(float2)) != cudaSuccess ||
      cudaMalloc((void**)&f.d_hd32, hsz * sizeof(float2)) != cudaSuccess ||
      cudaMalloc((void**)&f.d_twn32, (size_t)f.n1 * sizeof(float2)) != cudaSuccess ||
      cudaMalloc((void**)&f.d_tw232, (size_t)std::max(1, f.n2 / 2) * sizeof(float2)) != cudaSuccess) {
    cudaGetLastError();
    fmm_free(c);
    return ctx_fail(c, LSMS_ERR_OOM, "set_fmm: cudaMalloc failed for the box tables");
  }
  fft_attributes();
  k_fmm_shift_table<<<blocks_for((long long)tsz, 256), 256, 0, st>>>(c->d_cx, c->d_cy, f.d_dbox, n, f.x0, w,
                                                                      -0.5 * c->d, c->k2, f.S, f.d_tab);
  k_fft_twiddles<<<(f.n1 + 255) / 256, 256, 0, st>>>(f.d_twn, f.n1, f.n1);
  k_fft_twiddles<<<(f.n2 / 2 + 255) / 256, 256, 0, st>>>(f.d_tw2, f.n2, f.n2 / 2);
  // the box kernel and its two-dimensional transform (orders, then the four-step split along the
  // boxes over all n2 columns), scaled by 1 / (n1 n2)
  cudaMemsetAsync(f.d_khat, 0, gsz * sizeof(double2), st);
  const int nd = 2 * (nb - 1) + 1;
  k_fmm_box_kernel<<<(nd + 127) / 128, 128, 0, st>>>(nb, f.order, c->k2, w, f.n1, f.n2, f.dmin, f.d_khat);
  if (f.dmin > 2) k_fmm_direct_table<<<(2 * (f.dmin - 2) + 63) / 64, 64, 0, st>>>(f.order, c->k2, w, f.dmin, f.d_hd);
  launch_box_rows<double2>(f, f.d_khat, f.n1, nullptr, f.d_tw2, 0, st);
  launch_box_cols<double2>(f, f.d_khat, f.n2, f.n1, f.d_khat, f.n2, f.n1, f.n2, true, FFT_POST_TW, f.d_twn, st);
  launch_box_cols<double2>(f, f.d_khat, f.n2, f.n1, f.d_khat, f.n2, f.n1, f.n2, false, 0, f.d_twn, st);
  k_fmm_scale<<<blocks_for((long long)gsz, 256), 256, 0, st>>>(f.d_khat, (long long)gsz, 1.0 / (double)gsz);
  // FP32 copies for the mixed-precision far field
  k_fmm_d2f<<<blocks_for((long long)tsz, 256), 256, 0, st>>>(f.d_tab, f.d_tab32, (long long)tsz);
  k_fmm_d2f<<<blocks_for((long long)gsz, 256), 256, 0, st>>>(f.d_khat, f.d_khat32, (long long)gsz);
  k_fmm_d2f<<<blocks_for((long long)f.n1, 256), 256, 0, st>>>(f.d_twn, f.d_twn32, (long long)f.n1);
  k_fmm_d2f<<<blocks_for((long long)(f.n2 / 2), 256), 256, 0, st>>>(f.d_tw2, f.d_tw232, (long long)(f.n2 / 2));
  if (f.dmin > 2) k_fmm_d2f<<<blocks_for((long long)hsz, 256), 256, 0, st>>>(f.d_hd, f.d_hd32, (long long)hsz);
  cudaStreamSynchronize(st);
  f.ready = true;
  return check_cuda(c, "set_fmm");
}

// alpha = T xs for nrhs right-hand sides through the box method.  Launches: per right-hand side
// M2M, five transform passes, the direct offsets and L2L, plus the near-field launches.
int fmm_translate(lsms_ctx* c, int nrhs, const double2* xs, double2* alpha, bool mixed, cudaStream_t st) {
  FmmState& f = c->fmm;
  const int n = c->n, p = c->p, P = 2 * p + 1;
  if (!f.ready) return ctx_fail(c, LSMS_ERR_STATE, "box translation tables are not built");
  const bool timed = c->timing && !c->kids.size();
  if (timed && !f.ev[0])
    for (cudaEvent_t& e : f.ev) cudaEventCreate(&e);
  if (timed) cudaEventRecord(f.ev[0], st);
  if (!f.far) cudaMemsetAsync(alpha, 0, (size_t)nrhs * n * P * sizeof(double2), st);
  for (int r = 0; r < nrhs && f.far; ++r) {
    const double2* x = xs + (size_t)r * n * P;
    double2* a = alpha + (size_t)r * n * P;
    if (mixed)
      box_far<float2>(c, x, a, f.d_tab32, f.d_bq32, f.d_grid32, f.d_acc32, f.d_khat32, f.d_hd32, f.d_twn32,
                      f.d_tw232, st);
    else
      box_far<double2>(c, x, a, f.d_tab, f.d_bq, f.d_grid, f.d_acc, f.d_khat, f.d_hd, f.d_twn, f.d_tw2, st);
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
