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
#include "near_pairs.cuh"
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

// The mixed near field's pair sequences: row k of seq = h[s + 2p] = H_s(k rho) e^{i s phi}, s =
// -2p..2p (then one zero), for list entry k (target perm[t], source csrc[k]); built in FP64 (CUDA
// J0, Y0, J1, Y1, forward recurrence, angular powers) and stored in FP32.  One thread per target.
__global__ void k_fmm_pair_seq(const double* __restrict__ cx, const double* __restrict__ cy,
                               const int* __restrict__ perm, const int* __restrict__ cptr,
                               const int* __restrict__ csrc, int n, int p, double k, float2* __restrict__ seq) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int l = perm[t], RS = 4 * p + 2, c0 = 2 * p;
  for (int e = cptr[t]; e < cptr[t + 1]; ++e) {
    const int m = csrc[e];
    const double dx = cx[l] - cx[m], dy = cy[l] - cy[m];
    const double rho = hypot(dx, dy), z = k * rho;
    const double2 e1 = make_double2(dx / rho, dy / rho);
    float2* h = seq + (size_t)e * RS;
    double2 hm = make_double2(j0(z), y0(z)), hq = make_double2(j1(z), y1(z)), eq = e1;
    h[c0] = make_float2((float)hm.x, (float)hm.y);
    for (int q = 1; q <= 2 * p; ++q) {
      const double2 v = cmul(hq, eq);
      const double2 u = cmul(hq, make_double2(eq.x, -eq.y));
      const double sg = (q & 1) ? -1.0 : 1.0;
      h[c0 + q] = make_float2((float)v.x, (float)v.y);
      h[c0 - q] = make_float2((float)(sg * u.x), (float)(sg * u.y));
      if (q < 2 * p) {
        const double f = 2.0 * q / z;
        const double2 hn = make_double2(f * hq.x - hm.x, f * hq.y - hm.y);
        hm = hq;
        hq = hn;
        eq = cmul(eq, e1);
      }
    }
    h[4 * p + 1] = make_float2(0.f, 0.f);
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

// The shift kernels (M2M, L2L, the direct offsets) are Toeplitz contractions: a lane owns 4
// consecutive outputs and keeps the 4 sequence entries they need for the current input in
// registers, so that each input costs one shared-memory load of the sequence (the window slides by
// one) and one of the input.  A sequence row is stored as four sub-arrays by index mod 4, so the
// lanes of a warp, whose windows start 4 entries apart, read consecutive words.
constexpr int SH_W = 4;   // warps per CTA of the shift kernels

template <typename C>
__device__ __forceinline__ void row_put(C* sub, int L4, int j, C v) { sub[(j & 3) * L4 + (j >> 2)] = v; }
template <typename C>
__device__ __forceinline__ C row_get(const C* sub, int L4, int j, int jmax) {
  return (j >= 0 && j <= jmax) ? sub[(j & 3) * L4 + (j >> 2)] : czero<C>();
}

// M2M: one warp per box; lane <-> box orders w = w0 + 4 lane + i (w = q + Q, chunks of 128).
// B_i(q) = sum_{m in box i} sum_n conj(T_m[q - n]) beta^m_n, T_m[s] = J_s(k r_m) e^{i s phi_m}; with
// a = n + p the entry is T_m row index w - a + 2p.  Writes bq[i][w].  C: the complex type of the
// tables and the box coefficients (double2, or float2 in mixed precision); xs is FP64.
template <typename C>
__global__ void __launch_bounds__(SH_W * 32)
k_fmm_m2m(const double2* __restrict__ xs, const int* __restrict__ perm, const int* __restrict__ bstart,
          const C* __restrict__ tab, int nb, int p, int Q, int S, C* __restrict__ bq) {
  extern __shared__ __align__(16) unsigned char sh_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int P = 2 * p + 1, W = 2 * Q + 1, jmax = 2 * S, L4 = (2 * S + 4) / 4;
  C* sub = reinterpret_cast<C*>(sh_raw) + (size_t)warp * (4 * L4 + P);
  C* beta = sub + 4 * L4;
  const int box = blockIdx.x * SH_W + warp;
  if (box >= nb) return;
  const int j0 = bstart[box], j1 = bstart[box + 1];
  for (int w0 = 0; w0 < W; w0 += 128) {
    C acc[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) acc[i] = czero<C>();
    const int base = w0 + 4 * lane + 2 * p;
    for (int jj = j0; jj < j1; ++jj) {
      const int m = perm[jj];
      __syncwarp();
      for (int j = lane; j <= jmax; j += 32) row_put(sub, L4, j, tab[(size_t)m * (2 * S + 1) + j]);
      for (int a = lane; a < P; a += 32) beta[a] = from_d2<C>(xs[(size_t)m * P + a]);
      __syncwarp();
      C win[4];                                          // win[i] = T_m[base + i - a]
#pragma unroll
      for (int i = 0; i < 4; ++i) win[i] = row_get(sub, L4, base + i, jmax);
      for (int a = 0; a < P; ++a) {
        const C b = beta[a];
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[i] = cfma(cconj(win[i]), b, acc[i]);
        win[3] = win[2];
        win[2] = win[1];
        win[1] = win[0];
        win[0] = row_get(sub, L4, base - a - 1, jmax);
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int w = w0 + 4 * lane + i;
      if (w < W) bq[(size_t)box * W + w] = acc[i];
    }
  }
}

// ---------------------------------------------------------------------------------------------
// The box-to-box convolution.  smem_fft: Stockham (self-sorting) transforms of NF sequences of
// length L = 2^logL held in shared memory, natural order in and out; element (f, pos) at
// pos fs + f (FFAST: the sequences interleaved, fs = NF or a padded stride) or f L + pos.  Radix-4
// stages while two or more factors of 2 remain, then one radix-2 stage.  With Ls the length
// already transformed,
// tw[u] = e^{-2 pi i u / (L step)} (conjugated for the inverse), t = j Ls + k:
//   radix 4 (t < L/4, m = L / (4 Ls), w = tw[k m step], w^2, w^3 from the table (FP64) or as
//     products (FP32)):  a_r = w^r x[t + r L/4],
//     y[j 4Ls + k + q Ls] = sum_r (-i)^{q r} a_r   (+i for the inverse), q = 0..3;
//   radix 2 (t < L/2, m = L / (2 Ls), w = tw[k m step]):
//     y[j 2Ls + k] = x[t] + w x[t + L/2],   y[j 2Ls + k + Ls] = x[t] - w x[t + L/2].
// Returns the buffer that holds the result (x or y); every thread of the CTA takes part.
template <typename C> __device__ __forceinline__ C cplus(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C> __device__ __forceinline__ C cminus(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }

template <typename C, bool FFAST>
__device__ C* smem_fft(C* x, C* y, int logL, int logNF, const C* __restrict__ tw, int step, bool inv,
                       int fstride = 0) {
  const int L = 1 << logL, NF = 1 << logNF;
  const int fs = fstride > 0 ? fstride : NF;      // FFAST: element (f, pos) at pos fs + f
  auto at = [&](int f, int pos) { return FFAST ? pos * fs + f : f * L + pos; };
  int s = 0;
  while (s < logL) {
    const int Ls = 1 << s;
    if (logL - s >= 2) {
      const int q4 = L >> 2, msh = logL - 2 - s;
      const int total = q4 << logNF;
      for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        int f, t;
        if (FFAST) {
          f = idx & (NF - 1);
          t = idx >> logNF;
        } else {
          t = idx & (q4 - 1);
          f = idx >> (logL - 2);
        }
        const int k = t & (Ls - 1), j = t >> s;
        const size_t u = (size_t)(k << msh) * step;
        C w1 = tw[u], w2, w3;
        if (sizeof(C) == sizeof(double2)) {        // FP64: the table (the FP64 pipe is the limit)
          w2 = tw[2 * u];
          w3 = tw[3 * u];
        } else {                                   // FP32: products (the loads cost more)
          w2 = cmul(w1, w1);
          w3 = cmul(w1, w2);
        }
        if (inv) {
          w1.y = -w1.y;
          w2.y = -w2.y;
          w3.y = -w3.y;
        }
        const C a0 = x[at(f, t)];
        const C a1 = cmul(w1, x[at(f, t + q4)]);
        const C a2 = cmul(w2, x[at(f, t + 2 * q4)]);
        const C a3 = cmul(w3, x[at(f, t + 3 * q4)]);
        const C c0 = cplus(a0, a2), c1 = cminus(a0, a2), c2 = cplus(a1, a3), d = cminus(a1, a3);
        C c3;                                      // d (-i) forward, d (+i) inverse
        c3.x = inv ? -d.y : d.y;
        c3.y = inv ? d.x : -d.x;
        const int o = j * 4 * Ls + k;
        y[at(f, o)] = cplus(c0, c2);
        y[at(f, o + Ls)] = cplus(c1, c3);
        y[at(f, o + 2 * Ls)] = cminus(c0, c2);
        y[at(f, o + 3 * Ls)] = cminus(c1, c3);
      }
      s += 2;
    } else {
      const int half = L >> 1, msh = logL - 1 - s;
      const int total = half << logNF;
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
        const C a = x[at(f, t)], b = cmul(w, x[at(f, t + half)]);
        const int o = j * 2 * Ls + k;
        y[at(f, o)] = cplus(a, b);
        y[at(f, o + Ls)] = cminus(a, b);
      }
      s += 1;
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
constexpr int FFT_SMEM = 80 * 1024;   // two buffers (ping-pong) per CTA

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

// Transforms along the orders, 2^logNR frequency rows per CTA, held interleaved in shared memory
// (element (row r, frequency k) at k (NR + 1) + r: the odd stride keeps both the row loads and the
// butterflies free of bank conflicts).  conv = 0 (kernel setup): rows of width n2, forward transform
// in place.  conv = 1: the rows hold the 2Q + 1 orders q = -Q..Q (row width W), placed at q mod n2
// and zero elsewhere; forward transform, product with the transformed kernel khat (its row of the
// same frequency), inverse transform, the orders -Q..Q stored back.  tw2[u] = e^{-2 pi i u / n2},
// u < n2.
template <typename C>
__global__ void __launch_bounds__(FFT_THREADS)
k_box_fft_rows(C* Y, long long nrows, int W, int Q, const C* __restrict__ khat, int logn2,
               const C* __restrict__ tw2, int logNR, int conv) {
  extern __shared__ __align__(16) unsigned char fft_raw[];
  const int n2 = 1 << logn2, NR = 1 << logNR, S = NR + 1, n = n2 << logNR;
  C* x = reinterpret_cast<C*>(fft_raw);
  C* y = x + n2 * S;
  const long long r0 = (long long)blockIdx.x << logNR;
  for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
    const int rr = idx >> logn2, k = idx & (n2 - 1);
    const long long row = r0 + rr;
    C v = czero<C>();
    if (row < nrows) {
      if (!conv) {
        v = Y[row * n2 + k];
      } else {
        const int q = k <= Q ? k : k - n2;
        if (q >= -Q) v = Y[row * W + q + Q];
      }
    }
    x[k * S + rr] = v;
  }
  __syncthreads();
  C* r = smem_fft<C, true>(x, y, logn2, logNR, tw2, 1, false, S);
  if (conv) {
    for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
      const int rr = idx >> logn2, k = idx & (n2 - 1);
      const long long row = r0 + rr;
      if (row < nrows) r[k * S + rr] = cmul(r[k * S + rr], khat[row * n2 + k]);
    }
    __syncthreads();
    r = smem_fft<C, true>(r, r == x ? y : x, logn2, logNR, tw2, 1, true, S);
  }
  for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
    const int rr = idx >> logn2, k = idx & (n2 - 1);
    const long long row = r0 + rr;
    if (row >= nrows) continue;
    if (!conv) {
      Y[row * n2 + k] = r[k * S + rr];
    } else {
      const int q = k <= Q ? k : k - n2;
      if (q >= -Q) Y[row * W + q + Q] = r[k * S + rr];
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
// hd[d][q - nu + 2Q] B_{i-d}(q), hd[(sign, |d| - 2)][s + 2Q] = H_s(k |d| w) e^{i s phi_d}.  One warp
// per box; lane <-> outputs o = o0 + 4 lane + i (o = nu + Q, chunks of 128); the entry for input
// w = q + Q is hd row index 2Q + w - o.  Per offset the warp stages the kernel row and the source
// box's coefficients in shared memory.
template <typename C>
__global__ void __launch_bounds__(SH_W * 32)
k_fmm_m2l_direct(const C* __restrict__ bq, const C* __restrict__ hd, int nb, int Q, int dmin,
                 C* __restrict__ acc) {
  extern __shared__ __align__(16) unsigned char sh_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int W = 2 * Q + 1, H = 4 * Q + 1, jmax = 4 * Q, L4 = (H + 3) / 4;
  C* sub = reinterpret_cast<C*>(sh_raw) + (size_t)warp * (4 * L4 + W);
  C* brow = sub + 4 * L4;
  const int box = blockIdx.x * SH_W + warp;
  if (box >= nb) return;
  for (int o0 = 0; o0 < W; o0 += 128) {
    C a4[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) a4[i] = czero<C>();
    const int base = 2 * Q - o0 - 4 * lane;
    for (int ad = 2; ad < dmin; ++ad)
      for (int sg = 0; sg < 2; ++sg) {
        const int src = box - (sg ? -ad : ad);
        if (src < 0 || src >= nb) continue;
        const C* h = hd + (size_t)(2 * (ad - 2) + sg) * H;
        __syncwarp();
        for (int j = lane; j < H; j += 32) row_put(sub, L4, j, h[j]);
        for (int w = lane; w < W; w += 32) brow[w] = bq[(size_t)src * W + w];
        __syncwarp();
        C win[4];                                        // win[i] = hd[base + w - i]
#pragma unroll
        for (int i = 0; i < 4; ++i) win[i] = row_get(sub, L4, base - i, jmax);
        for (int w = 0; w < W; ++w) {
          const C b = brow[w];
#pragma unroll
          for (int i = 0; i < 4; ++i) a4[i] = cfma(win[i], b, a4[i]);
          win[3] = win[2];
          win[2] = win[1];
          win[1] = win[0];
          win[0] = row_get(sub, L4, base + w + 1, jmax);
        }
      }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int o = o0 + 4 * lane + i;
      if (o < W) {
        C* g = acc + (size_t)box * W + o;
        *g = cadd(*g, a4[i]);
      }
    }
  }
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

// L2L: 4 discs per warp, 8 lanes per disc; lane <-> outputs o = 4 (lane & 7) + i (o = nu + p).
// alpha_l(nu) = sum_q T_l[q - nu] A_box(q), A(q) = acc[b][q + Q]; with w = q + Q the entry is T_l row
// index w - o + 2p.  The discs' T rows are staged in shared memory, A is read through the cache.
template <typename C>
__global__ void __launch_bounds__(SH_W * 32)
k_fmm_l2l(const C* __restrict__ acc, const int* __restrict__ dbox, const C* __restrict__ tab, int n, int p,
          int Q, int S, double2* __restrict__ alpha) {
  extern __shared__ __align__(16) unsigned char sh_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 3, j8 = lane & 7;
  const int P = 2 * p + 1, W = 2 * Q + 1, jmax = 2 * S, L4 = (2 * S + 4) / 4;
  C* sub = reinterpret_cast<C*>(sh_raw) + (size_t)(warp * 4 + g) * 4 * L4;
  const int l = (blockIdx.x * SH_W + warp) * 4 + g;
  const bool valid = l < n;
  if (valid)
    for (int j = j8; j <= jmax; j += 8) row_put(sub, L4, j, tab[(size_t)l * (2 * S + 1) + j]);
  __syncwarp();
  if (!valid) return;
  const C* arow = acc + (size_t)dbox[l] * W;
  const int base = 2 * p - 4 * j8;
  C a4[4], win[4];                                       // win[i] = T_l[base + w - i]
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    a4[i] = czero<C>();
    win[i] = row_get(sub, L4, base - i, jmax);
  }
  for (int w = 0; w < W; ++w) {
    const C b = arow[w];
#pragma unroll
    for (int i = 0; i < 4; ++i) a4[i] = cfma(win[i], b, a4[i]);
    win[3] = win[2];
    win[2] = win[1];
    win[1] = win[0];
    win[0] = row_get(sub, L4, base + w + 1, jmax);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int o = 4 * j8 + i;
    if (o < P) alpha[(size_t)l * P + o] = make_double2(a4[i].x, a4[i].y);
  }
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


__global__ void k_fmm_d2f(const double2* __restrict__ a, float2* __restrict__ b, long long total) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x)
    b[i] = make_float2((float)a[i].x, (float)a[i].y);
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
  const int elems = FFT_SMEM / (2 * (int)sizeof(C));   // per buffer: n2 (NR + 1) elements
  int lnr = 0;
  while (lnr < 4 && f.n2 * ((1 << (lnr + 1)) + 1) <= elems) ++lnr;
  const long long blocks = (nrows + (1 << lnr) - 1) >> lnr;
  const size_t smem = 2 * (size_t)f.n2 * ((1 << lnr) + 1) * sizeof(C);
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
    // the shift kernels need up to 4 warps x 4 rows x (2 (400 + 15) + 4) FP64 entries (L2L, order 400)
    const int sh = 220 * 1024;
    cudaFuncSetAttribute(k_fmm_m2m<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, sh);
    cudaFuncSetAttribute(k_fmm_m2m<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, sh);
    cudaFuncSetAttribute(k_fmm_l2l<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, sh);
    cudaFuncSetAttribute(k_fmm_l2l<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, sh);
    cudaFuncSetAttribute(k_fmm_m2l_direct<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, sh);
    cudaFuncSetAttribute(k_fmm_m2l_direct<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, sh);
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
  const int L4s = (2 * f.S + 4) / 4, L4h = (4 * f.order + 4) / 4;
  const unsigned gb = (unsigned)((f.nb + SH_W - 1) / SH_W);
  k_fmm_m2m<C><<<gb, SH_W * 32, SH_W * (4 * L4s + P) * sizeof(C), st>>>(x, f.d_perm, f.d_bstart, tab, f.nb, p,
                                                                      f.order, f.S, bq);
  launch_box_cols<C>(f, bq, W, f.nb, Y, W, f.n1, W, true, FFT_POST_TW, twn, st);
  launch_box_cols<C>(f, Y, W, f.n1, Y, W, f.n1, W, false, 0, twn, st);
  launch_box_rows<C>(f, Y, f.n1, khat, tw2, 1, st);
  launch_box_cols<C>(f, Y, W, f.n1, Y, W, f.n1, W, false, FFT_INV, twn, st);
  launch_box_cols<C>(f, Y, W, f.n1, acc, W, f.nb, W, true, FFT_INV | FFT_PRE_TW, twn, st);
  if (f.dmin > 2)
    k_fmm_m2l_direct<C><<<gb, SH_W * 32, SH_W * (4 * L4h + W) * sizeof(C), st>>>(bq, hd, f.nb, f.order, f.dmin, acc);
  k_fmm_l2l<C><<<(unsigned)((n + 4 * SH_W - 1) / (4 * SH_W)), SH_W * 32, SH_W * 4 * 4 * L4s * sizeof(C), st>>>(
      acc, f.d_dbox, tab, n, p, f.order, f.S, a);
}

}  // namespace

void fmm_free(lsms_ctx* c) {
  FmmState& f = c->fmm;
  void* ptrs[] = {f.d_perm,  f.d_bstart, f.d_dbox,   f.d_sbox,   f.d_scx,  f.d_scy,   f.d_tab,   f.d_khat,
                  f.d_grid,  f.d_bq,     f.d_acc,    f.d_hd,     f.d_twn,  f.d_tw2,   f.d_cptr,  f.d_csrc,
                  f.d_cseq,  f.ws.ptr,
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
  // pair lists of the mixed near field by target in box order: every pair in the same or adjacent
  // boxes (their sequences are built on the device below)
  std::vector<int> cptr(n + 1, 0), csrc;
  csrc.reserve((size_t)f.near_pairs);
  for (int t = 0; t < n; ++t) {
    const int l = perm[t], b = dbox[l];
    for (int j = bstart[std::max(b - 1, 0)]; j < bstart[std::min(b + 2, nb)]; ++j)
      if (perm[j] != l) csrc.push_back(perm[j]);
    cptr[t + 1] = (int)csrc.size();
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
      cudaMalloc((void**)&f.d_cptr, (n + 1) * sizeof(int)) != cudaSuccess ||
      cudaMalloc((void**)&f.d_csrc, std::max<size_t>(1, csrc.size()) * sizeof(int)) != cudaSuccess ||
      cudaMalloc((void**)&f.d_cseq, std::max<size_t>(1, csrc.size()) * (4 * p + 2) * sizeof(float2)) !=
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
  cudaMemcpy(f.d_cptr, cptr.data(), (n + 1) * sizeof(int), cudaMemcpyHostToDevice);
  if (!csrc.empty()) cudaMemcpy(f.d_csrc, csrc.data(), csrc.size() * sizeof(int), cudaMemcpyHostToDevice);
  cudaStream_t st = c->stream;
  k_fmm_pair_seq<<<(n + 127) / 128, 128, 0, st>>>(c->d_cx, c->d_cy, f.d_perm, f.d_cptr, f.d_csrc, n, p, c->k2,
                                                  f.d_cseq);
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
      cudaMalloc((void**)&f.d_tw2, (size_t)f.n2 * sizeof(double2)) != cudaSuccess ||
      cudaMalloc((void**)&f.d_tab32, tsz * sizeof(float2)) != cudaSuccess ||
      cudaMalloc((void**)&f.d_khat32, gsz * sizeof(float2)) != cudaSuccess ||
      cudaMalloc((void**)&f.d_grid32, ysz * sizeof(float2)) != cudaSuccess ||
      cudaMalloc((void**)&f.d_bq32, asz * sizeof(float2)) != cudaSuccess ||
      cudaMalloc((void**)&f.d_acc32, asz * sizeof(float2)) != cudaSuccess ||
      cudaMalloc((void**)&f.d_hd32, hsz * sizeof(float2)) != cudaSuccess ||
      cudaMalloc((void**)&f.d_twn32, (size_t)f.n1 * sizeof(float2)) != cudaSuccess ||
      cudaMalloc((void**)&f.d_tw232, (size_t)f.n2 * sizeof(float2)) != cudaSuccess) {
    cudaGetLastError();
    fmm_free(c);
    return ctx_fail(c, LSMS_ERR_OOM, "set_fmm: cudaMalloc failed for the box tables");
  }
  fft_attributes();
  k_fmm_shift_table<<<blocks_for((long long)tsz, 256), 256, 0, st>>>(c->d_cx, c->d_cy, f.d_dbox, n, f.x0, w,
                                                                      -0.5 * c->d, c->k2, f.S, f.d_tab);
  k_fft_twiddles<<<(f.n1 + 255) / 256, 256, 0, st>>>(f.d_twn, f.n1, f.n1);
  k_fft_twiddles<<<(f.n2 + 255) / 256, 256, 0, st>>>(f.d_tw2, f.n2, f.n2);
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
  k_fmm_d2f<<<blocks_for((long long)f.n2, 256), 256, 0, st>>>(f.d_tw2, f.d_tw232, (long long)f.n2);
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
    // near field in FP32: an FP32 copy of the coefficients, then the stored-sequence kernel
    // (near_pairs.cuh) adds the same-box and adjacent-box pairs, in box order, into alpha
    const long long len = (long long)nrhs * n * P;
    int rc;
    if ((rc = ensure(c, f.ws, (size_t)len * sizeof(float2)))) return rc;
    float2* x32 = (float2*)f.ws.ptr;
    if (timed) cudaEventRecord(f.ev[1], st);
    k_fmm_d2f<<<blocks_for(len, 256), 256, 0, st>>>(xs, x32, len);
    launch_pair_seq(p, nrhs, st, f.d_perm, f.d_cptr, f.d_csrc, f.d_cseq, n, x32, alpha);
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
