// FP64 kernels of the multiple-scattering operator y = x - S (T + R) x.
//
//   translation (Sec. 3.2 Lemma 3.1): tiled all pairs, one warp per target disc, lanes over the
//     output order nu; each lane of the warp generates the Hankel sequence of one source disc
//     (warp-cooperative: 32 pair sequences at once) into shared memory, then the warp contracts
//     the Toeplitz block against the staged source coefficients.
//   aggregate / disaggregate (Sec. 5.3 Thm 5.2; Sec. 5.2.1 Lemma 5.1): complex GEMMs against the
//     precomputed plane-wave tables, then per-node order-factor dots.
//   per-node reflection (Sec. 2 Eq. "sommerfeldsys"): closed-form 2x2 response per node.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "lsms_internal.h"

#include "c64.cuh"

namespace {

// ---------------------------------------------------------------------------------------------
// xs = scale[n] * x
// ---------------------------------------------------------------------------------------------
__global__ void k_scale_in(const double2* __restrict__ x, const double* __restrict__ scale,
                           double2* __restrict__ xs, long long total, int P) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const double s = scale[i % P];
    const double2 v = x[i];
    xs[i] = make_double2(v.x * s, v.y * s);
  }
}

// ---------------------------------------------------------------------------------------------
// Translation, FP64
// ---------------------------------------------------------------------------------------------
constexpr int TW = 4;    // target discs (warps) per CTA
constexpr int CH = 32;   // source discs per staged chunk (one per lane for the Hankel sequences)
constexpr int HS = 65;   // length of a pair's sequence h_s, s = -2p..2p (4p + 1 <= 61); odd stride avoids bank conflicts

// alpha^l_nu = sum_{m != l} sum_n h^{lm}_{n - nu} xs^m_n.  One warp per target disc, lane = nu.
// Complex products use three real FMAs (Gauss): A += hr br, B += hi bi, C += (hr+hi)(br+bi);
// alpha = (A - B) + i (C - A - B).  The sums hr+hi and br+bi are formed once, when the sequence is
// generated and when the source coefficients are staged.
// Target discs l = row0 .. row0 + nrows - 1 (all sources); alpha holds those rows only,
// [nrhs][nrows][P].
__global__ void __launch_bounds__(TW * 32, 1)
k_translate_f64(const double* __restrict__ cx, const double* __restrict__ cy, int n, int p,
                double k, const double2* __restrict__ xs, double2* __restrict__ alpha, int row0,
                int nrows) {
  extern __shared__ double2 smem[];
  double2* sb = smem;                                   // [CH][32] staged source coefficients
  double* sbs = (double*)(sb + CH * 32);                // [CH][32] their re + im
  double2* sh = (double2*)(sbs + CH * 32);              // [TW][CH][HS] pair sequences
  double* shs = (double*)(sh + TW * CH * HS);           // [TW][CH][HS] their re + im
  __shared__ double scx[CH], scy[CH];
  const int P = 2 * p + 1;
  const int r = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int l = row0 + blockIdx.x * TW + warp;
  const bool lvalid = l < row0 + nrows && l < n;
  const double xl = lvalid ? cx[l] : 0.0, yl = lvalid ? cy[l] : 0.0;
  const double2* xr = xs + (size_t)r * n * P;
  double2* hw = sh + (size_t)warp * CH * HS;
  double* hsw = shs + (size_t)warp * CH * HS;
  double A = 0.0, B = 0.0, C = 0.0;
  for (int j0c = 0; j0c < n; j0c += CH) {
    const int cnt = min(CH, n - j0c);
    __syncthreads();
    for (int i = threadIdx.x; i < cnt * P; i += blockDim.x) {
      const int s = i / P, q = i - s * P;
      const double2 v = xr[(size_t)(j0c + s) * P + q];
      sb[s * 32 + q] = v;
      sbs[s * 32 + q] = v.x + v.y;
    }
    if (threadIdx.x < cnt) {
      scx[threadIdx.x] = cx[j0c + threadIdx.x];
      scy[threadIdx.x] = cy[j0c + threadIdx.x];
    }
    __syncthreads();
    if (lane < cnt) {
      double2* h = hw + lane * HS;
      double* hsm = hsw + lane * HS;
      if (lvalid && j0c + lane != l) {
        hankel_sequence_f64(xl - scx[lane], yl - scy[lane], k, p, h, hsm);
      } else {
        for (int q = 0; q <= 4 * p; ++q) {
          h[q] = make_double2(0.0, 0.0);
          hsm[q] = 0.0;
        }
      }
    }
    __syncwarp();
    if (lvalid && lane < P) {
      for (int s = 0; s < cnt; ++s) {
        const double2* hs = hw + s * HS + 2 * p - lane;   // hs[q] = h_{n - nu}, n = q - p
        const double* hss = hsw + s * HS + 2 * p - lane;
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
  if (lvalid && lane < P)
    alpha[((size_t)r * nrows + (l - row0)) * P + lane] = make_double2(A - B, C - A - B);
}

// One sequence per unordered pair.  Turning phi by pi gives h_s(m <- l) = (-1)^s h_s(l <- m), so
// alpha^m_nu = (-1)^nu sum_n h^{lm}_{n - nu} ((-1)^n xs^l_n): the sequence generated for l <- m,
// read with the same window, also contracts l's sign-flipped coefficients into m's outputs.  A CTA
// of TW warps owns a block of TW target discs and a run of CH-disc source chunks; warp w (target
// l = TW b + w) generates the sequences of its pairs with the chunk's sources m > l (one per
// lane), contracts them into l's outputs (lanes over nu, as in k_translate_f64) and into every
// source's outputs, which it adds into alpha with FP64 atomics; l's own outputs are added when
// the CTA's target block changes.  Blocks form double rows (block h with its chunks, then block
// B - 1 - h with its chunks: about as many chunks as one full row), cut into runs of
// `chunks_per_cta` chunks.  alpha must be zero on entry; all n discs are targets.
__global__ void __launch_bounds__(TW * 32, 1)
k_translate_f64_sym(const double* __restrict__ cx, const double* __restrict__ cy, int n, int p,
                    double k, const double2* __restrict__ xs, double2* __restrict__ alpha,
                    int chunks_per_cta, int per_row) {
  extern __shared__ double2 smem[];
  double2* sb = smem;                                   // [CH][32] staged source coefficients
  double* sbs = (double*)(sb + CH * 32);                // [CH][32] their re + im
  double2* sh = (double2*)(sbs + CH * 32);              // [TW][CH][HS] pair sequences
  double* shs = (double*)(sh + TW * CH * HS);           // [TW][CH][HS] their re + im
  double2* sl = (double2*)(shs + TW * CH * HS);         // [TW][32] (-1)^n xs^l_n of each warp's target
  double* sls = (double*)(sl + TW * 32);                // [TW][32] their re + im
  __shared__ double scx[CH], scy[CH];
  const int P = 2 * p + 1;
  const int r = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nb = (n + TW - 1) / TW, nc = (n + CH - 1) / CH;
  const int h = blockIdx.x / per_row;                   // the grid holds ceil(nb / 2) per_row CTAs
  const int b1 = h, b2 = nb - 1 - h;
  const int c1 = (TW * b1 + 1) / CH, c2 = (TW * b2 + 1) / CH;   // first chunk with a source > TW b
  const int len1 = max(0, nc - c1), len2 = b2 != b1 ? max(0, nc - c2) : 0;
  const int pos0 = (blockIdx.x - h * per_row) * chunks_per_cta;
  const int pos1 = min(len1 + len2, pos0 + chunks_per_cta);
  const double2* xr = xs + (size_t)r * n * P;
  double2* ar = alpha + (size_t)r * n * P;
  double2* hw = sh + (size_t)warp * CH * HS;
  double* hsw = shs + (size_t)warp * CH * HS;
  double2* slw = sl + warp * 32;
  double* slsw = sls + warp * 32;
  const double sgn = (lane & 1) ? -1.0 : 1.0;           // (-1)^nu of the lane's output
  double A = 0.0, B = 0.0, C = 0.0;
  int bcur = -1, l = 0;
  bool lvalid = false;
  double xl = 0.0, yl = 0.0;
  // the chunk loop is the same for every warp of the CTA (it depends on blockIdx only)
  for (int pos = pos0; pos < pos1; ++pos) {
    const int b = pos < len1 ? b1 : b2;
    const int c = pos < len1 ? c1 + pos : c2 + (pos - len1);
    if (b != bcur) {
      if (lvalid && lane < P) {
        atomicAdd(&ar[(size_t)l * P + lane].x, A - B);
        atomicAdd(&ar[(size_t)l * P + lane].y, C - A - B);
      }
      A = B = C = 0.0;
      bcur = b;
      l = TW * b + warp;
      lvalid = l < n;
      xl = lvalid ? cx[l] : 0.0;
      yl = lvalid ? cy[l] : 0.0;
      __syncwarp();
      double2 v = lvalid && lane < P ? xr[(size_t)l * P + lane] : make_double2(0.0, 0.0);
      if (lane & 1) v = make_double2(-v.x, -v.y);
      slw[lane] = v;
      slsw[lane] = v.x + v.y;
      __syncwarp();
    }
    const int j0c = c * CH;
    const int cnt = min(CH, n - j0c);
    __syncthreads();
    for (int i = threadIdx.x; i < cnt * P; i += blockDim.x) {
      const int s = i / P, q = i - s * P;
      const double2 v = xr[(size_t)(j0c + s) * P + q];
      sb[s * 32 + q] = v;
      sbs[s * 32 + q] = v.x + v.y;
    }
    if (threadIdx.x < cnt) {
      scx[threadIdx.x] = cx[j0c + threadIdx.x];
      scy[threadIdx.x] = cy[j0c + threadIdx.x];
    }
    __syncthreads();
    if (lane < cnt) {
      double2* hq = hw + lane * HS;
      double* hsm = hsw + lane * HS;
      if (lvalid && j0c + lane > l) {
        hankel_sequence_f64(xl - scx[lane], yl - scy[lane], k, p, hq, hsm);
      } else {
        for (int q = 0; q <= 4 * p; ++q) {
          hq[q] = make_double2(0.0, 0.0);
          hsm[q] = 0.0;
        }
      }
    }
    __syncwarp();
    if (lvalid && lane < P) {
      for (int s = 0; s < cnt; ++s) {                   // l <- m
        const double2* hs = hw + s * HS + 2 * p - lane;   // hs[q] = h_{n - nu}, n = q - p
        const double* hss = hsw + s * HS + 2 * p - lane;
        const double2* bs = sb + s * 32;
        const double* bss = sbs + s * 32;
        for (int q = 0; q < P; ++q) {
          const double2 hv = hs[q], bv = bs[q];
          A = fma(hv.x, bv.x, A);
          B = fma(hv.y, bv.y, B);
          C = fma(hss[q], bss[q], C);
        }
      }
      for (int s = max(0, l + 1 - j0c); s < cnt; ++s) {  // m <- l, sources m = j0c + s > l
        const double2* hs = hw + s * HS + 2 * p - lane;
        const double* hss = hsw + s * HS + 2 * p - lane;
        double Ar = 0.0, Br = 0.0, Cr = 0.0;
        for (int q = 0; q < P; ++q) {
          const double2 hv = hs[q], bv = slw[q];
          Ar = fma(hv.x, bv.x, Ar);
          Br = fma(hv.y, bv.y, Br);
          Cr = fma(hss[q], slsw[q], Cr);
        }
        double2* o = &ar[(size_t)(j0c + s) * P + lane];
        atomicAdd(&o->x, sgn * (Ar - Br));
        atomicAdd(&o->y, sgn * (Cr - Ar - Br));
      }
    }
  }
  if (lvalid && lane < P) {
    atomicAdd(&ar[(size_t)l * P + lane].x, A - B);
    atomicAdd(&ar[(size_t)l * P + lane].y, C - A - B);
  }
}

// ---------------------------------------------------------------------------------------------
// Plane-wave tables of the discs (Thm 5.2 / Lemma 5.1 factors that depend on the disc position)
// ---------------------------------------------------------------------------------------------
__global__ void k_etables(const double* __restrict__ cx, const double* __restrict__ cy, int n,
                          const double2* __restrict__ lam, const double2* __restrict__ g2, int ns,
                          double d, double2* __restrict__ eagg, double2* __restrict__ edis) {
  const long long total = (long long)ns * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int v = (int)(i / n), j = (int)(i - (long long)v * n);
    const double2 L = lam[v], g = g2[v];
    const double x = cx[j], y = cy[j], yd = y + d;
    // -i lambda x = (lam.y x) + i (-lam.x x)
    const double ax = L.y * x, ay = -L.x * x;
    eagg[(size_t)v * n + j] = cexp_(g.x * y + ax, g.y * y + ay);               // exp(g2 y - i l x)
    eagg[(size_t)(ns + v) * n + j] = cexp_(-g.x * yd + ax, -g.y * yd + ay);   // exp(-g2(y+d) - i l x)
    edis[(size_t)j * 2 * ns + v] = cexp_(g.x * y - ax, g.y * y - ay);         // exp(g2 y + i l x)
    edis[(size_t)j * 2 * ns + ns + v] = cexp_(-g.x * yd - ax, -g.y * yd - ay);
  }
}

// ---------------------------------------------------------------------------------------------
// C[r][m][n] += sum_k A[m][k] B[r][k][n]  (complex FP64, split-K with atomics)
// ---------------------------------------------------------------------------------------------
constexpr int GT = 32;

__global__ void __launch_bounds__(256)
k_zgemm_rows(const double2* __restrict__ A, int M, int K, const double2* __restrict__ B,
             double2* __restrict__ C, int P, int kchunk) {
  __shared__ double2 As[GT][GT + 1];
  __shared__ double2 Bs[GT][GT + 1];
  const int r = blockIdx.y;
  const int m0 = blockIdx.x * GT;
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(K, kbeg + kchunk);
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const double2* Br = B + (size_t)r * K * P;
  double2 acc[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) acc[q] = make_double2(0.0, 0.0);
  for (int k0 = kbeg; k0 < kend; k0 += GT) {
    for (int e = threadIdx.x; e < GT * GT; e += blockDim.x) {
      const int i = e >> 5, kk = e & 31;
      const int m = m0 + i, kx = k0 + kk;
      As[i][kk] = (m < M && kx < kend) ? A[(size_t)m * K + kx] : make_double2(0.0, 0.0);
      const int nn = kk;   // reuse e for B: row i is k, column kk is n
      Bs[i][nn] = (k0 + i < kend && nn < P) ? Br[(size_t)(k0 + i) * P + nn] : make_double2(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < GT; ++kk) {
      const double2 b = Bs[kk][tx];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = cfma(As[ty + 8 * q][kk], b, acc[q]);
    }
    __syncthreads();
  }
  if (tx < P) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int m = m0 + ty + 8 * q;
      if (m < M) {
        double2* c = C + ((size_t)r * M + m) * P + tx;
        atomicAdd(&c->x, acc[q].x);
        atomicAdd(&c->y, acc[q].y);
      }
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Per-node stage: order dots (aggregate epilogue), reflection (Eq. "sommerfeldsys" closed form),
// and the disaggregate's right operand V = U * sigma.
// G, V: [r][2ns][P]; pq, sig: [r][2][ns].
// ---------------------------------------------------------------------------------------------
__global__ void k_node_stage(int ns, int P, int nrhs, const double2* __restrict__ G,
                             const double2* __restrict__ fagg, const double2* __restrict__ pq_in,
                             const double2* __restrict__ refl, const double2* __restrict__ udis,
                             double2* __restrict__ pq_out, double2* __restrict__ sig_out,
                             double2* __restrict__ V) {
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (gw >= ns * nrhs) return;
  const int r = gw / ns, v = gw - r * ns;
  double2 Pp, Qm;
  if (G) {
    double2 a = make_double2(0.0, 0.0), b = make_double2(0.0, 0.0);
    if (lane < P) {
      a = cmul(fagg[(size_t)v * P + lane], G[((size_t)r * 2 * ns + v) * P + lane]);
      b = cmul(fagg[(size_t)(ns + v) * P + lane], G[((size_t)r * 2 * ns + ns + v) * P + lane]);
    }
    Pp = warp_sum(a);
    Qm = warp_sum(b);
  } else {
    Pp = pq_in[(size_t)r * 2 * ns + v];
    Qm = pq_in[(size_t)r * 2 * ns + ns + v];
  }
  if (pq_out && lane == 0) {
    pq_out[(size_t)r * 2 * ns + v] = Pp;
    pq_out[(size_t)r * 2 * ns + ns + v] = Qm;
  }
  if (!refl) return;
  const double2 a11 = refl[4 * v], a12 = refl[4 * v + 1], a21 = refl[4 * v + 2], a22 = refl[4 * v + 3];
  const double2 sp = cadd(cmul(a11, Pp), cmul(a12, Qm));
  const double2 sm = cadd(cmul(a21, Pp), cmul(a22, Qm));
  if (sig_out && lane == 0) {
    sig_out[(size_t)r * 2 * ns + v] = sp;
    sig_out[(size_t)r * 2 * ns + ns + v] = sm;
  }
  if (V && lane < P) {
    V[((size_t)r * 2 * ns + v) * P + lane] = cmul(udis[(size_t)v * P + lane], sp);
    V[((size_t)r * 2 * ns + ns + v) * P + lane] = cmul(udis[(size_t)(ns + v) * P + lane], sm);
  }
}

__global__ void k_sigma_to_v(int ns, int P, int nrhs, const double2* __restrict__ sig,
                             const double2* __restrict__ udis, double2* __restrict__ V) {
  const long long total = (long long)nrhs * 2 * ns * P;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(i % P);
    const long long rv = i / P;            // r * 2ns + row
    const int row = (int)(rv % (2 * ns));
    V[i] = cmul(udis[(size_t)row * P + q], sig[rv]);
  }
}

// sigma2+- of the particle-free layered field of each line source (Eq. "sommerfeldsys"):
// I = exp(-g1 y0 - i lambda (x0 - xc)); sigma2+ = t1 I, sigma2- = t2 I.   sig: [src][2][ns]
__global__ void k_incident_sigma(int ns, int nsrc, const double* __restrict__ src, double xc,
                                 const double2* __restrict__ lam, const double2* __restrict__ g1,
                                 const double2* __restrict__ inc, double2* __restrict__ sig) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ns * nsrc) return;
  const int s = i / ns, v = i - s * ns;
  const double sx0 = src[2 * s] - xc, sy0 = src[2 * s + 1];
  const double2 L = lam[v], g = g1[v];
  const double2 I = cexp_(-g.x * sy0 + L.y * sx0, -g.y * sy0 - L.x * sx0);
  sig[(size_t)s * 2 * ns + v] = cmul(inc[2 * v], I);
  sig[(size_t)s * 2 * ns + ns + v] = cmul(inc[2 * v + 1], I);
}

__global__ void k_combine(const double2* __restrict__ x, const double2* __restrict__ alpha,
                          const double2* __restrict__ s_out, double2* __restrict__ y,
                          long long total, int P, int alpha_only) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const double2 a = alpha[i];
    if (alpha_only) {
      y[i] = a;
    } else {
      const double2 sa = cmul(s_out[i % P], a);
      const double2 xv = x[i];
      y[i] = make_double2(xv.x - sa.x, xv.y - sa.y);
    }
  }
}

// Field in layer 1 (Eq. "layer1"): one warp per target; sigma1 per node from the particle sums
// P+, Q- (pq, [2][ns]) and the incident density.
__global__ void k_field(int ns, int ntgt, const double* __restrict__ tgt, double xc,
                        const double2* __restrict__ lam, const double2* __restrict__ g1,
                        const double2* __restrict__ ft, const double2* __restrict__ pq,
                        const double* __restrict__ src, double k1, int which,
                        double2* __restrict__ out) {
  const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (t >= ntgt) return;
  const double xt = tgt[2 * t] - xc, yt = tgt[2 * t + 1];
  const double sx0 = src[0] - xc, sy0 = src[1];
  double2 acc = make_double2(0.0, 0.0);
  for (int v = lane; v < ns; v += 32) {
    const double2 L = lam[v], g = g1[v];
    const double2 I = cexp_(-g.x * sy0 + L.y * sx0, -g.y * sy0 - L.x * sx0);
    const double2 Pp = pq ? pq[v] : make_double2(0.0, 0.0);
    const double2 Qm = pq ? pq[ns + v] : make_double2(0.0, 0.0);
    // sigma_1 = f_I I + f_P P + f_Q Q (the layer response of every interface, per node)
    double2 s1 = cadd(cmul(ft[4 * v + 1], Pp), cmul(ft[4 * v + 2], Qm));
    if (which != LSMS_FIELD_PARTICLE) s1 = cadd(s1, cmul(ft[4 * v], I));
    const double2 ex = cexp_(-g.x * yt - L.y * xt, -g.y * yt + L.x * xt);   // exp(-g1 y + i l x)
    acc = cfma(cmul(ft[4 * v + 3], s1), ex, acc);
  }
  acc = warp_sum(acc);
  if (lane == 0) {
    if (which == LSMS_FIELD_TOTAL) {
      const double z = k1 * hypot(tgt[2 * t] - src[0], tgt[2 * t + 1] - src[1]);
      acc.x += -0.25 * y0(z);      // (i/4)(J0 + i Y0)
      acc.y += 0.25 * j0(z);
    }
    out[t] = acc;
  }
}

inline int grid_for(long long total, int block) {
  long long g = (total + block - 1) / block;
  if (g > 152LL * 32) g = 152LL * 32;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

// ---------------------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------------------
void launch_scale_in(const double2* x, const double* scale, double2* xs, int nrhs, int n, int P,
                     cudaStream_t st) {
  const long long total = (long long)nrhs * n * P;
  if (total == 0) return;
  k_scale_in<<<grid_for(total, 256), 256, 0, st>>>(x, scale, xs, total, P);
}

void launch_translate_f64(const double* cx, const double* cy, int n, int p, double k,
                          const double2* xs, double2* alpha, int nrhs, cudaStream_t st, int row0,
                          int nrows) {
  if (nrows < 0) nrows = n - row0;
  if (n == 0 || nrhs == 0 || nrows <= 0) return;
  const size_t smem = (size_t)(CH * 32 + TW * CH * HS) * (sizeof(double2) + sizeof(double));
  static std::once_flag attr;
  std::call_once(attr, [smem] {
    cudaFuncSetAttribute(k_translate_f64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  if (row0 == 0 && nrows == n && n > CH) {
    // all rows of more than one chunk: one sequence per unordered pair, runs of chunks sized for
    // about 24 waves of one CTA per SM (with a single chunk both kernels launch the same CTAs, and
    // the one-way kernel's single contraction pass has less latency)
    const size_t smem_sym = smem + (size_t)TW * 32 * (sizeof(double2) + sizeof(double));
    static std::once_flag attr_sym;
    std::call_once(attr_sym, [smem_sym] {
      cudaFuncSetAttribute(k_translate_f64_sym, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_sym);
    });
    const int nb = (n + TW - 1) / TW, nc = (n + CH - 1) / CH, H = (nb + 1) / 2;
    long long total = 0;
    int dmax = 0;
    for (int h = 0; h < H; ++h) {
      const int b2 = nb - 1 - h;
      const int d = std::max(0, nc - (TW * h + 1) / CH) + (b2 != h ? std::max(0, nc - (TW * b2 + 1) / CH) : 0);
      total += d;
      dmax = std::max(dmax, d);
    }
    const int run = (int)std::max<long long>(1, (total + 152 * 24 - 1) / (152 * 24));
    const int per_row = std::max(1, (dmax + run - 1) / run);
    cudaMemsetAsync(alpha, 0, (size_t)nrhs * n * (2 * p + 1) * sizeof(double2), st);
    dim3 grid(H * per_row, nrhs);
    k_translate_f64_sym<<<grid, TW * 32, smem_sym, st>>>(cx, cy, n, p, k, xs, alpha, run, per_row);
    return;
  }
  dim3 grid((nrows + TW - 1) / TW, nrhs);
  k_translate_f64<<<grid, TW * 32, smem, st>>>(cx, cy, n, p, k, xs, alpha, row0, nrows);
}

void launch_etables(const double* cx, const double* cy, int n, const double2* lam,
                    const double2* g2, int ns, double d, double2* eagg, double2* edis,
                    cudaStream_t st) {
  const long long total = (long long)ns * n;
  if (total == 0) return;
  k_etables<<<grid_for(total, 256), 256, 0, st>>>(cx, cy, n, lam, g2, ns, d, eagg, edis);
}

void launch_zgemm_rows(const double2* A, int M, int K, const double2* B, double2* C, int P,
                       int nrhs, cudaStream_t st) {
  if (M == 0 || K == 0 || nrhs == 0) return;
  const int mt = (M + GT - 1) / GT;
  const int kt = (K + GT - 1) / GT;
  int split = (152 * 4 + mt * nrhs - 1) / (mt * nrhs);
  if (split > kt) split = kt;
  if (split < 1) split = 1;
  const int kchunk = ((kt + split - 1) / split) * GT;
  split = (K + kchunk - 1) / kchunk;
  dim3 grid(mt, nrhs, split);
  k_zgemm_rows<<<grid, 256, 0, st>>>(A, M, K, B, C, P, kchunk);
}

void launch_node_stage(int ns, int P, int nrhs, const double2* G, const double2* fagg,
                       const double2* pq_in, const double2* refl, const double2* udis,
                       double2* pq_out, double2* sig_out, double2* V, cudaStream_t st) {
  const long long threads = (long long)ns * nrhs * 32;
  if (threads == 0) return;
  k_node_stage<<<(int)((threads + 255) / 256), 256, 0, st>>>(ns, P, nrhs, G, fagg, pq_in, refl,
                                                             udis, pq_out, sig_out, V);
}

void launch_sigma_to_v(int ns, int P, int nrhs, const double2* sig, const double2* udis,
                       double2* V, cudaStream_t st) {
  const long long total = (long long)nrhs * 2 * ns * P;
  if (total == 0) return;
  k_sigma_to_v<<<grid_for(total, 256), 256, 0, st>>>(ns, P, nrhs, sig, udis, V);
}

// y = x - D(-theta_j) M D(theta_j) alpha for every (right-hand side, particle): one warp per pair,
// lane = order (alpha_n e^{i n theta} broadcast by shuffles, M^T staged in shared memory so that a
// warp reads one contiguous row per source order).
__global__ void k_scatter_dense(const double2* __restrict__ x, const double2* __restrict__ alpha,
                                const double2* __restrict__ mt, const double* __restrict__ theta,
                                long long units, int n, int P, double2* __restrict__ y) {
  extern __shared__ double2 s_mt[];
  for (int i = threadIdx.x; i < P * P; i += blockDim.x) s_mt[i] = mt[i];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int p = (P - 1) / 2;
  const long long stride = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long u = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < units; u += stride) {
    double sn = 0.0, cs = 1.0;
    if (theta) sincos((double)(lane - p) * theta[u % n], &sn, &cs);
    double2 a = make_double2(0.0, 0.0);
    if (lane < P) a = cmul(alpha[u * P + lane], make_double2(cs, sn));
    double2 acc = make_double2(0.0, 0.0);
    for (int q = 0; q < P; ++q) {
      const double2 b = make_double2(__shfl_sync(0xffffffffu, a.x, q), __shfl_sync(0xffffffffu, a.y, q));
      if (lane < P) acc = cfma(s_mt[q * P + lane], b, acc);
    }
    if (lane < P) {
      const double2 v = cmul(acc, make_double2(cs, -sn));
      if (x) {
        const double2 xv = x[u * P + lane];
        y[u * P + lane] = make_double2(xv.x - v.x, xv.y - v.y);
      } else {
        y[u * P + lane] = v;
      }
    }
  }
}

void launch_scatter_dense(const double2* x, const double2* alpha, const double2* mt, const double* theta,
                          int nrhs, int n, int P, double2* y, cudaStream_t st) {
  const long long units = (long long)nrhs * n;
  if (units == 0) return;
  long long blocks = (units + 7) / 8;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_scatter_dense<<<(int)blocks, 256, (size_t)P * P * sizeof(double2), st>>>(x, alpha, mt, theta, units, n, P, y);
}

void launch_incident_sigma(int ns, int nsrc, const double* src, double xc, const double2* lam,
                           const double2* g1, const double2* inc, double2* sig, cudaStream_t st) {
  const int total = ns * nsrc;
  if (total == 0) return;
  k_incident_sigma<<<(total + 255) / 256, 256, 0, st>>>(ns, nsrc, src, xc, lam, g1, inc, sig);
}

void launch_combine(const double2* x, const double2* alpha, const double2* s_out, double2* y,
                    int nrhs, int n, int P, int alpha_only, cudaStream_t st) {
  const long long total = (long long)nrhs * n * P;
  if (total == 0) return;
  k_combine<<<grid_for(total, 256), 256, 0, st>>>(x, alpha, s_out, y, total, P, alpha_only);
}

void launch_field(int ns, int ntgt, const double* tgt, double xc, const double2* lam,
                  const double2* g1, const double2* fieldtab, const double2* pq, const double* src,
                  double k1, int which, double2* out, cudaStream_t st) {
  if (ntgt == 0) return;
  const long long threads = (long long)ntgt * 32;
  k_field<<<(int)((threads + 127) / 128), 128, 0, st>>>(ns, ntgt, tgt, xc, lam, g1, fieldtab, pq, src,
                                                        k1, which, out);
}
