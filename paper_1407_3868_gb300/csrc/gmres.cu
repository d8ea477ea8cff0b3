// Device-resident GMRES (Saad-Schultz, cited in Sec. 3.2 of the paper) on the scaled,
// preconditioned disc system (I - D S (T + R) D^{-1}) b = D S a_inc, D = diag |H_n(k2 R)|, for one
// or many right-hand sides at once, and the FP64 iterative-refinement loop of the mixed solve.
//
// Several systems (one per line source) iterate in lockstep: the Krylov basis is laid out
// [iteration][system][N P], so every Arnoldi step is one multi-right-hand-side application of the
// operator.  Each system keeps its own Hessenberg matrix, Givens rotations and residual estimate on
// the device; classical Gram-Schmidt takes a second pass only when the first one cancels much of the
// new vector.  The iteration runs on the device as one graph launch: a conditional while node
// whose body is one Arnoldi step of all systems followed by the stopping test, which records for
// each system the iteration at which it met its tolerance (later iterations are discarded by solving
// its least-squares problem on that many columns only) and ends the loop when none is left.  Where
// that graph cannot be built, the host launches the captured step once per step and reads the
// residual estimates two iterations late (pinned ring + events), so the next steps stay queued.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "lsms_internal.h"
#include "lsms_ops.h"

namespace {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cjmul(double2 a, double2 b) {   // conj(a) b
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double2 warp_sum(double2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}

// Krylov basis arithmetic: FP64 (double2 basis) for FP64 solves; FP32 storage and FP32 products
// (float2 basis) for the inner solves of the mixed refinement, whose tolerances are >= 1e-5.  The
// FP64 pipe of this GPU is narrow enough that FP64 Gram-Schmidt products are arithmetic-bound near
// 1-2 TB/s; in FP32 they are bound by the (halved) memory traffic.  Reductions across threads and
// CTAs, the Hessenberg matrix, the rotations and the iterate stay FP64.
template <typename T> struct Vec2;
template <> struct Vec2<double> { using type = double2; };
template <> struct Vec2<float> { using type = float2; };
template <typename T> using vec2 = typename Vec2<T>::type;
template <typename T> __device__ __forceinline__ vec2<T> mk2(double x, double y);
template <> __device__ __forceinline__ double2 mk2<double>(double x, double y) { return make_double2(x, y); }
template <> __device__ __forceinline__ float2 mk2<float>(double x, double y) { return make_float2((float)x, (float)y); }
template <typename V2> __device__ __forceinline__ double2 to_d2(V2 v) { return make_double2(v.x, v.y); }
template <typename V2> __device__ __forceinline__ V2 cjmul_t(V2 a, V2 b) {   // conj(a) b
  V2 r;
  r.x = a.x * b.x + a.y * b.y;
  r.y = a.x * b.y - a.y * b.x;
  return r;
}

struct GmState {
  double beta0;   // ||r0||
  double ref;     // ||rhs||: residuals are reported relative to it
  double res;     // |g_{k+1}| / ||rhs||
  double hn;      // ||w|| of the last Arnoldi step
  double inv;     // scale for the next basis vector
  int flag;       // 1: non-finite value seen
  int reorth;     // 1: the current Arnoldi step needs a second Gram-Schmidt pass
};

constexpr int DOT_T = 2048;    // elements of w staged per CTA
constexpr int DOT_GY = 8;      // groups of 8 vectors in the grid; a CTA loops over every 8th group
constexpr int GIVENS_MAX = 4096;

// System b = blockIdx.z:  out[b][i] += sum_t conj(V[i][b][t]) w[b][t] for i < nv, and, with
// self_norm, out[b][nv] += ||w_b||^2 (out pre-zeroed).  nv = nv0 (+ *kp when kp is given, so that a
// captured graph follows the Arnoldi step).  V slots are ldv apart; system b occupies elements
// off[b] .. off[b + 1] of a slot (systems may differ in length: the layouts of a batch).  With a
// gate the kernel does nothing unless system b needs a second Gram-Schmidt pass.
// A CTA stages a chunk of DOT_T elements of w in shared memory; each warp takes one basis vector
// at a time (vectors blockIdx.y * 8 + warp, stepping gridDim.y * 8) with 8 loads in flight per lane
// and reduces it with shuffles only, so the multi-dot streams the basis at memory speed.
template <typename T>
__global__ void __launch_bounds__(256)
k_mdot(const vec2<T>* __restrict__ V, long long ldv, int nv0, const int* __restrict__ kp,
       int self_norm, const double2* __restrict__ w, const long long* __restrict__ off,
       double2* __restrict__ out, int out_stride, const GmState* __restrict__ gate) {
  using V2 = vec2<T>;
  constexpr int U = 8;
  const int b = blockIdx.z;
  if (gate && !gate[b].reorth) return;
  const int nv = nv0 + (kp ? *kp : 0);
  const int ntot = nv + (self_norm ? 1 : 0);
  const long long L = off[b + 1] - off[b];
  const long long c0 = blockIdx.x * (long long)DOT_T;
  if (c0 >= L || (int)blockIdx.y * 8 >= ntot) return;
  const int cnt = (int)min((long long)DOT_T, L - c0);
  V += off[b] + c0;
  w += off[b] + c0;
  out += (long long)b * out_stride;
  __shared__ V2 ws[DOT_T];
  for (int i = threadIdx.x; i < DOT_T; i += blockDim.x) {
    const double2 u = i < cnt ? w[i] : make_double2(0.0, 0.0);
    ws[i] = mk2<T>(u.x, u.y);
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = blockIdx.y * 8 + warp; i < ntot; i += gridDim.y * 8) {
    T ax = 0, ay = 0, bx = 0, by = 0;
    if (i < nv) {
      const V2* vi = V + (long long)i * ldv;
      for (int t = lane; t < DOT_T; t += 32 * U) {
        V2 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int tt = t + 32 * u;
          v[u] = tt < cnt ? vi[tt] : mk2<T>(0.0, 0.0);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const V2 c = cjmul_t(v[u], ws[t + 32 * u]);
          if (u & 1) {
            bx += c.x;
            by += c.y;
          } else {
            ax += c.x;
            ay += c.y;
          }
        }
      }
    } else {                                        // ||w||^2
      for (int t = lane; t < cnt; t += 32) ax += ws[t].x * ws[t].x + ws[t].y * ws[t].y;
    }
    const double2 s = warp_sum(make_double2((double)ax + (double)bx, (double)ay + (double)by));
    if (lane == 0) {
      atomicAdd(&out[i].x, s.x);
      atomicAdd(&out[i].y, s.y);
    }
  }
}

// System b = blockIdx.y:  w[b][t] += sign sum_{i < nv_b} V[i][b][t] h[b][i] over the system's
// elements off[b] .. off[b + 1].  nv_b = nv, or nv_arr[b] when given; with a gate only when system b
// needs a second pass.
template <typename T>
__global__ void __launch_bounds__(256)
k_maxpy(const vec2<T>* __restrict__ V, long long ldv, int nv, const int* __restrict__ nv_arr,
        const int* __restrict__ kp, const double2* __restrict__ h, int h_stride,
        double2* __restrict__ w, const long long* __restrict__ off, double sign,
        const GmState* __restrict__ gate) {
  using V2 = vec2<T>;
  const int b = blockIdx.y;
  if (gate && !gate[b].reorth) return;
  const long long L = off[b + 1] - off[b];
  if (blockIdx.x * (long long)blockDim.x >= L) return;
  if (nv_arr) nv = nv_arr[b];
  if (kp) nv += *kp;
  V += off[b];
  w += off[b];
  h += (long long)b * h_stride;
  __shared__ V2 hs[256];
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  V2 a0 = mk2<T>(0.0, 0.0), a1 = mk2<T>(0.0, 0.0);
  for (int i0 = 0; i0 < nv; i0 += 256) {
    const int c = min(256, nv - i0);
    __syncthreads();
    if (threadIdx.x < c) {
      const double2 u = h[i0 + threadIdx.x];
      hs[threadIdx.x] = mk2<T>(u.x, u.y);
    }
    __syncthreads();
    if (t < L) {
      int i = 0;
      for (; i + 3 < c; i += 4) {
        const V2 v0 = V[(long long)(i0 + i) * ldv + t];
        const V2 v1 = V[(long long)(i0 + i + 1) * ldv + t];
        const V2 v2 = V[(long long)(i0 + i + 2) * ldv + t];
        const V2 v3 = V[(long long)(i0 + i + 3) * ldv + t];
        const V2 h0 = hs[i], h1 = hs[i + 1], h2 = hs[i + 2], h3 = hs[i + 3];
        a0.x = fma(v0.x, h0.x, fma(-v0.y, h0.y, a0.x));
        a0.y = fma(v0.x, h0.y, fma(v0.y, h0.x, a0.y));
        a1.x = fma(v1.x, h1.x, fma(-v1.y, h1.y, a1.x));
        a1.y = fma(v1.x, h1.y, fma(v1.y, h1.x, a1.y));
        a0.x = fma(v2.x, h2.x, fma(-v2.y, h2.y, a0.x));
        a0.y = fma(v2.x, h2.y, fma(v2.y, h2.x, a0.y));
        a1.x = fma(v3.x, h3.x, fma(-v3.y, h3.y, a1.x));
        a1.y = fma(v3.x, h3.y, fma(v3.y, h3.x, a1.y));
      }
      for (; i < c; ++i) {
        const V2 v0 = V[(long long)(i0 + i) * ldv + t];
        const V2 h0 = hs[i];
        a0.x = fma(v0.x, h0.x, fma(-v0.y, h0.y, a0.x));
        a0.y = fma(v0.x, h0.y, fma(v0.y, h0.x, a0.y));
      }
    }
  }
  if (t < L) {
    w[t].x += sign * ((double)a0.x + (double)a1.x);
    w[t].y += sign * ((double)a0.y + (double)a1.y);
  }
}

// After the first Gram-Schmidt pass of system b = blockIdx.x: h1[0..k] = V^H w, h1[k+1] = ||w||^2.
// The first pass removes ||h1||^2 from ||w||^2; if more than about half of it goes
// (||w'|| < 0.7 ||w||), cancellation may have left w' not orthogonal enough and a second pass runs.
__global__ void __launch_bounds__(32) k_gm_prep(const int* __restrict__ kp, const double2* __restrict__ h1,
                                                int stride, GmState* __restrict__ st) {
  const int k = *kp;
  h1 += (long long)blockIdx.x * stride;
  double s = 0.0;
  for (int i = threadIdx.x; i <= k; i += 32) s += h1[i].x * h1[i].x + h1[i].y * h1[i].y;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (threadIdx.x == 0) {
    const double a = h1[k + 1].x;
    st[blockIdx.x].reorth = (a - s < 0.49 * a) ? 1 : 0;
  }
}

// Column k of system b = blockIdx.x: H[0..k][k] = h1 + h2, H[k+1][k] = ||w_final||; apply the
// previous Givens rotations, form the new one, update g and the residual estimate.  The lanes
// stage the column and the rotations in shared memory, lane 0 sweeps them.
__global__ void __launch_bounds__(32)
k_gm_column(const int* __restrict__ kp, const double2* __restrict__ h1, const double2* __restrict__ h2,
            int stride, double2* __restrict__ H, long long hstride, int ldh, double2* __restrict__ cs,
            double2* __restrict__ sn, double2* __restrict__ g, GmState* __restrict__ st) {
  extern __shared__ double2 sm[];
  const int k = *kp;
  const int b = blockIdx.x;
  h1 += (long long)b * stride;
  h2 += (long long)b * stride;
  cs += (long long)b * stride;
  sn += (long long)b * stride;
  g += (long long)b * stride;
  H += (long long)b * hstride;
  GmState* s = st + b;
  double2* col = sm;                    // [k + 2]
  double2* c_s = sm + (k + 2);          // [k]
  double2* s_s = c_s + k;               // [k]
  const int lane = threadIdx.x;
  for (int i = lane; i <= k; i += 32) col[i] = make_double2(h1[i].x + h2[i].x, h1[i].y + h2[i].y);
  for (int i = lane; i < k; i += 32) {
    c_s[i] = cs[i];
    s_s[i] = sn[i];
  }
  // ||w_final||^2 = (second pass ? ||w'||^2 - ||h2||^2 : ||w||^2 - ||h1||^2)
  const double2* hl = s->reorth ? h2 : h1;
  double s2 = 0.0;
  for (int i = lane; i <= k; i += 32) s2 += hl[i].x * hl[i].x + hl[i].y * hl[i].y;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  __syncwarp();
  if (lane == 0) {
    const double hn = sqrt(fmax(hl[k + 1].x - s2, 0.0));
    s->hn = hn;
    s->inv = hn > 0.0 ? 1.0 / hn : 0.0;
    col[k + 1] = make_double2(hn, 0.0);
    for (int i = 0; i < k; ++i) {
      const double2 a = col[i], bb = col[i + 1];
      const double2 ci = c_s[i], si = s_s[i];
      // [conj(c) conj(s); -s c] [a; b]
      const double2 t = make_double2(cjmul(ci, a).x + cjmul(si, bb).x, cjmul(ci, a).y + cjmul(si, bb).y);
      const double2 u = make_double2(-cmul(si, a).x + cmul(ci, bb).x, -cmul(si, a).y + cmul(ci, bb).y);
      col[i] = t;
      col[i + 1] = u;
    }
    const double2 a = col[k];
    const double r = hypot(hypot(a.x, a.y), hn);
    double2 c, sg;
    if (r > 0.0) {
      c = make_double2(a.x / r, a.y / r);
      sg = make_double2(hn / r, 0.0);
    } else {
      c = make_double2(1.0, 0.0);
      sg = make_double2(0.0, 0.0);
    }
    cs[k] = c;
    sn[k] = sg;
    col[k] = make_double2(r, 0.0);
    col[k + 1] = make_double2(0.0, 0.0);
    const double2 gk = g[k];
    g[k] = cjmul(c, gk);
    g[k + 1] = make_double2(-cmul(sg, gk).x, -cmul(sg, gk).y);
    const double res = hypot(g[k + 1].x, g[k + 1].y) / s->ref;
    s->res = res;
    if (!isfinite(res) || !isfinite(hn)) s->flag = 1;
  }
  __syncwarp();
  double2* Hc = H + (long long)k * ldh;
  for (int i = lane; i <= k + 1; i += 32) Hc[i] = col[i];
}

// Back substitution of system b = blockIdx.x: H[0..k_b)[0..k_b) y = g, one warp.
__global__ void k_gm_backsolve(const int* __restrict__ kk, const double2* __restrict__ H,
                               long long hstride, int ldh, const double2* __restrict__ g, int stride,
                               double2* __restrict__ y) {
  const int b = blockIdx.x;
  const int k = kk[b];
  H += (long long)b * hstride;
  g += (long long)b * stride;
  y += (long long)b * stride;
  const int lane = threadIdx.x;
  for (int i = k - 1; i >= 0; --i) {
    double2 s = make_double2(0.0, 0.0);
    for (int j = i + 1 + lane; j < k; j += 32) {
      const double2 c = cmul(H[(long long)j * ldh + i], y[j]);
      s.x += c.x;
      s.y += c.y;
    }
    s = warp_sum(s);
    if (lane == 0) {
      const double2 num = make_double2(g[i].x - s.x, g[i].y - s.y);
      const double2 d = H[(long long)i * ldh + i];
      const double dd = d.x * d.x + d.y * d.y;
      y[i] = dd > 0.0 ? make_double2((num.x * d.x + num.y * d.y) / dd, (num.y * d.x - num.x * d.y) / dd)
                      : make_double2(0.0, 0.0);
    }
    __syncwarp();
  }
}

// System b = blockIdx.y: dst[b] = src[b] * st[b].inv
template <typename T>
__global__ void k_scale_by(vec2<T>* __restrict__ dst, const double2* __restrict__ src,
                           const GmState* __restrict__ st, const long long* __restrict__ off) {
  const int b = blockIdx.y;
  const double s = st[b].inv;
  const long long L = off[b + 1] - off[b];
  dst += off[b];
  src += off[b];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < L;
       t += (long long)gridDim.x * blockDim.x) {
    const double2 v = src[t];
    dst[t] = mk2<T>(v.x * s, v.y * s);
  }
}

// X[b] = V[k][b] (the operator's fixed input buffer)
template <typename T>
__global__ void k_copy_slot(double2* __restrict__ X, const vec2<T>* __restrict__ V, long long slot,
                            const int* __restrict__ kp) {
  const vec2<T>* src = V + (long long)(*kp) * slot;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < slot;
       t += (long long)gridDim.x * blockDim.x)
    X[t] = to_d2(src[t]);
}

// V[k + 1][b] = W[b] * st[b].inv   (system b = blockIdx.y)
template <typename T>
__global__ void k_scale_into_slot(vec2<T>* __restrict__ V, long long slot, const double2* __restrict__ W,
                                  const GmState* __restrict__ st, const long long* __restrict__ off,
                                  const int* __restrict__ kp) {
  const int b = blockIdx.y;
  const double s = st[b].inv;
  const long long L = off[b + 1] - off[b];
  vec2<T>* dst = V + (long long)(*kp + 1) * slot + off[b];
  const double2* src = W + off[b];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < L;
       t += (long long)gridDim.x * blockDim.x) {
    const double2 v = src[t];
    dst[t] = mk2<T>(v.x * s, v.y * s);
  }
}

// ring[k mod ring_slots][b] = st[b] (host-mapped memory), then k += 1.  One block.
__global__ void k_gm_snapshot(const GmState* __restrict__ st, int nb, GmState* __restrict__ ring,
                              int ring_slots, int* __restrict__ kp) {
  const int k = *kp;
  GmState* dst = ring + (size_t)(k % ring_slots) * nb;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) dst[b] = st[b];
  __syncthreads();
  if (threadIdx.x == 0) *kp = k + 1;
}

// The stopping test of the graph-resident loop, after the step counter has counted this Arnoldi
// step (k steps done): a system that met its tolerance, broke down (hn = 0) or saw a non-finite
// value keeps k as its iteration count; the loop's condition becomes 0 when no system is left, a
// non-finite value appeared or k reached maxiter.  hist (one system): its residual after each step.
// One block.
__global__ void k_gm_decide(const GmState* __restrict__ st, int nb, const double* __restrict__ tol,
                            int* __restrict__ kdone, double* __restrict__ res, const int* __restrict__ kp,
                            int maxiter, int* __restrict__ nonfinite, int* __restrict__ guard,
                            double* __restrict__ hist, int hist_cap, cudaGraphConditionalHandle cond) {
  __shared__ int active, bad;
  if (threadIdx.x == 0) {
    active = 0;
    bad = 0;
  }
  __syncthreads();
  const int k = *kp;
  const int runs = *guard + 1;                    // executions of this test: bounds the loop by itself
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    if (kdone[b] >= 0) continue;
    const GmState sb = st[b];
    res[b] = sb.res;
    if (sb.flag) atomicOr(&bad, 1);
    if (sb.flag || sb.res <= tol[b] || sb.hn == 0.0) kdone[b] = k;
    else atomicAdd(&active, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (hist && k >= 1 && k <= hist_cap) hist[k - 1] = st[0].res;
    if (bad) *nonfinite = 1;
    *guard = runs;
    cudaGraphSetConditional(cond, (active > 0 && !bad && k < maxiter && runs < maxiter) ? 1u : 0u);
  }
}

// Start of system b = blockIdx.x: beta0 = ||r0||, ref = ||rhs|| (nrm[2b], nrm[2b + 1] hold their
// squares), g = (beta0, 0, ...).
__global__ void k_gm_start(const double2* __restrict__ nrm, GmState* __restrict__ st,
                           double2* __restrict__ g, int stride) {
  const int b = blockIdx.x;
  const double bt = sqrt(nrm[2 * b].x);
  const double ref = sqrt(nrm[2 * b + 1].x);
  GmState* s = st + b;
  s->beta0 = bt;
  s->ref = ref > 0.0 ? ref : 1.0;
  s->inv = bt > 0.0 ? 1.0 / bt : 0.0;
  s->res = bt / s->ref;
  s->flag = (isfinite(bt) && isfinite(ref)) ? 0 : 1;
  s->reorth = 0;
  s->hn = 0.0;
  g[(long long)b * stride] = make_double2(bt, 0.0);
}

// dst = a - b
__global__ void k_sub(double2* __restrict__ dst, const double2* __restrict__ a,
                      const double2* __restrict__ b, long long L) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < L;
       t += (long long)gridDim.x * blockDim.x) {
    const double2 u = a[t], v = b[t];
    dst[t] = make_double2(u.x - v.x, u.y - v.y);
  }
}

// x += d
__global__ void k_add(double2* __restrict__ x, const double2* __restrict__ d, long long L) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < L;
       t += (long long)gridDim.x * blockDim.x) {
    x[t].x += d[t].x;
    x[t].y += d[t].y;
  }
}

// Zero the systems whose mask is 0: v[off[b] .. off[b + 1])
__global__ void k_mask_zero(double2* __restrict__ v, const int* __restrict__ mask,
                            const long long* __restrict__ off) {
  const int b = blockIdx.y;
  if (mask[b]) return;
  const long long L = off[b + 1] - off[b];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < L;
       t += (long long)gridDim.x * blockDim.x)
    v[off[b] + t] = make_double2(0.0, 0.0);
}

__global__ void k_diag_mul(const double2* __restrict__ x, const double2* __restrict__ s,
                           double2* __restrict__ y, long long total, int P) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = cmul(s[i % P], x[i]);
}
__global__ void k_diag_scale(const double2* __restrict__ x, const double* __restrict__ s,
                             double2* __restrict__ y, long long total, int P) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const double f = s[i % P];
    y[i] = make_double2(x[i].x * f, x[i].y * f);
  }
}

inline int grid_for(long long total, int block) {
  long long g = (total + block - 1) / block;
  if (g > 152LL * 32) g = 152LL * 32;
  if (g < 1) g = 1;
  return (int)g;
}

// out[b * out_stride + i] = V_b[i]^H w_b, i < nv, for the systems of s
template <typename T>
void mdot(const vec2<T>* V, long long ldv, int nv, const double2* w, const GmSys& s, double2* out,
          int out_stride, cudaStream_t st) {
  for (int b = 0; b < s.nb; ++b)
    cudaMemsetAsync(out + (long long)b * out_stride, 0, (size_t)nv * sizeof(double2), st);
  dim3 grid((unsigned)((s.maxlen + DOT_T - 1) / DOT_T), (unsigned)std::min(DOT_GY, (nv + 7) / 8), (unsigned)s.nb);
  k_mdot<T><<<grid, 256, 0, st>>>(V, ldv, nv, nullptr, 0, w, s.d_off, out, out_stride, nullptr);
}

template <typename T>
void maxpy(const vec2<T>* V, long long ldv, int nv, const int* nv_arr, const double2* h, int h_stride,
           double2* w, const GmSys& s, double sign, cudaStream_t st) {
  dim3 grid((unsigned)((s.maxlen + 255) / 256), (unsigned)s.nb);
  k_maxpy<T><<<grid, 256, 0, st>>>(V, ldv, nv, nv_arr, nullptr, h, h_stride, w, s.d_off, sign, nullptr);
}

// Device scratch of one batched GMRES run.
struct GmPtrs {
  void* V;                 // basis [maxiter + 1][slot] of double2 or float2
  double2 *H, *h1, *h2, *g, *cs, *sn, *y, *nrm;
  double2 *X, *W;          // the operator's fixed input and output buffers, [nb][L]
  GmState* st;
  int* kk;                 // iterations kept per system (back substitution)
  int* dk;                 // the Arnoldi step counter on the device
  int ldh, stride;
  long long hstride;
};

int gm_alloc(lsms_ctx* c, const GmSys& sys, int maxiter, size_t basis_elem, GmPtrs& p) {
  int rc;
  const int nb = sys.nb;
  p.ldh = maxiter + 1;
  p.stride = maxiter + 2;
  p.hstride = (long long)maxiter * p.ldh;
  if ((rc = ensure(c, c->gm_v, (size_t)(maxiter + 1) * sys.slot * basis_elem))) return rc;
  if ((rc = ensure(c, c->gm_h, (size_t)nb * p.hstride * sizeof(double2)))) return rc;
  if ((rc = ensure(c, c->gm_w, (size_t)2 * sys.slot * sizeof(double2)))) return rc;
  const size_t small = (size_t)nb * (7 * (size_t)p.stride + 2) * sizeof(double2) + nb * sizeof(GmState) +
                       nb * sizeof(int) + 512;
  if ((rc = ensure(c, c->gm_small, small))) return rc;
  p.V = c->gm_v.ptr;
  p.H = (double2*)c->gm_h.ptr;
  p.X = (double2*)c->gm_w.ptr;
  p.W = p.X + sys.slot;
  double2* s = (double2*)c->gm_small.ptr;
  const long long bs = (long long)nb * p.stride;
  p.h1 = s; s += bs;
  p.h2 = s; s += bs;
  p.g = s; s += bs;
  p.cs = s; s += bs;
  p.sn = s; s += bs;
  p.y = s; s += bs;
  p.nrm = s; s += 2 * (long long)nb;
  p.st = (GmState*)s;
  p.kk = (int*)(p.st + nb);
  p.dk = p.kk + nb;
  return LSMS_OK;
}

// host-mapped ring of per-system states: RING slots of nb states, read LAG iterations late
constexpr int LAG = 2, RING = 8;

int ensure_ring(lsms_ctx* c, int nb) {
  const size_t need = (size_t)RING * nb * sizeof(GmState);
  if (c->gm_ring_bytes < need) {
    if (c->gm_ring) cudaFreeHost(c->gm_ring);
    c->gm_ring = nullptr;
    c->gm_ring_dev = nullptr;
    c->gm_ring_bytes = 0;
    if (cudaHostAlloc(&c->gm_ring, need, cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer(&c->gm_ring_dev, c->gm_ring, 0) != cudaSuccess) {
      cudaGetLastError();
      return ctx_fail(c, LSMS_ERR_OOM, "cudaHostAlloc failed for the GMRES state ring");
    }
    c->gm_ring_bytes = need;
  }
  if (!c->gm_ev[0])
    for (int i = 0; i < RING; ++i)
      if (cudaEventCreateWithFlags(&c->gm_ev[i], cudaEventDisableTiming) != cudaSuccess)
        return check_cuda(c, "cudaEventCreate");
  return LSMS_OK;
}

// One Arnoldi step of every system, with the step index read on the device (capturable).
template <typename T>
int enqueue_iteration(lsms_ctx* c, const GmPtrs& g, const GmSys& s, int maxiter, int flags,
                      cudaStream_t st) {
  const long long slot = s.slot;
  const int nb = s.nb;
  vec2<T>* V = (vec2<T>*)g.V;
  int rc;
  k_copy_slot<T><<<grid_for(slot, 256), 256, 0, st>>>(g.X, V, slot, g.dk);
  if ((rc = apply_device(c, s.apply_nrhs, g.X, g.W, flags, st))) return rc;
  const dim3 gd((unsigned)((s.maxlen + DOT_T - 1) / DOT_T), (unsigned)std::min(DOT_GY, (maxiter + 2 + 7) / 8),
                (unsigned)nb);
  const dim3 ga((unsigned)((s.maxlen + 255) / 256), (unsigned)nb);
  // classical Gram-Schmidt; the second pass runs only when the first cancels much of w
  cudaMemsetAsync(g.h1, 0, (size_t)nb * g.stride * sizeof(double2), st);
  k_mdot<T><<<gd, 256, 0, st>>>(V, slot, 1, g.dk, 1, g.W, s.d_off, g.h1, g.stride, nullptr);   // V^H w, ||w||^2
  k_gm_prep<<<nb, 32, 0, st>>>(g.dk, g.h1, g.stride, g.st);
  k_maxpy<T><<<ga, 256, 0, st>>>(V, slot, 1, nullptr, g.dk, g.h1, g.stride, g.W, s.d_off, -1.0, nullptr);
  cudaMemsetAsync(g.h2, 0, (size_t)nb * g.stride * sizeof(double2), st);
  k_mdot<T><<<gd, 256, 0, st>>>(V, slot, 1, g.dk, 1, g.W, s.d_off, g.h2, g.stride, g.st);
  k_maxpy<T><<<ga, 256, 0, st>>>(V, slot, 1, nullptr, g.dk, g.h2, g.stride, g.W, s.d_off, -1.0, g.st);
  k_gm_column<<<nb, 32, (size_t)(3 * maxiter + 2) * sizeof(double2), st>>>(
      g.dk, g.h1, g.h2, g.stride, g.H, g.hstride, g.ldh, g.cs, g.sn, g.g, g.st);
  k_scale_into_slot<T><<<dim3(grid_for(s.maxlen, 256), nb), 256, 0, st>>>(V, slot, g.W, g.st, s.d_off, g.dk);
  k_gm_snapshot<<<1, 256, 0, st>>>(g.st, nb, (GmState*)c->gm_ring_dev, RING, g.dk);
  return check_cuda(c, "gmres iteration");
}

}  // namespace

void launch_diag_mul(const double2* x, const double2* s, double2* y, long long total, int P,
                     cudaStream_t st) {
  if (total) k_diag_mul<<<grid_for(total, 256), 256, 0, st>>>(x, s, y, total, P);
}
void launch_diag_scale(const double2* x, const double* s, double2* y, long long total, int P,
                       cudaStream_t st) {
  if (total) k_diag_scale<<<grid_for(total, 256), 256, 0, st>>>(x, s, y, total, P);
}

// The end of a batched GMRES run: systems still iterating keep `done` iterations; solve each
// system's least-squares problem on its columns and add V y to x.
template <typename T>
int gmres_finish(lsms_ctx* c, const GmPtrs& g, const GmSys& s, std::vector<int>& kdone, int done, int maxiter,
                 int flags, int* iters, double2* x, cudaStream_t stream) {
  int rc;
  (void)maxiter;
  if ((flags & LSMS_APPLY_MIXED) && (rc = mixed_check(c))) return rc;
  const int nb = s.nb;
  bool all = true;
  for (int b = 0; b < nb; ++b) {
    if (kdone[b] < 0) {
      kdone[b] = done;
      all = false;
    }
    iters[b] = kdone[b];
  }
  cudaMemcpyAsync(g.kk, kdone.data(), nb * sizeof(int), cudaMemcpyHostToDevice, stream);
  k_gm_backsolve<<<nb, 32, 0, stream>>>(g.kk, g.H, g.hstride, g.ldh, g.g, g.stride, g.y);
  int kmax = 0;
  for (int b = 0; b < nb; ++b) kmax = std::max(kmax, kdone[b]);
  if (kmax > 0) maxpy<T>((const vec2<T>*)g.V, s.slot, kmax, g.kk, g.y, g.stride, x, s, 1.0, stream);
  cudaStreamSynchronize(stream);
  if ((rc = check_cuda(c, "gmres update"))) return rc;
  return all ? LSMS_OK : LSMS_ERR_NOT_CONVERGED;
}

// The iteration of a batched GMRES run as one graph launch (see gmres_batch_t).  On return
// *loop_k = the Arnoldi steps done, or -1 when the conditional graph could not be built (nothing
// ran; the caller falls back to the host loop); kdone, res, hist and *nonfinite as the host loop
// leaves them.
template <typename T>
int gmres_device_loop(lsms_ctx* c, const GmPtrs& g, const GmSys& s, const double* tol, std::vector<int>& kdone,
                      int maxiter, int flags, double* res, double* hist, int hist_cap, int* n_hist,
                      cudaStream_t stream, int* loop_k, bool* nonfinite) {
  *loop_k = -1;
  const int nb = s.nb;
  const int hcap = (nb == 1 && hist && n_hist) ? std::max(0, std::min(hist_cap - *n_hist, maxiter)) : 0;
  const size_t need =
      (size_t)nb * (sizeof(double) * 2 + sizeof(int)) + 2 * sizeof(int) + (size_t)hcap * sizeof(double) + 64;
  int rc;
  if ((rc = ensure(c, c->gm_loop, need))) return rc;
  double* d_tol = (double*)c->gm_loop.ptr;
  double* d_res = d_tol + nb;
  double* d_hist = d_res + nb;
  int* d_kdone = (int*)(d_hist + hcap);
  int* d_bad = d_kdone + nb;
  int* d_guard = d_bad + 1;
  cudaMemcpyAsync(d_tol, tol, nb * sizeof(double), cudaMemcpyHostToDevice, stream);
  cudaMemcpyAsync(d_res, res, nb * sizeof(double), cudaMemcpyHostToDevice, stream);
  cudaMemcpyAsync(d_kdone, kdone.data(), nb * sizeof(int), cudaMemcpyHostToDevice, stream);
  cudaMemsetAsync(d_bad, 0, 2 * sizeof(int), stream);
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool built = false;
  const int timing = c->timing;
  c->timing = 0;
  if (cudaGraphCreate(&graph, 0) == cudaSuccess) {
    cudaGraphConditionalHandle cond;
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cudaGraphNode_t node;
    if (cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault) == cudaSuccess) {
      cp.conditional.handle = cond;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      if (cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp) == cudaSuccess) {
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        if (cudaStreamBeginCaptureToGraph(stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
            cudaSuccess) {
          int erc = enqueue_iteration<T>(c, g, s, maxiter, flags, stream);
          if (erc == LSMS_OK)
            k_gm_decide<<<1, 256, 0, stream>>>(g.st, nb, d_tol, d_kdone, d_res, g.dk, maxiter, d_bad, d_guard,
                                                hcap ? d_hist : nullptr, hcap, cond);
          cudaGraph_t cap = nullptr;
          const cudaError_t e = cudaStreamEndCapture(stream, &cap);
          built = erc == LSMS_OK && e == cudaSuccess && cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
        }
      }
    }
  }
  c->timing = timing;
  if (graph) cudaGraphDestroy(graph);
  cudaGetLastError();
  c->err.clear();
  if (!built) {
    if (exec) cudaGraphExecDestroy(exec);
    return LSMS_OK;
  }
  const cudaError_t le = cudaGraphLaunch(exec, stream);
  cudaStreamSynchronize(stream);
  cudaGraphExecDestroy(exec);
  if (le != cudaSuccess) return check_cuda(c, "gmres loop graph");
  if ((rc = check_cuda(c, "gmres loop"))) return rc;
  int k = 0, bad = 0;
  cudaMemcpy(&k, g.dk, sizeof(int), cudaMemcpyDeviceToHost);
  cudaMemcpy(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost);
  cudaMemcpy(kdone.data(), d_kdone, nb * sizeof(int), cudaMemcpyDeviceToHost);
  cudaMemcpy(res, d_res, nb * sizeof(double), cudaMemcpyDeviceToHost);
  if (hcap > 0) {
    const int got = std::min(k, hcap);
    if (got > 0) cudaMemcpy(hist + *n_hist, d_hist, got * sizeof(double), cudaMemcpyDeviceToHost);
    *n_hist += got;
  }
  *nonfinite = bad != 0;
  *loop_k = k;
  return check_cuda(c, "gmres loop results");
}

// Batched GMRES for A x_b = rhs_b over the systems of s (rhs, x: one slot).  x: initial guesses if
// x_nonzero, solutions on return.  tol[b]: relative tolerance per system.  iters[b], res[b]:
// iterations used and final residual estimate.  Returns LSMS_OK when every system converged,
// LSMS_ERR_NOT_CONVERGED or LSMS_ERR_NONFINITE otherwise.
template <typename T>
int gmres_batch_t(lsms_ctx* c, const GmSys& s, const double2* rhs, double2* x, bool x_nonzero, const double* tol,
                  int maxiter, int flags, int* iters, double* res, double* hist, int hist_cap,
                  int* n_hist, cudaStream_t stream) {
  const int nb = s.nb;
  GmPtrs g;
  int rc;
  if ((rc = gm_alloc(c, s, maxiter, sizeof(vec2<T>), g))) return rc;
  vec2<T>* V = (vec2<T>*)g.V;
  if ((rc = ensure_ring(c, nb))) return rc;
  GmState* ring = (GmState*)c->gm_ring;
  static std::once_flag attr;
  std::call_once(attr, [] {
    cudaFuncSetAttribute(k_gm_column, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)((3 * GIVENS_MAX + 2) * sizeof(double2)));
  });
  const long long slot = s.slot;                         // distance between basis slots
  // r0 = rhs - A x (in the operator's input buffer X when x is given); basis slot 0 = r0 / ||r0||
  const double2* r0 = rhs;
  if (x_nonzero) {
    if ((rc = apply_device(c, s.apply_nrhs, x, g.W, flags, stream))) return rc;
    k_sub<<<grid_for(slot, 256), 256, 0, stream>>>(g.X, rhs, g.W, slot);
    r0 = g.X;
  } else {
    cudaMemsetAsync(x, 0, slot * sizeof(double2), stream);
  }
  mdot<double>(r0, slot, 1, r0, s, g.nrm, 2, stream);        // ||r0||^2 at nrm[2b]
  mdot<double>(rhs, slot, 1, rhs, s, g.nrm + 1, 2, stream);  // ||rhs||^2 at nrm[2b + 1]
  k_gm_start<<<nb, 1, 0, stream>>>(g.nrm, g.st, g.g, g.stride);
  k_scale_by<T><<<dim3(grid_for(s.maxlen, 256), nb), 256, 0, stream>>>(V, r0, g.st, s.d_off);
  cudaMemsetAsync(g.dk, 0, sizeof(int), stream);
  cudaStreamSynchronize(stream);
  if ((rc = check_cuda(c, "gmres start"))) return rc;
  std::vector<GmState> s0(nb);
  cudaMemcpy(s0.data(), g.st, nb * sizeof(GmState), cudaMemcpyDeviceToHost);
  std::vector<int> kdone(nb, -1);        // -1: still iterating; else iterations kept
  bool nonfinite = false;
  int active = 0;
  for (int b = 0; b < nb; ++b) {
    iters[b] = 0;
    res[b] = s0[b].res;
    if (s0[b].flag) nonfinite = true;
    if (s0[b].beta0 == 0.0 || s0[b].res <= tol[b]) kdone[b] = 0;
    else ++active;
  }
  if (nonfinite) return ctx_fail(c, LSMS_ERR_NONFINITE, "non-finite right-hand side");
  // The whole iteration as one graph launch: a conditional while node whose body is one Arnoldi
  // step of all systems followed by the stopping test on the device (after one uncaptured
  // application, so that every workspace the operator needs exists).  If the graph cannot be built,
  // the step is captured alone and launched once per step from the host loop below.
  if (active > 0 && c->use_graphs) {
    if ((rc = apply_device(c, s.apply_nrhs, g.X, g.W, flags, stream))) return rc;
    int loop_k = -1;
    if ((rc = gmres_device_loop<T>(c, g, s, tol, kdone, maxiter, flags, res, hist, hist_cap, n_hist, stream,
                                   &loop_k, &nonfinite)))
      return rc;
    if (loop_k >= 0) {
      if (nonfinite) {
        if ((flags & LSMS_APPLY_MIXED) && (rc = mixed_check(c))) return rc;
        return ctx_fail(c, LSMS_ERR_NONFINITE, "non-finite value in GMRES");
      }
      return gmres_finish<T>(c, g, s, kdone, loop_k, maxiter, flags, iters, x, stream);
    }
  }
  // Capture one Arnoldi step of all systems as a CUDA graph; launch it once per step.
  cudaGraphExec_t exec = nullptr;
  if (active > 0 && c->use_graphs) {
    const int timing = c->timing;
    c->timing = 0;
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      const int erc = enqueue_iteration<T>(c, g, s, maxiter, flags, stream);
      const cudaError_t e = cudaStreamEndCapture(stream, &graph);
      if (erc == LSMS_OK && e == cudaSuccess && graph &&
          cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess)
        exec = nullptr;
      if (graph) cudaGraphDestroy(graph);
    }
    cudaGetLastError();
    c->timing = timing;
    c->err.clear();
  }
  int k = 0, checked = 0;
  auto check = [&](int j) {              // consume the states after iteration j
    cudaEventSynchronize(c->gm_ev[j % RING]);
    const GmState* sj = ring + (size_t)(j % RING) * nb;
    for (int b = 0; b < nb; ++b) {
      if (kdone[b] >= 0) continue;
      res[b] = sj[b].res;
      if (nb == 1 && hist && n_hist && *n_hist < hist_cap) hist[(*n_hist)++] = res[b];
      if (sj[b].flag) nonfinite = true;
      if (sj[b].flag || res[b] <= tol[b] || sj[b].hn == 0.0) {
        kdone[b] = j + 1;
        --active;
      }
    }
    checked = j + 1;
  };
  while (k < maxiter && active > 0 && !nonfinite) {
    if (exec) {
      if (cudaGraphLaunch(exec, stream) != cudaSuccess) {
        cudaGraphExecDestroy(exec);
        return check_cuda(c, "cudaGraphLaunch");
      }
    } else if ((rc = enqueue_iteration<T>(c, g, s, maxiter, flags, stream))) {
      return rc;
    }
    cudaEventRecord(c->gm_ev[k % RING], stream);
    if (k - LAG >= checked) check(k - LAG);
    ++k;
  }
  while (active > 0 && !nonfinite && checked < k) check(checked);   // drain
  if (exec) cudaGraphExecDestroy(exec);
  cudaStreamSynchronize(stream);
  if (nonfinite) {
    if ((flags & LSMS_APPLY_MIXED) && (rc = mixed_check(c))) return rc;
    return ctx_fail(c, LSMS_ERR_NONFINITE, "non-finite value in GMRES");
  }
  return gmres_finish<T>(c, g, s, kdone, checked, maxiter, flags, iters, x, stream);
}

// Batched GMRES for A x_b = rhs_b over the systems of s: the inner solves of the mixed refinement
// (every tolerance >= 1e-5) keep and multiply their Krylov basis in FP32, FP64 solves in FP64.
int gmres_batch(lsms_ctx* c, const GmSys& s, const double2* rhs, double2* x, bool x_nonzero, const double* tol,
                int maxiter, int flags, int* iters, double* res, double* hist, int hist_cap,
                int* n_hist, cudaStream_t stream) {
  bool f32 = (flags & LSMS_APPLY_MIXED) != 0;
  for (int b = 0; b < s.nb && f32; ++b) f32 = tol[b] >= 1e-5;
  if (f32)
    return gmres_batch_t<float>(c, s, rhs, x, x_nonzero, tol, maxiter, flags, iters, res, hist, hist_cap, n_hist,
                                stream);
  return gmres_batch_t<double>(c, s, rhs, x, x_nonzero, tol, maxiter, flags, iters, res, hist, hist_cap, n_hist,
                               stream);
}

// ||v_b||_2 for the systems of s (read back synchronously)
static void norms_device(const double2* v, const GmSys& s, double2* tmp, cudaStream_t st,
                         std::vector<double>& out) {
  mdot<double>(v, s.slot, 1, v, s, tmp, 1, st);
  std::vector<double2> h(s.nb);
  cudaMemcpyAsync(h.data(), tmp, s.nb * sizeof(double2), cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  out.resize(s.nb);
  for (int b = 0; b < s.nb; ++b) out[b] = std::sqrt(std::max(h[b].x, 0.0));
}

// Systems of equal length L (the sources of one layout), offsets b L kept in c->gm_off.
int gm_uniform_systems(lsms_ctx* c, int nb, long long L, GmSys& s, cudaStream_t st) {
  std::vector<long long> off(nb + 1);
  for (int b = 0; b <= nb; ++b) off[b] = (long long)b * L;
  int rc;
  if ((rc = ensure(c, c->gm_off, off.size() * sizeof(long long)))) return rc;
  cudaMemcpyAsync(c->gm_off.ptr, off.data(), off.size() * sizeof(long long), cudaMemcpyHostToDevice, st);
  cudaStreamSynchronize(st);
  s.nb = nb;
  s.slot = (long long)nb * L;
  s.maxlen = L;
  s.d_off = (const long long*)c->gm_off.ptr;
  s.apply_nrhs = nb;
  return check_cuda(c, "gmres systems");
}

// Solve (I - D S (T + R) D^{-1}) xs_b = rhs_b for the systems of s (rhs = D S a_inc, xs scaled
// unknowns; xs holds initial guesses if nonzero).  FP64 GMRES, or for a mixed context FP64
// refinement around batched inner GMRES on the mixed operator.  Per system: it[b] iterations,
// rest[b] final residual estimate, rel64[b] FP64 relative residual.
int solve_systems(lsms_ctx* c, const GmSys& s, const double2* rhs, double2* xs, bool nonzero, double tol,
                  int maxiter, std::vector<int>& it, std::vector<double>& rest, std::vector<double>& rel64,
                  int* outer_out, double* hist, int hcap, int* nh, cudaStream_t st) {
  const int nb = s.nb;
  const long long LT = s.slot;
  int rc;
  if ((rc = ensure(c, c->gm_r, (size_t)2 * LT * sizeof(double2) + 64))) return rc;
  if ((rc = ensure(c, c->gm_x, (size_t)LT * sizeof(double2)))) return rc;
  if ((rc = ensure(c, c->gm_mask, (size_t)nb * sizeof(int) + 64))) return rc;
  double2* resv = (double2*)c->gm_r.ptr;
  double2* tmp = resv + LT;
  double2* dx = (double2*)c->gm_x.ptr;
  int* d_mask = (int*)c->gm_mask.ptr;
  it.assign(nb, 0);
  rest.assign(nb, 0.0);
  rel64.assign(nb, -1.0);
  int outer = 0, status = LSMS_OK;
  c->refine_stagnated = false;
  if (c->precision != LSMS_MIXED) {
    std::vector<double> tv(nb, tol);
    status = gmres_batch(c, s, rhs, xs, nonzero, tv.data(), maxiter, LSMS_APPLY_SCALED, it.data(), rest.data(),
                         hist, hcap, nh, st);
    if (status != LSMS_OK && status != LSMS_ERR_NOT_CONVERGED) return status;
    outer = 1;
  } else {
    // FP64 refinement: r = rhs - A x with the FP64 operator; batched inner GMRES on the mixed
    // operator for the systems not yet converged (the others get a zero right-hand side).
    std::vector<double> bn;
    norms_device(rhs, s, tmp, st, bn);
    if (!nonzero) cudaMemsetAsync(xs, 0, LT * sizeof(double2), st);
    const int max_outer = 20;
    const double inner_tol = 1e-5;
    status = LSMS_ERR_NOT_CONVERGED;
    std::vector<int> mask(nb, 1), it_in(nb, 0), stall(nb, 0);
    std::vector<double> rn(nb, 1.0), tol_in(nb), r_in(nb), best(nb, HUGE_VAL);
    int used = 0;
    bool stagnated = false;
    for (outer = 0; outer < max_outer && used < maxiter; ++outer) {
      if (outer == 0 && !nonzero) {
        cudaMemcpyAsync(resv, rhs, LT * sizeof(double2), cudaMemcpyDeviceToDevice, st);
        std::fill(rn.begin(), rn.end(), 1.0);
      } else {
        if ((rc = apply_device(c, s.apply_nrhs, xs, tmp, LSMS_APPLY_SCALED | LSMS_APPLY_RESIDUAL_INTERNAL, st)))
          return rc;
        k_sub<<<grid_for(LT, 256), 256, 0, st>>>(resv, rhs, tmp, LT);
        std::vector<double> r;
        norms_device(resv, s, tmp, st, r);
        for (int b = 0; b < nb; ++b) rn[b] = bn[b] > 0 ? r[b] / bn[b] : 0.0;
      }
      bool all = true, bad = false;
      for (int b = 0; b < nb; ++b) {
        rel64[b] = rn[b];
        rest[b] = rn[b];
        if (!std::isfinite(rn[b])) bad = true;
        // stagnation: a refinement step gains about five digits (the inner tolerance); a system
        // whose FP64 residual has not halved over three steps sits at the floor the FP64
        // operator's rounding allows and is refined no further
        if (rn[b] < 0.5 * best[b]) {
          best[b] = rn[b];
          stall[b] = 0;
        } else if (rn[b] > tol && ++stall[b] >= 3) {
          stagnated = true;
        }
        mask[b] = (rn[b] > tol && stall[b] < 3) ? 1 : 0;
        if (mask[b]) all = false;
        tol_in[b] = std::max(inner_tol, 0.5 * tol / std::max(rn[b], 1e-300));
      }
      if (bad) { status = ctx_fail(c, LSMS_ERR_NONFINITE, "non-finite refinement residual"); break; }
      if (all) { status = stagnated ? LSMS_ERR_NOT_CONVERGED : LSMS_OK; break; }
      cudaMemcpyAsync(d_mask, mask.data(), nb * sizeof(int), cudaMemcpyHostToDevice, st);
      k_mask_zero<<<dim3(grid_for(s.maxlen, 256), nb), 256, 0, st>>>(resv, d_mask, s.d_off);
      const int rci = gmres_batch(c, s, resv, dx, false, tol_in.data(), maxiter - used,
                                  LSMS_APPLY_SCALED | LSMS_APPLY_MIXED, it_in.data(), r_in.data(),
                                  hist, hcap, nh, st);
      int mx = 0;
      for (int b = 0; b < nb; ++b) {
        it[b] += it_in[b];
        mx = std::max(mx, it_in[b]);
      }
      used += mx;
      if (rci != LSMS_OK && rci != LSMS_ERR_NOT_CONVERGED) { status = rci; break; }
      k_add<<<grid_for(LT, 256), 256, 0, st>>>(xs, dx, LT);              // x += dx
      std::fill(rel64.begin(), rel64.end(), -1.0);
    }
    if (status == LSMS_ERR_NONFINITE) return status;
    c->refine_stagnated = stagnated;
  }
  // true FP64 residuals of the final iterates (the refinement loop has them when it stopped on a
  // fresh residual)
  bool need = false;
  for (int b = 0; b < nb; ++b) need = need || rel64[b] < 0.0;
  if (need) {
    if ((rc = apply_device(c, s.apply_nrhs, xs, tmp, LSMS_APPLY_SCALED | LSMS_APPLY_RESIDUAL_INTERNAL, st)))
      return rc;
    k_sub<<<grid_for(LT, 256), 256, 0, st>>>(resv, rhs, tmp, LT);
    std::vector<double> r, b2;
    norms_device(resv, s, tmp, st, r);
    norms_device(rhs, s, tmp, st, b2);
    for (int b = 0; b < nb; ++b) rel64[b] = b2[b] > 0 ? r[b] / b2[b] : 0.0;
  }
  if (outer_out) *outer_out = outer;
  return status;
}

extern "C" int lsms_solve(lsms_ctx* c, int nsrc, const double* src_xy, double tol, int maxiter,
                          const double* x0, double* beta_out, lsms_solve_info* info) {
  int rc;
  if ((rc = need_particles(c))) return rc;
  if ((rc = validate_sources(c, nsrc, src_xy))) return rc;
  if (!(tol > 0.0) || maxiter <= 0 || maxiter > GIVENS_MAX)
    return ctx_fail(c, LSMS_ERR_ARG, "tol must be > 0 and 0 < maxiter <= 4096");
  if (is_batch(c)) return batch_solve(c, nsrc, src_xy, tol, maxiter, x0, beta_out, info);
  const long long L = (long long)c->n * c->P;
  const long long LT = (long long)nsrc * L;
  cudaStream_t st = c->stream;
  if (info) { info->iters = 0; info->outer_iters = 0; info->rel_res = 0; info->rel_res_fp64 = 0; info->n_history = 0; }
  c->n_src = 0;
  c->src_xy.assign(src_xy, src_xy + 2 * nsrc);
  if ((rc = ensure(c, c->sol, (size_t)(LT > 0 ? LT : 1) * sizeof(double2)))) return rc;
  if (nsrc == 0) return LSMS_OK;
  if (L == 0) { c->n_src = nsrc; return LSMS_OK; }
  if ((rc = ensure(c, c->gm_b, (size_t)2 * LT * sizeof(double2)))) return rc;
  if ((rc = ensure(c, c->ws_aux, (size_t)2 * nsrc * sizeof(double) + 64))) return rc;
  double* d_src = (double*)c->ws_aux.ptr;
  cudaMemcpyAsync(d_src, src_xy, (size_t)2 * nsrc * sizeof(double), cudaMemcpyHostToDevice, st);
  double2* beta = (double2*)c->sol.ptr;                 // a_inc for every source, replaced by beta
  if ((rc = incident_device(c, nsrc, d_src, beta, st))) return rc;
  double2* rhs = (double2*)c->gm_b.ptr;                 // [nsrc][L]
  double2* xs = rhs + LT;                               // scaled iterates
  if (c->dense)                                          // D S_j a_inc (rotated dense matrices)
    launch_scatter_dense(nullptr, beta, c->d_smt + (size_t)c->P * c->P,
                         c->has_theta ? (const double*)c->theta_buf.ptr : nullptr, nsrc, c->n, c->P, rhs, st);
  else
    launch_diag_mul(beta, c->d_scale_out + c->P, rhs, LT, c->P, st);   // D S a_inc
  bool nonzero = false;
  if (x0) {
    double acc = 0.0;                     // v * 0 is NaN exactly for NaN and +-Inf
    for (long long i = 0; i < 2 * LT; ++i) acc += x0[i] * 0.0;
    if (acc != 0.0) return ctx_fail(c, LSMS_ERR_ARG, "non-finite value in the initial guess x0");
    cudaMemcpyAsync(beta, x0, LT * sizeof(double2), cudaMemcpyHostToDevice, st);
    launch_diag_scale(beta, c->d_hscale, xs, LT, c->P, st);
    nonzero = true;
  }
  GmSys s;
  if ((rc = gm_uniform_systems(c, nsrc, L, s, st))) return rc;
  std::vector<int> it;
  std::vector<double> rest, rel64;
  int outer = 0, nh = 0;
  const int status = solve_systems(c, s, rhs, xs, nonzero, tol, maxiter, it, rest, rel64, &outer,
                                   info ? info->history : nullptr, info ? info->history_cap : 0, &nh, st);
  if (status != LSMS_OK && status != LSMS_ERR_NOT_CONVERGED) return status;
  launch_diag_scale(xs, c->d_scale_in + c->P, beta, LT, c->P, st);   // beta = D^{-1} b
  if ((rc = check_cuda(c, "solve"))) return rc;
  if (info) {
    int mi = 0;
    double mr = 0.0, m64 = 0.0;
    for (int b = 0; b < nsrc; ++b) {
      mi = std::max(mi, it[b]);
      mr = std::max(mr, rest[b]);
      m64 = std::max(m64, rel64[b]);
    }
    info->iters = mi;                 // the most iterations any source needed
    info->outer_iters = outer;
    info->rel_res = mr;               // the worst source
    info->rel_res_fp64 = m64;
    info->n_history = nh;
  }
  c->n_src = nsrc;
  if (beta_out) {
    cudaMemcpyAsync(beta_out, c->sol.ptr, (size_t)LT * sizeof(double2), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    if ((rc = check_cuda(c, "solve copy"))) return rc;
  }
  if (status == LSMS_ERR_NOT_CONVERGED)
    ctx_fail(c, status, c->refine_stagnated ? "refinement stagnated: the FP64 residual stopped decreasing above tol"
                                            : "GMRES reached maxiter");
  return status;
}
