// Device-resident GMRES (Saad-Schultz, cited in Sec. 3.2 of the paper) on the scaled,
// preconditioned disc system (I - D S (T + R) D^{-1}) b = D S a_inc, D = diag |H_n(k2 R)|, and the
// FP64 iterative-refinement loop of the mixed-precision solve.
//
// Arnoldi uses classical Gram-Schmidt applied twice (CGS2); the Hessenberg matrix, the Givens
// rotations and the residual estimate stay on the device.  The host only launches kernels and reads
// one double (the residual estimate) per iteration to decide when to stop.
#include <cmath>
#include <cstring>

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

struct GmState {
  double beta0;   // ||r0||
  double ref;     // ||rhs||: residuals are reported relative to it
  double res;     // |g_{k+1}| / ||rhs||
  double hn;      // ||w|| of the last Arnoldi step
  double inv;     // scale for the next basis vector
  int flag;       // 1: non-finite value seen
};

constexpr int DOT_T = 1024;    // elements per CTA
constexpr int DOT_V = 32;      // vectors per CTA (4 per warp)

// out[i] += sum_t conj(V[i][t]) w[t] for i < nv (out pre-zeroed).  Grid: (element chunks, vector
// groups), so that the whole GPU works even for short Krylov bases.
__global__ void __launch_bounds__(256)
k_mdot(const double2* __restrict__ V, long long ldv, int nv, const double2* __restrict__ w,
       long long L, double2* __restrict__ out) {
  __shared__ double2 ws[DOT_T];
  const long long t0 = blockIdx.x * (long long)DOT_T;
  const int cnt = (int)min((long long)DOT_T, L - t0);
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) ws[i] = w[t0 + i];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int i1 = min(nv, (int)(blockIdx.y + 1) * DOT_V);
  for (int i = blockIdx.y * DOT_V + warp; i < i1; i += nw) {
    const double2* vi = V + (long long)i * ldv + t0;
    double2 acc = make_double2(0.0, 0.0);
    for (int t = lane; t < cnt; t += 32) {
      const double2 c = cjmul(vi[t], ws[t]);
      acc.x += c.x;
      acc.y += c.y;
    }
    acc = warp_sum(acc);
    if (lane == 0) {
      atomicAdd(&out[i].x, acc.x);
      atomicAdd(&out[i].y, acc.y);
    }
  }
}

// w[t] += sign sum_i V[i][t] h[i]
__global__ void __launch_bounds__(256)
k_maxpy(const double2* __restrict__ V, long long ldv, int nv, const double2* __restrict__ h,
        double2* __restrict__ w, long long L, double sign) {
  __shared__ double2 hs[256];
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  double2 acc = make_double2(0.0, 0.0);
  for (int i0 = 0; i0 < nv; i0 += 256) {
    const int c = min(256, nv - i0);
    __syncthreads();
    if (threadIdx.x < c) hs[threadIdx.x] = h[i0 + threadIdx.x];
    __syncthreads();
    if (t < L) {
      for (int i = 0; i < c; ++i) {
        const double2 v = V[(long long)(i0 + i) * ldv + t];
        const double2 hh = hs[i];
        acc.x = fma(v.x, hh.x, fma(-v.y, hh.y, acc.x));
        acc.y = fma(v.x, hh.y, fma(v.y, hh.x, acc.y));
      }
    }
  }
  if (t < L) {
    w[t].x += sign * acc.x;
    w[t].y += sign * acc.y;
  }
}

// dst = src * (*scale)
__global__ void k_scale_by(double2* __restrict__ dst, const double2* __restrict__ src,
                           const GmState* __restrict__ st, long long L) {
  const double s = st->inv;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < L;
       t += (long long)gridDim.x * blockDim.x) {
    const double2 v = src[t];
    dst[t] = make_double2(v.x * s, v.y * s);
  }
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

__global__ void k_gm_start(const double2* __restrict__ nrm2, const double2* __restrict__ nrm2_rhs,
                           GmState* __restrict__ st, double2* __restrict__ g) {
  const double b = sqrt(nrm2[0].x);
  const double ref = sqrt(nrm2_rhs[0].x);
  st->beta0 = b;
  st->ref = ref > 0.0 ? ref : 1.0;
  st->inv = b > 0.0 ? 1.0 / b : 0.0;
  st->res = b / st->ref;
  st->flag = (isfinite(b) && isfinite(ref)) ? 0 : 1;
  g[0] = make_double2(b, 0.0);
}

// Column k of the Hessenberg matrix: H[0..k][k] = h1 + h2, H[k+1][k] = ||w||; apply the previous
// Givens rotations, form the new one, update g and the residual estimate |g_{k+1}| / ||rhs||.
// One warp: the lanes stage the column and the rotations in shared memory, lane 0 sweeps them.
constexpr int GIVENS_MAX = 4096;

__global__ void __launch_bounds__(32)
k_gm_column(int k, const double2* __restrict__ h1, const double2* __restrict__ h2,
            const double2* __restrict__ nrm2, double2* __restrict__ H, int ldh,
            double2* __restrict__ cs, double2* __restrict__ sn, double2* __restrict__ g,
            GmState* __restrict__ st) {
  extern __shared__ double2 sm[];
  double2* col = sm;                    // [k + 2]
  double2* c_s = sm + (k + 2);          // [k]
  double2* s_s = c_s + k;               // [k]
  const int lane = threadIdx.x;
  for (int i = lane; i <= k; i += 32) col[i] = make_double2(h1[i].x + h2[i].x, h1[i].y + h2[i].y);
  for (int i = lane; i < k; i += 32) {
    c_s[i] = cs[i];
    s_s[i] = sn[i];
  }
  __syncwarp();
  if (lane == 0) {
    const double hn = sqrt(nrm2[0].x);
    st->hn = hn;
    st->inv = hn > 0.0 ? 1.0 / hn : 0.0;
    col[k + 1] = make_double2(hn, 0.0);
    for (int i = 0; i < k; ++i) {
      const double2 a = col[i], b = col[i + 1];
      const double2 ci = c_s[i], si = s_s[i];
      // [conj(c) conj(s); -s c] [a; b]
      const double2 t = make_double2(cjmul(ci, a).x + cjmul(si, b).x, cjmul(ci, a).y + cjmul(si, b).y);
      const double2 u = make_double2(-cmul(si, a).x + cmul(ci, b).x, -cmul(si, a).y + cmul(ci, b).y);
      col[i] = t;
      col[i + 1] = u;
    }
    const double2 a = col[k];
    const double r = hypot(hypot(a.x, a.y), hn);
    double2 c, s;
    if (r > 0.0) {
      c = make_double2(a.x / r, a.y / r);
      s = make_double2(hn / r, 0.0);
    } else {
      c = make_double2(1.0, 0.0);
      s = make_double2(0.0, 0.0);
    }
    cs[k] = c;
    sn[k] = s;
    col[k] = make_double2(r, 0.0);
    col[k + 1] = make_double2(0.0, 0.0);
    const double2 gk = g[k];
    g[k] = cjmul(c, gk);
    g[k + 1] = make_double2(-cmul(s, gk).x, -cmul(s, gk).y);
    const double res = hypot(g[k + 1].x, g[k + 1].y) / st->ref;
    st->res = res;
    if (!isfinite(res) || !isfinite(hn)) st->flag = 1;
  }
  __syncwarp();
  double2* Hc = H + (long long)k * ldh;
  for (int i = lane; i <= k + 1; i += 32) Hc[i] = col[i];
}

// Back substitution H[0..k)[0..k) y = g, one warp (lanes over the column index).
__global__ void k_gm_backsolve(int k, const double2* __restrict__ H, int ldh,
                               const double2* __restrict__ g, double2* __restrict__ y) {
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
      y[i] = make_double2((num.x * d.x + num.y * d.y) / dd, (num.y * d.x - num.x * d.y) / dd);
    }
    __syncwarp();
  }
}

inline int grid_for(long long total, int block) {
  long long g = (total + block - 1) / block;
  if (g > 152LL * 32) g = 152LL * 32;
  if (g < 1) g = 1;
  return (int)g;
}

void mdot(const double2* V, long long ldv, int nv, const double2* w, long long L, double2* out,
          cudaStream_t st) {
  cudaMemsetAsync(out, 0, (size_t)nv * sizeof(double2), st);
  dim3 grid((unsigned)((L + DOT_T - 1) / DOT_T), (unsigned)((nv + DOT_V - 1) / DOT_V));
  k_mdot<<<grid, 256, 0, st>>>(V, ldv, nv, w, L, out);
}

void maxpy(const double2* V, long long ldv, int nv, const double2* h, double2* w, long long L,
           double sign, cudaStream_t st) {
  k_maxpy<<<(int)((L + 255) / 256), 256, 0, st>>>(V, ldv, nv, h, w, L, sign);
}

// Small device scratch of one GMRES run.
struct GmPtrs {
  double2 *V, *H, *h1, *h2, *g, *cs, *sn, *y, *nrm;
  GmState* st;
  double2* w;
  int ldh;
};

int gm_alloc(lsms_ctx* c, long long L, int maxiter, GmPtrs& p) {
  int rc;
  if ((rc = ensure(c, c->gm_v, (size_t)(maxiter + 1) * L * sizeof(double2)))) return rc;
  if ((rc = ensure(c, c->gm_h, (size_t)(maxiter + 1) * maxiter * sizeof(double2)))) return rc;
  const size_t small = (size_t)(7 * (maxiter + 2) + 8) * sizeof(double2) + sizeof(GmState) + 64;
  if ((rc = ensure(c, c->gm_small, small))) return rc;
  if ((rc = ensure(c, c->gm_w, (size_t)L * sizeof(double2)))) return rc;
  p.V = (double2*)c->gm_v.ptr;
  p.H = (double2*)c->gm_h.ptr;
  p.ldh = maxiter + 1;
  double2* s = (double2*)c->gm_small.ptr;
  p.h1 = s; s += maxiter + 2;
  p.h2 = s; s += maxiter + 2;
  p.g = s; s += maxiter + 2;
  p.cs = s; s += maxiter + 2;
  p.sn = s; s += maxiter + 2;
  p.y = s; s += maxiter + 2;
  p.nrm = s; s += maxiter + 2;
  p.st = (GmState*)s;
  p.w = (double2*)c->gm_w.ptr;
  return LSMS_OK;
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

// GMRES for A x = rhs with A = apply_device(flags), x (in: initial guess if x_nonzero, out:
// solution).  Returns LSMS_OK, LSMS_ERR_NOT_CONVERGED or LSMS_ERR_NONFINITE.
int gmres_device(lsms_ctx* c, const double2* rhs, double2* x, bool x_nonzero, double tol,
                 int maxiter, int flags, int* iters, double* res_out, double* hist, int hist_cap,
                 int* n_hist, cudaStream_t stream) {
  const long long L = (long long)c->n * c->P;
  GmPtrs g;
  int rc;
  if ((rc = gm_alloc(c, L, maxiter, g))) return rc;
  volatile GmState* hs = (volatile GmState*)c->h_pinned;
  *iters = 0;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_gm_column, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)((3 * GIVENS_MAX + 2) * sizeof(double2)));
    attr = true;
  }
  // r0 = rhs - A x
  if (x_nonzero) {
    if ((rc = apply_device(c, 1, x, g.w, flags, stream))) return rc;
    k_sub<<<grid_for(L, 256), 256, 0, stream>>>(g.V, rhs, g.w, L);
  } else {
    cudaMemsetAsync(x, 0, L * sizeof(double2), stream);
    cudaMemcpyAsync(g.V, rhs, L * sizeof(double2), cudaMemcpyDeviceToDevice, stream);
  }
  mdot(g.V, L, 1, g.V, L, g.nrm, stream);
  mdot(rhs, L, 1, rhs, L, g.nrm + 1, stream);
  k_gm_start<<<1, 1, 0, stream>>>(g.nrm, g.nrm + 1, g.st, g.g);
  k_scale_by<<<grid_for(L, 256), 256, 0, stream>>>(g.V, g.V, g.st, L);
  cudaMemcpyAsync((void*)hs, g.st, sizeof(GmState), cudaMemcpyDeviceToHost, stream);
  cudaStreamSynchronize(stream);
  if ((rc = check_cuda(c, "gmres start"))) return rc;
  if (hs->flag) return ctx_fail(c, LSMS_ERR_NONFINITE, "non-finite right-hand side");
  if (hs->beta0 == 0.0 || hs->res <= tol) {
    *res_out = hs->res;
    return LSMS_OK;
  }
  int k = 0;
  double res = 1.0;
  bool converged = false, nonfinite = false;
  while (k < maxiter) {
    double2* vk = g.V + (long long)k * L;
    if ((rc = apply_device(c, 1, vk, g.w, flags, stream))) return rc;
    mdot(g.V, L, k + 1, g.w, L, g.h1, stream);
    maxpy(g.V, L, k + 1, g.h1, g.w, L, -1.0, stream);
    mdot(g.V, L, k + 1, g.w, L, g.h2, stream);
    maxpy(g.V, L, k + 1, g.h2, g.w, L, -1.0, stream);
    mdot(g.w, L, 1, g.w, L, g.nrm, stream);
    k_gm_column<<<1, 32, (size_t)(3 * k + 2) * sizeof(double2), stream>>>(k, g.h1, g.h2, g.nrm, g.H, g.ldh,
                                                                        g.cs, g.sn, g.g, g.st);
    k_scale_by<<<grid_for(L, 256), 256, 0, stream>>>(g.V + (long long)(k + 1) * L, g.w, g.st, L);
    cudaMemcpyAsync((void*)hs, g.st, sizeof(GmState), cudaMemcpyDeviceToHost, stream);
    cudaStreamSynchronize(stream);
    if ((rc = check_cuda(c, "gmres iteration"))) return rc;
    if ((flags & LSMS_APPLY_MIXED) && (rc = mixed_check(c))) return rc;
    ++k;
    res = hs->res;
    if (hist && n_hist && *n_hist < hist_cap) hist[(*n_hist)++] = res;
    if (hs->flag) { nonfinite = true; break; }
    if (res <= tol || hs->hn == 0.0) { converged = true; break; }
  }
  *iters = k;
  *res_out = res;
  if (nonfinite) return ctx_fail(c, LSMS_ERR_NONFINITE, "non-finite value in GMRES");
  k_gm_backsolve<<<1, 32, 0, stream>>>(k, g.H, g.ldh, g.g, g.y);
  maxpy(g.V, L, k, g.y, x, L, 1.0, stream);
  if ((rc = check_cuda(c, "gmres update"))) return rc;
  return converged ? LSMS_OK : LSMS_ERR_NOT_CONVERGED;
}

// ||v||_2 on the device (read back synchronously)
static double norm_device(lsms_ctx* c, const double2* v, long long L, double2* tmp, cudaStream_t st) {
  mdot(v, L, 1, v, L, tmp, st);
  double2 h;
  cudaMemcpyAsync(&h, tmp, sizeof(double2), cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  return std::sqrt(h.x);
}

extern "C" int lsms_solve(lsms_ctx* c, int nsrc, const double* src_xy, double tol, int maxiter,
                          const double* x0, double* beta_out, lsms_solve_info* info) {
  int rc;
  if ((rc = need_particles(c))) return rc;
  if ((rc = validate_sources(c, nsrc, src_xy))) return rc;
  if (!(tol > 0.0) || maxiter <= 0 || maxiter > GIVENS_MAX)
    return ctx_fail(c, LSMS_ERR_ARG, "tol must be > 0 and 0 < maxiter <= 4096");
  const long long L = (long long)c->n * c->P;
  cudaStream_t st = c->stream;
  if (info) { info->iters = 0; info->outer_iters = 0; info->rel_res = 0; info->rel_res_fp64 = 0; info->n_history = 0; }
  c->n_src = 0;
  c->src_xy.assign(src_xy, src_xy + 2 * nsrc);
  if ((rc = ensure(c, c->sol, (size_t)(nsrc > 0 ? nsrc : 1) * (L > 0 ? L : 1) * sizeof(double2)))) return rc;
  if (nsrc == 0) return LSMS_OK;
  if (L == 0) { c->n_src = nsrc; return LSMS_OK; }
  if ((rc = ensure(c, c->gm_r, (size_t)3 * L * sizeof(double2) + 64))) return rc;
  if ((rc = ensure(c, c->gm_x, (size_t)2 * L * sizeof(double2)))) return rc;
  if ((rc = ensure(c, c->ws_aux, (size_t)2 * nsrc * sizeof(double)))) return rc;
  cudaMemcpyAsync(c->ws_aux.ptr, src_xy, (size_t)2 * nsrc * sizeof(double), cudaMemcpyHostToDevice, st);
  double2* ainc = (double2*)c->sol.ptr;                 // a_inc for every source, replaced by beta
  if ((rc = incident_device(c, nsrc, (const double*)c->ws_aux.ptr, ainc, st))) return rc;
  double2* rhs = (double2*)c->gm_r.ptr;
  double2* res = rhs + L;
  double2* tmp = res + L;
  double2* xs = (double2*)c->gm_x.ptr;                  // scaled iterate
  double2* dx = xs + L;
  const bool mixed = c->precision == LSMS_MIXED;
  int status = LSMS_OK;
  for (int s = 0; s < nsrc; ++s) {
    double2* beta = ainc + (long long)s * L;
    launch_diag_mul(beta, c->d_scale_out + c->P, rhs, L, c->P, st);   // D S a_inc
    bool nonzero = false;
    if (x0) {
      cudaMemcpyAsync(dx, x0 + (size_t)2 * s * L, L * sizeof(double2), cudaMemcpyHostToDevice, st);
      launch_diag_scale(dx, c->d_hscale, xs, L, c->P, st);
      nonzero = true;
    }
    int it = 0, outer = 0, nh = 0;
    double r_est = 0.0, true_res = -1.0;
    int rc_s = LSMS_OK;
    double* hist = info ? info->history : nullptr;
    const int hcap = info ? info->history_cap : 0;
    if (!mixed) {
      rc_s = gmres_device(c, rhs, xs, nonzero, tol, maxiter, LSMS_APPLY_SCALED, &it, &r_est, hist, hcap, &nh, st);
      outer = 1;
    } else {
      // FP64 refinement: r = rhs - A x (FP64 operator); inner GMRES on the mixed operator.
      const double rhs_norm = norm_device(c, rhs, L, tmp, st);
      const double inv_norm = rhs_norm > 0 ? 1.0 / rhs_norm : 1.0;
      if (!nonzero) cudaMemsetAsync(xs, 0, L * sizeof(double2), st);
      const int max_outer = 20;
      const double inner_tol = 1e-5;
      rc_s = LSMS_ERR_NOT_CONVERGED;
      for (outer = 0; outer < max_outer && it < maxiter; ++outer) {
        double rn;
        if (outer == 0 && !nonzero) {
          // x = 0: the residual is the right-hand side itself
          cudaMemcpyAsync(res, rhs, L * sizeof(double2), cudaMemcpyDeviceToDevice, st);
          rn = 1.0;
        } else {
          if ((rc = apply_device(c, 1, xs, tmp, LSMS_APPLY_SCALED, st))) return rc;
          k_sub<<<grid_for(L, 256), 256, 0, st>>>(res, rhs, tmp, L);
          rn = norm_device(c, res, L, tmp, st) * inv_norm;
        }
        r_est = rn;
        true_res = rn;
        if (!std::isfinite(rn)) { rc_s = ctx_fail(c, LSMS_ERR_NONFINITE, "non-finite refinement residual"); break; }
        if (rn <= tol) { rc_s = LSMS_OK; break; }
        int it_in = 0;
        double r_in = 0.0;
        const double tol_in = std::max(inner_tol, 0.5 * tol / rn);
        int rci = gmres_device(c, res, dx, false, tol_in, maxiter - it, LSMS_APPLY_SCALED | LSMS_APPLY_MIXED,
                               &it_in, &r_in, hist, hcap, &nh, st);
        it += it_in;
        if (rci != LSMS_OK && rci != LSMS_ERR_NOT_CONVERGED) { rc_s = rci; break; }
        k_add<<<grid_for(L, 256), 256, 0, st>>>(xs, dx, L);              // x += dx
        true_res = -1.0;
      }
    }
    // true FP64 residual of the final iterate (the refinement loop already has it when it stopped
    // on a fresh residual)
    double rel_fp64 = true_res;
    if (rel_fp64 < 0.0) {
      if ((rc = apply_device(c, 1, xs, tmp, LSMS_APPLY_SCALED, st))) return rc;
      k_sub<<<grid_for(L, 256), 256, 0, st>>>(res, rhs, tmp, L);
      const double rn = norm_device(c, res, L, tmp, st);
      const double bn = norm_device(c, rhs, L, tmp, st);
      rel_fp64 = bn > 0 ? rn / bn : 0.0;
    }
    launch_diag_scale(xs, c->d_scale_in + c->P, beta, L, c->P, st);   // beta = D^{-1} b
    if (info) {
      info->iters += it;
      info->outer_iters += outer;
      info->rel_res = r_est;
      info->rel_res_fp64 = rel_fp64;
      info->n_history = nh;
    }
    if (rc_s != LSMS_OK && status == LSMS_OK) status = rc_s;
    if (rc_s == LSMS_ERR_NONFINITE) break;
  }
  if ((rc = check_cuda(c, "solve"))) return rc;
  c->n_src = nsrc;
  if (beta_out) {
    cudaMemcpyAsync(beta_out, c->sol.ptr, (size_t)nsrc * L * sizeof(double2), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    if ((rc = check_cuda(c, "solve copy"))) return rc;
  }
  if (status == LSMS_ERR_NOT_CONVERGED) ctx_fail(c, status, "GMRES reached maxiter");
  return status;
}
