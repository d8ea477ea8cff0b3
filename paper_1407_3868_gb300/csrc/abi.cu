// The C ABI of liblsms (include/lsms.h): argument checks, context state, device buffers, and the
// composition of the kernels into the operator, its individual steps, the solve and the field.
#include <cmath>
#include <cstring>
#include <new>

#include "lsms_internal.h"
#include "lsms_ops.h"

namespace {

thread_local std::string g_create_err;

int fail(lsms_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  else g_create_err = msg;
  return code;
}

template <typename T>
int upload(lsms_ctx* c, T** dptr, const std::vector<cplx>& v) {
  static_assert(sizeof(T) == sizeof(cplx), "complex layout");
  if (*dptr) cudaFree(*dptr);
  *dptr = nullptr;
  if (v.empty()) return LSMS_OK;
  if (cudaMalloc((void**)dptr, v.size() * sizeof(cplx)) != cudaSuccess)
    return fail(c, LSMS_ERR_OOM, "cudaMalloc failed for a constant table");
  if (cudaMemcpy(*dptr, v.data(), v.size() * sizeof(cplx), cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(c, LSMS_ERR_CUDA, "cudaMemcpy failed for a constant table");
  return LSMS_OK;
}

// exp(sign i lambda xc) per node: converts densities between absolute x and the centred x the
// device tables use.
std::vector<cplx> shift_phase(const lsms_ctx* c, double sign) {
  std::vector<cplx> ph(c->ns);
  for (int v = 0; v < c->ns; ++v) ph[v] = std::exp(cplx(0.0, sign) * c->nodes.lam[v] * c->xc);
  return ph;
}

}  // namespace

// ---------------------------------------------------------------------------------------------
// helpers shared with the solver (lsms_ops.h)
// ---------------------------------------------------------------------------------------------
int ctx_fail(lsms_ctx* c, int code, const std::string& msg) { return fail(c, code, msg); }

int ensure(lsms_ctx* c, DevBuf& b, size_t bytes) {
  if (bytes <= b.bytes && b.ptr) return LSMS_OK;
  if (b.ptr) cudaFree(b.ptr);
  b.ptr = nullptr;
  b.bytes = 0;
  if (bytes == 0) bytes = 16;
  if (cudaMalloc(&b.ptr, bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, LSMS_ERR_OOM, "cudaMalloc failed for a workspace of " + std::to_string(bytes) + " bytes");
  }
  b.bytes = bytes;
  return LSMS_OK;
}

int check_cuda(lsms_ctx* c, const char* where) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return fail(c, LSMS_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
  return LSMS_OK;
}

int need_particles(lsms_ctx* c) {
  if (!c) return LSMS_ERR_ARG;
  if (c->n < 0) return fail(c, LSMS_ERR_STATE, "call lsms_set_particles first");
  return LSMS_OK;
}

// Reflected coupling, FP64: alpha += E' (U * sigma(P, Q)), with P, Q from E * xs.
int reflection_f64(lsms_ctx* c, int nrhs, const double2* xs, double2* alpha, cudaStream_t st) {
  const int ns = c->ns, P = c->P, n = c->n;
  int rc;
  if ((rc = ensure(c, c->ws_g, (size_t)nrhs * 2 * ns * P * sizeof(double2)))) return rc;
  if ((rc = ensure(c, c->ws_v, (size_t)nrhs * 2 * ns * P * sizeof(double2)))) return rc;
  double2* G = (double2*)c->ws_g.ptr;
  double2* V = (double2*)c->ws_v.ptr;
  cudaMemsetAsync(G, 0, (size_t)nrhs * 2 * ns * P * sizeof(double2), st);
  launch_zgemm_rows(c->d_eagg, 2 * ns, n, xs, G, P, nrhs, st);
  launch_node_stage(ns, P, nrhs, G, c->d_fagg, nullptr, c->d_refl, c->d_udis, nullptr, nullptr, V, st);
  launch_zgemm_rows(c->d_edis, n, 2 * ns, V, alpha, P, nrhs, st);
  return LSMS_OK;
}

// y = x - s_out (T + R)(s_in x) on device buffers (the operator of lsms_apply_dev).
int apply_device(lsms_ctx* c, int nrhs, const double2* x, double2* y, int flags, cudaStream_t st) {
  int rc;
  if ((rc = need_particles(c))) return rc;
  if (is_batch(c)) return batch_apply(c, nrhs, x, y, flags, st);
  if (nrhs < 0) return fail(c, LSMS_ERR_ARG, "nrhs must be >= 0");
  const int n = c->n, P = c->P;
  const size_t len = (size_t)nrhs * n * P;
  if (len == 0) return LSMS_OK;
  const int mode = (flags & LSMS_APPLY_SCALED) ? 1 : 0;
  const bool mixed = (flags & LSMS_APPLY_MIXED) != 0;
  if ((rc = ensure(c, c->ws_xs, len * sizeof(double2)))) return rc;
  if ((rc = ensure(c, c->ws_alpha, len * sizeof(double2)))) return rc;
  double2* xs = (double2*)c->ws_xs.ptr;
  const bool given = (flags & LSMS_APPLY_TRANSLATION_GIVEN) && c->alpha_given;
  double2* alpha = given ? c->alpha_given : (double2*)c->ws_alpha.ptr;
  int launches = 0;
  launch_scale_in(x, c->d_scale_in + mode * P, xs, nrhs, n, P, st);
  ++launches;
  if (c->timing) cudaEventRecord(c->ev[0], st);
  // mixed: the reflected coupling (tensor-core contour contractions) on the side stream, beside
  // the translation; its result is added into alpha after the join (same arithmetic, same order)
  const bool overlap = mixed && c->side && !(flags & LSMS_APPLY_NO_TRANSLATION) &&
                       !(flags & LSMS_APPLY_NO_REFLECTION);
  if (overlap) {
    cudaEventRecord(c->ev_fork, st);
    cudaStreamWaitEvent(c->side, c->ev_fork, 0);
    if ((rc = reflection_mixed_stage(c, nrhs, xs, c->side))) return rc;
    cudaEventRecord(c->ev_join, c->side);
  }
  if (!(flags & LSMS_APPLY_NO_TRANSLATION)) {
    // box method (fmm.cu): per right-hand side M2M, five transform passes, the direct offsets
    // and L2L; then the near field (FP64: one kernel; mixed: FP32 copy of xs and the pair-list
    // kernel).  All pairs: FP64 one kernel; mixed: FP32 copy of xs, the translation (+ the
    // partial-sum reduction, or the packing of the tensor-core operands) and the near pairs
    if (given) {
      // computed for every layout of the batch at once (translate_mixed_batch)
      cudaStreamWaitEvent(st, c->alpha_ready, 0);
    } else if (c->fmm.ready && (c->fmm.scope == 0 || (flags & LSMS_APPLY_RESIDUAL_INTERNAL))) {
      if (c->fmm.far) launches += (c->fmm.dmin > 2 ? 8 : 7) * nrhs;
      launches += mixed ? 2 : 1;
      if ((rc = fmm_translate(c, nrhs, xs, alpha, mixed, st))) return rc;
    } else if (mixed) {
      launches += 3 + (c->near_nnz > 0 ? 1 : 0);
      if ((rc = translate_mixed(c, nrhs, xs, alpha, st))) return rc;
    } else {
      launches += 1;
      launch_translate_f64(c->d_cx, c->d_cy, n, c->p, c->k2, xs, alpha, nrhs, st);
    }
  } else {
    cudaMemsetAsync(alpha, 0, len * sizeof(double2), st);
  }
  if (c->timing) cudaEventRecord(c->ev[1], st);
  if (!(flags & LSMS_APPLY_NO_REFLECTION)) {
    if (overlap) {
      cudaStreamWaitEvent(st, c->ev_join, 0);
      reflection_mixed_add(c, nrhs, alpha, st);
    } else if (mixed) {
      if ((rc = reflection_mixed(c, nrhs, xs, alpha, st))) return rc;
    } else {
      if ((rc = reflection_f64(c, nrhs, xs, alpha, st))) return rc;
    }
    launches += mixed ? 5 : 3;   // split, GEMM, per-node stage, GEMM, add / GEMM, stage, GEMM
  }
  if (c->timing) cudaEventRecord(c->ev[2], st);
  if (c->dense && !(flags & LSMS_APPLY_ALPHA))
    launch_scatter_dense(x, alpha, c->d_smt + (size_t)mode * P * P,
                         c->has_theta ? (const double*)c->theta_buf.ptr : nullptr, nrhs, n, P, y, st);
  else
    launch_combine(x, alpha, c->d_scale_out + mode * P, y, nrhs, n, P, (flags & LSMS_APPLY_ALPHA) ? 1 : 0, st);
  ++launches;
  c->last_launches = launches;
  return check_cuda(c, "apply");
}

// alpha_rows[r][i] += alpha_full[r][row0 + i] for i < nrows (complex, P per disc)
__global__ void k_add_rows(const double2* __restrict__ full, int n, int row0, int nrows, int P, int nrhs,
                           double2* __restrict__ rows) {
  const long long total = (long long)nrhs * nrows * P;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long per = (long long)nrows * P;
    const long long r = i / per, e = i - r * per;
    const double2 v = full[(r * n + row0) * P + e];
    rows[i] = make_double2(rows[i].x + v.x, rows[i].y + v.y);
  }
}

// The operator for the target rows row0 .. row1 - 1 of x (all discs): y_rows = x_rows - S (T x + R x)_rows.
// The translation runs for those rows only (the O(N^2) part, split between ranks); the reflected
// coupling is formed whole (aggregate over every disc, per-node response, disaggregate) and its
// rows taken, so that a rank needs only the gathered x.
int apply_rows_device(lsms_ctx* c, int nrhs, int row0, int row1, const double2* x, double2* y, int flags,
                      cudaStream_t st) {
  int rc;
  if ((rc = need_particles(c))) return rc;
  if (is_batch(c)) return fail(c, LSMS_ERR_ARG, "apply_rows: not available on a layout batch");
  const int n = c->n, P = c->P;
  if (nrhs < 0 || row0 < 0 || row1 < row0 || row1 > n)
    return fail(c, LSMS_ERR_ARG, "apply_rows: need nrhs >= 0 and 0 <= row0 <= row1 <= number of discs");
  if (c->fmm.ready && c->fmm.scope == LSMS_FMM_ALL)
    return fail(c, LSMS_ERR_ARG, "apply_rows: the translation through boxes is on (use LSMS_FMM_RESIDUAL or turn it off)");
  const int nrows = row1 - row0;
  const size_t len = (size_t)nrhs * n * P, len_rows = (size_t)nrhs * nrows * P;
  if (len_rows == 0) return LSMS_OK;
  const int mode = (flags & LSMS_APPLY_SCALED) ? 1 : 0;
  const bool mixed = (flags & LSMS_APPLY_MIXED) != 0;
  if ((rc = ensure(c, c->ws_xs, len * sizeof(double2)))) return rc;
  if ((rc = ensure(c, c->ws_alpha, len * sizeof(double2)))) return rc;
  if ((rc = ensure(c, c->ws_rows, len_rows * sizeof(double2)))) return rc;
  double2* xs = (double2*)c->ws_xs.ptr;
  double2* alpha = (double2*)c->ws_alpha.ptr;          // reflected coupling, all rows
  double2* arows = (double2*)c->ws_rows.ptr;           // translation + reflection, the rows
  launch_scale_in(x, c->d_scale_in + mode * P, xs, nrhs, n, P, st);
  if (!(flags & LSMS_APPLY_NO_TRANSLATION)) {
    if (mixed) {
      if ((rc = translate_mixed_rows(c, nrhs, xs, arows, row0, nrows, st))) return rc;
    } else {
      launch_translate_f64(c->d_cx, c->d_cy, n, c->p, c->k2, xs, arows, nrhs, st, row0, nrows);
    }
  } else {
    cudaMemsetAsync(arows, 0, len_rows * sizeof(double2), st);
  }
  if (!(flags & LSMS_APPLY_NO_REFLECTION)) {
    cudaMemsetAsync(alpha, 0, len * sizeof(double2), st);
    if ((rc = mixed ? reflection_mixed(c, nrhs, xs, alpha, st) : reflection_f64(c, nrhs, xs, alpha, st))) return rc;
    k_add_rows<<<(int)std::min<long long>((len_rows + 255) / 256, 152 * 16), 256, 0, st>>>(alpha, n, row0, nrows, P,
                                                                                        nrhs, arows);
  }
  for (int r = 0; r < nrhs; ++r) {
    const double2* xr = x + ((size_t)r * n + row0) * P;
    const double2* ar = arows + (size_t)r * nrows * P;
    double2* yr = y + (size_t)r * nrows * P;
    if (c->dense && !(flags & LSMS_APPLY_ALPHA))
      launch_scatter_dense(xr, ar, c->d_smt + (size_t)mode * P * P,
                           c->has_theta ? (const double*)c->theta_buf.ptr + row0 : nullptr, 1, nrows, P, yr, st);
    else
      launch_combine(xr, ar, c->d_scale_out + mode * P, yr, 1, nrows, P, (flags & LSMS_APPLY_ALPHA) ? 1 : 0, st);
  }
  return check_cuda(c, "apply_rows");
}

extern "C" int lsms_apply_rows_dev(lsms_ctx* c, int nrhs, int row0, int row1, const double* x_dev, double* y_dev,
                                   int flags, void* stream) {
  if (!c) return LSMS_ERR_ARG;
  if (nrhs > 0 && row1 > row0 && (!x_dev || !y_dev)) return fail(c, LSMS_ERR_ARG, "apply_rows: NULL array");
  return apply_rows_device(c, nrhs, row0, row1, (const double2*)x_dev, (double2*)y_dev, flags, (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------------------------
// create / destroy / particles
// ---------------------------------------------------------------------------------------------
int create_stack(const std::vector<cplx>& kc, const std::vector<double>& ds, int layer, double kp,
                 double radius, int p, const lsms_contour* contour, int precision, lsms_ctx** out) {
  if (!out) return fail(nullptr, LSMS_ERR_ARG, "out is NULL");
  *out = nullptr;
  const int L = (int)kc.size();
  if (L < 3 || (int)ds.size() != L - 2 || layer < 2 || layer > L - 1)
    return fail(nullptr, LSMS_ERR_ARG, "need n_layers >= 3, n_layers - 2 thicknesses and 2 <= particle_layer <= n_layers - 1");
  for (const cplx& v : kc)
    if (!std::isfinite(v.real()) || !std::isfinite(v.imag()) || !(v.real() > 0.0) || !(v.imag() >= 0.0))
      return fail(nullptr, LSMS_ERR_ARG, "wavenumbers must be finite with Re k > 0 and Im k >= 0");
  if (kc[0].imag() != 0.0 || kc[layer - 1].imag() != 0.0)
    return fail(nullptr, LSMS_ERR_ARG, "the source half-space (layer 1) and the particle layer must be lossless");
  std::vector<double> ks(L);
  for (int j = 0; j < L; ++j) ks[j] = kc[j].real();
  for (double v : ds)
    if (!std::isfinite(v) || !(v > 0.0)) return fail(nullptr, LSMS_ERR_ARG, "thicknesses must be finite and > 0");
  if (!std::isfinite(kp) || !(kp > 0.0) || !std::isfinite(radius) || !(radius > 0.0))
    return fail(nullptr, LSMS_ERR_ARG, "kp and radius must be finite and > 0");
  const double d = ds[layer - 2];
  if (!(radius < 0.5 * d)) return fail(nullptr, LSMS_ERR_ARG, "radius must be < half the disc layer's thickness");
  if (p < 0 || p > LSMS_MAX_P) return fail(nullptr, LSMS_ERR_ARG, "p must be in [0, 15]");
  if (!contour) return fail(nullptr, LSMS_ERR_ARG, "contour is NULL");
  if (precision != LSMS_FP64 && precision != LSMS_MIXED)
    return fail(nullptr, LSMS_ERR_ARG, "precision must be LSMS_FP64 or LSMS_MIXED");
  lsms_ctx* c = new (std::nothrow) lsms_ctx();
  if (!c) return fail(nullptr, LSMS_ERR_OOM, "host allocation failed");
  c->ks = ks;
  c->kc = kc;
  c->ds = ds;
  c->layer = layer;
  c->depth = 0.0;
  for (int j = 2; j < layer; ++j) c->depth += ds[j - 2];
  c->k1 = ks[0]; c->k2 = ks[layer - 1]; c->k3 = ks[L - 1]; c->d = d; c->kp = kp; c->R = radius;
  c->p = p; c->P = 2 * p + 1; c->precision = precision; c->contour = *contour;
  const double k2 = c->k2;
  std::string err;
  int rc = build_contour(*contour, ks, c->nodes.lam, c->nodes.wt, err);
  if (rc) { delete c; return fail(nullptr, rc, err); }
  c->ns = (int)c->nodes.lam.size();
  c->S = mie_diagonal(p, k2, kp, radius);
  c->hscale = hankel_scale(p, k2, radius);
  build_node_tables(c);
  for (const cplx& s : c->S)
    if (!std::isfinite(s.real()) || !std::isfinite(s.imag())) { delete c; return fail(nullptr, LSMS_ERR_ARG, "non-finite scattering matrix"); }
  if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return fail(nullptr, LSMS_ERR_CUDA, "cudaStreamCreate failed (no CUDA device?)");
  }
  if (cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    lsms_destroy(c);
    return fail(nullptr, LSMS_ERR_CUDA, "side stream creation failed");
  }
  std::vector<cplx> s_out(2 * c->P);
  std::vector<double> s_in(2 * c->P);
  for (int q = 0; q < c->P; ++q) {
    s_in[q] = 1.0;
    s_in[c->P + q] = 1.0 / c->hscale[q];
    s_out[q] = c->S[q];
    s_out[c->P + q] = c->hscale[q] * c->S[q];
  }
  if ((rc = upload(c, &c->d_lam, c->nodes.lam)) || (rc = upload(c, &c->d_g1, c->nodes.g1)) ||
      (rc = upload(c, &c->d_refl, c->nodes.refl)) || (rc = upload(c, &c->d_inc, c->nodes.inc)) ||
      (rc = upload(c, &c->d_field, c->nodes.field)) || (rc = upload(c, &c->d_fagg, c->nodes.fagg)) ||
      (rc = upload(c, &c->d_udis, c->nodes.udis)) || (rc = upload(c, &c->d_scale_out, s_out))) {
    std::string m = c->err;
    lsms_destroy(c);
    return fail(nullptr, rc, m);
  }
  if (cudaMalloc((void**)&c->d_scale_in, s_in.size() * sizeof(double)) != cudaSuccess ||
      cudaMemcpy(c->d_scale_in, s_in.data(), s_in.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMalloc((void**)&c->d_hscale, c->P * sizeof(double)) != cudaSuccess ||
      cudaMemcpy(c->d_hscale, c->hscale.data(), c->P * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
    lsms_destroy(c);
    return fail(nullptr, LSMS_ERR_CUDA, "upload of the order scales failed");
  }
  if ((rc = upload(c, &c->d_g2, c->nodes.g2))) { std::string m = c->err; lsms_destroy(c); return fail(nullptr, rc, m); }
  if (cudaMallocHost((void**)&c->h_pinned, 64 * sizeof(double)) != cudaSuccess) {
    lsms_destroy(c);
    return fail(nullptr, LSMS_ERR_CUDA, "cudaMallocHost failed");
  }
  *out = c;
  return LSMS_OK;
}

extern "C" int lsms_create(double k1, double k2, double k3, double d, double kp, double radius,
                           int p, const lsms_contour* contour, int precision, lsms_ctx** out) {
  return create_stack({cplx(k1, 0.0), cplx(k2, 0.0), cplx(k3, 0.0)}, {d}, 2, kp, radius, p, contour, precision, out);
}

extern "C" int lsms_create_stack(int n_layers, const double* k, const double* thickness, int particle_layer,
                                 double kp, double radius, int p, const lsms_contour* contour,
                                 int precision, lsms_ctx** out) {
  if (n_layers < 3 || !k || !thickness) {
    if (out) *out = nullptr;
    return fail(nullptr, LSMS_ERR_ARG, "need n_layers >= 3 and non-NULL k and thickness arrays");
  }
  std::vector<cplx> kc(n_layers);
  for (int j = 0; j < n_layers; ++j) kc[j] = cplx(k[j], 0.0);
  return create_stack(kc, std::vector<double>(thickness, thickness + n_layers - 2), particle_layer, kp, radius, p,
                      contour, precision, out);
}

extern "C" int lsms_create_stack_c(int n_layers, const double* k, const double* thickness, int particle_layer,
                                   double kp, double radius, int p, const lsms_contour* contour,
                                   int precision, lsms_ctx** out) {
  if (n_layers < 3 || !k || !thickness) {
    if (out) *out = nullptr;
    return fail(nullptr, LSMS_ERR_ARG, "need n_layers >= 3 and non-NULL k and thickness arrays");
  }
  std::vector<cplx> kc(n_layers);
  for (int j = 0; j < n_layers; ++j) kc[j] = cplx(k[2 * j], k[2 * j + 1]);
  return create_stack(kc, std::vector<double>(thickness, thickness + n_layers - 2), particle_layer, kp, radius, p,
                      contour, precision, out);
}

extern "C" void lsms_destroy(lsms_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->side) cudaStreamSynchronize(c->side);
  batch_free(c);
  void* ptrs[] = {c->d_lam, c->d_g1, c->d_g2, c->d_refl, c->d_inc, c->d_field, c->d_fagg, c->d_udis,
                  c->d_scale_in, c->d_hscale, c->d_scale_out, c->d_cx, c->d_cy, c->d_eagg, c->d_edis,
                  c->d_eagg_lp, c->d_edis_lp, c->d_lp_misc, c->d_near_ptr, c->d_near_idx, c->d_near_h,
                  c->d_smt};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  DevBuf* bufs[] = {&c->ws_x, &c->ws_y, &c->ws_xs, &c->ws_alpha, &c->ws_g, &c->ws_v, &c->ws_pq,
                    &c->ws_sig, &c->ws_aux, &c->ws_rows, &c->gm_v, &c->gm_h, &c->gm_small, &c->gm_x, &c->gm_r,
                    &c->gm_w, &c->sol, &c->ws_lp, &c->ws_tcb, &c->gm_b, &c->gm_mask, &c->gm_off, &c->theta_buf};
  for (DevBuf* b : bufs)
    if (b->ptr) cudaFree(b->ptr);
  tc_free(c);
  fmm_free(c);
  if (c->h_pinned) cudaFreeHost(c->h_pinned);
  if (c->gm_ring) cudaFreeHost(c->gm_ring);
  for (cudaEvent_t e : c->ev)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : c->gm_ev)
    if (e) cudaEventDestroy(e);
  if (c->side) cudaStreamSynchronize(c->side);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

extern "C" int lsms_set_particles(lsms_ctx* c, int n, const double* xy) {
  if (!c) return LSMS_ERR_ARG;
  if (n < 0 || (n > 0 && !xy)) return fail(c, LSMS_ERR_ARG, "n must be >= 0 and centres non-NULL");
  std::string err;
  int rc = validate_geometry(c, n, xy, err);
  if (rc) return fail(c, rc, err);
  cudaStreamSynchronize(c->stream);
  batch_free(c);
  c->cx.assign(n, 0.0);
  c->cy.assign(n, 0.0);
  double xmin = 0.0, xmax = 0.0;
  for (int j = 0; j < n; ++j) {
    c->cx[j] = xy[2 * j];
    c->cy[j] = xy[2 * j + 1] + c->depth;       // the disc layer's frame: its top interface at y = 0
    if (j == 0 || xy[2 * j] < xmin) xmin = xy[2 * j];
    if (j == 0 || xy[2 * j] > xmax) xmax = xy[2 * j];
  }
  c->xc = n > 0 ? 0.5 * (xmin + xmax) : 0.0;
  std::vector<double> xs(n);
  for (int j = 0; j < n; ++j) xs[j] = c->cx[j] - c->xc;
  tc_free(c);
  void* old[] = {c->d_cx, c->d_cy, c->d_eagg, c->d_edis, c->d_eagg_lp, c->d_edis_lp, c->d_lp_misc};
  for (void* q : old)
    if (q) cudaFree(q);
  c->d_cx = c->d_cy = nullptr;
  c->d_eagg = c->d_edis = nullptr;
  c->d_eagg_lp = c->d_edis_lp = nullptr;
  c->d_lp_misc = nullptr;
  c->n = n;
  c->n_src = 0;
  c->has_theta = false;                      // orientations refer to the previous particles
  const size_t nb = (size_t)(n > 0 ? n : 1) * sizeof(double);
  const size_t eb = (size_t)2 * c->ns * (n > 0 ? n : 1) * sizeof(double2);
  if (cudaMalloc((void**)&c->d_cx, nb) != cudaSuccess || cudaMalloc((void**)&c->d_cy, nb) != cudaSuccess ||
      cudaMalloc((void**)&c->d_eagg, eb) != cudaSuccess || cudaMalloc((void**)&c->d_edis, eb) != cudaSuccess) {
    cudaGetLastError();
    c->n = -1;
    return fail(c, LSMS_ERR_OOM, "cudaMalloc failed for the layout tables");
  }
  if (n > 0) {
    cudaMemcpy(c->d_cx, xs.data(), n * sizeof(double), cudaMemcpyHostToDevice);
    cudaMemcpy(c->d_cy, c->cy.data(), n * sizeof(double), cudaMemcpyHostToDevice);
    launch_etables(c->d_cx, c->d_cy, n, c->d_lam, c->d_g2, c->ns, c->d, c->d_eagg, c->d_edis, c->stream);
    cudaStreamSynchronize(c->stream);
    if ((rc = check_cuda(c, "set_particles"))) return rc;
    if ((rc = build_lowp_tables(c))) return rc;
  }
  if (c->fmm.box_width > 0.0) return fmm_setup(c);
  fmm_free(c);
  return LSMS_OK;
}

// ---------------------------------------------------------------------------------------------
// operator
// ---------------------------------------------------------------------------------------------
// True when every one of the n doubles is finite: v * 0 is NaN exactly for NaN and +-Inf, and the
// sum has no early exit, so the loop vectorises (a 5000-disc vector takes tens of microseconds).
static bool host_finite(const double* h, size_t n) {
  double acc = 0.0;
  for (size_t i = 0; i < n; ++i) acc += h[i] * 0.0;
  return acc == 0.0;
}
static int need_finite(lsms_ctx* c, const double* h, size_t ncplx, const char* what) {
  if (h && !host_finite(h, 2 * ncplx)) return fail(c, LSMS_ERR_ARG, std::string("non-finite value in ") + what);
  return LSMS_OK;
}

static int copy_in(lsms_ctx* c, DevBuf& b, const double* h, size_t ncplx) {
  int rc;
  if ((rc = ensure(c, b, ncplx * sizeof(double2)))) return rc;
  if (ncplx && cudaMemcpyAsync(b.ptr, h, ncplx * sizeof(double2), cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
    return fail(c, LSMS_ERR_CUDA, "host to device copy failed");
  return LSMS_OK;
}
static int copy_out(lsms_ctx* c, double* h, const void* d, size_t ncplx) {
  if (ncplx && cudaMemcpyAsync(h, d, ncplx * sizeof(double2), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
    return fail(c, LSMS_ERR_CUDA, "device to host copy failed");
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return check_cuda(c, "synchronize");
  return check_cuda(c, "copy_out");
}

extern "C" int lsms_apply_ex(lsms_ctx* c, int nrhs, const double* x, double* y, int flags) {
  int rc;
  if ((rc = need_particles(c))) return rc;
  if (nrhs < 0 || (nrhs > 0 && c->n > 0 && (!x || !y))) return fail(c, LSMS_ERR_ARG, "bad nrhs or NULL array");
  const size_t len = (size_t)nrhs * c->n * c->P;
  if (len == 0) return LSMS_OK;
  if ((rc = need_finite(c, x, len, "the coefficients x"))) return rc;
  if ((rc = copy_in(c, c->ws_x, x, len))) return rc;
  if ((rc = ensure(c, c->ws_y, len * sizeof(double2)))) return rc;
  if ((rc = apply_device(c, nrhs, (const double2*)c->ws_x.ptr, (double2*)c->ws_y.ptr, flags, c->stream))) return rc;
  if ((rc = copy_out(c, y, c->ws_y.ptr, len))) return rc;
  if (!(flags & LSMS_APPLY_MIXED)) return LSMS_OK;
  return is_batch(c) ? batch_mixed_check(c) : mixed_check(c);
}

extern "C" int lsms_apply(lsms_ctx* c, int nrhs, const double* x, double* y) {
  if (!c) return LSMS_ERR_ARG;
  return lsms_apply_ex(c, nrhs, x, y, c->precision == LSMS_MIXED ? LSMS_APPLY_MIXED : 0);
}

extern "C" int lsms_apply_dev(lsms_ctx* c, int nrhs, const double* x, double* y, int flags, void* stream) {
  return apply_device(c, nrhs, (const double2*)x, (double2*)y, flags, (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------------------------
// individual steps
// ---------------------------------------------------------------------------------------------
extern "C" int lsms_translate(lsms_ctx* c, int nrhs, const double* beta, double* alpha, int precision) {
  int rc;
  if ((rc = need_particles(c))) return rc;
  if (is_batch(c)) return fail(c, LSMS_ERR_ARG, "not available on a layout batch");
  const size_t len = (size_t)nrhs * c->n * c->P;
  if (nrhs < 0) return fail(c, LSMS_ERR_ARG, "nrhs must be >= 0");
  if (len == 0) return LSMS_OK;
  if ((rc = need_finite(c, beta, len, "beta"))) return rc;
  if ((rc = copy_in(c, c->ws_x, beta, len))) return rc;
  if ((rc = ensure(c, c->ws_alpha, len * sizeof(double2)))) return rc;
  if (c->fmm.ready && c->fmm.scope == 0) {
    if ((rc = fmm_translate(c, nrhs, (const double2*)c->ws_x.ptr, (double2*)c->ws_alpha.ptr,
                            precision == LSMS_MIXED, c->stream)))
      return rc;
  } else if (precision == LSMS_MIXED) {
    if ((rc = translate_mixed(c, nrhs, (const double2*)c->ws_x.ptr, (double2*)c->ws_alpha.ptr, c->stream))) return rc;
  } else
    launch_translate_f64(c->d_cx, c->d_cy, c->n, c->p, c->k2, (const double2*)c->ws_x.ptr, (double2*)c->ws_alpha.ptr, nrhs, c->stream);
  if ((rc = check_cuda(c, "translate"))) return rc;
  return copy_out(c, alpha, c->ws_alpha.ptr, len);
}

extern "C" int lsms_aggregate(lsms_ctx* c, int nrhs, const double* beta, double* p_plus,
                              double* q_minus, int precision) {
  int rc;
  if ((rc = need_particles(c))) return rc;
  if (is_batch(c)) return fail(c, LSMS_ERR_ARG, "not available on a layout batch");
  if (nrhs < 0) return fail(c, LSMS_ERR_ARG, "nrhs must be >= 0");
  const int ns = c->ns, P = c->P;
  const size_t len = (size_t)nrhs * c->n * P;
  if (nrhs == 0) return LSMS_OK;
  if ((rc = need_finite(c, beta, len, "beta"))) return rc;
  if ((rc = copy_in(c, c->ws_x, beta, len ? len : 1))) return rc;
  if ((rc = ensure(c, c->ws_g, (size_t)nrhs * 2 * ns * P * sizeof(double2)))) return rc;
  if ((rc = ensure(c, c->ws_pq, (size_t)nrhs * 2 * ns * sizeof(double2)))) return rc;
  double2* G = (double2*)c->ws_g.ptr;
  cudaMemsetAsync(G, 0, (size_t)nrhs * 2 * ns * P * sizeof(double2), c->stream);
  if (precision == LSMS_MIXED) {
    if ((rc = aggregate_mixed(c, nrhs, (const double2*)c->ws_x.ptr, G, c->stream))) return rc;
  } else {
    launch_zgemm_rows(c->d_eagg, 2 * ns, c->n, (const double2*)c->ws_x.ptr, G, P, nrhs, c->stream);
  }
  launch_node_stage(ns, P, nrhs, G, c->d_fagg, nullptr, nullptr, nullptr, (double2*)c->ws_pq.ptr,
                    nullptr, nullptr, c->stream);
  if ((rc = check_cuda(c, "aggregate"))) return rc;
  std::vector<cplx> pq((size_t)nrhs * 2 * ns);
  if ((rc = copy_out(c, (double*)pq.data(), c->ws_pq.ptr, pq.size()))) return rc;
  if (precision == LSMS_MIXED && (rc = mixed_check(c))) return rc;
  // the device works in x - xc; densities in absolute x carry exp(-i lambda xc)
  const std::vector<cplx> ph = shift_phase(c, -1.0);
  cplx* pp = reinterpret_cast<cplx*>(p_plus);
  cplx* qm = reinterpret_cast<cplx*>(q_minus);
  for (int r = 0; r < nrhs; ++r)
    for (int v = 0; v < ns; ++v) {
      pp[(size_t)r * ns + v] = pq[(size_t)r * 2 * ns + v] * ph[v];
      qm[(size_t)r * ns + v] = pq[(size_t)r * 2 * ns + ns + v] * ph[v];
    }
  return LSMS_OK;
}

extern "C" int lsms_reflect(lsms_ctx* c, int nrhs, const double* p_plus, const double* q_minus,
                            double* s_plus, double* s_minus) {
  if (!c) return LSMS_ERR_ARG;
  if (nrhs <= 0) return nrhs == 0 ? LSMS_OK : fail(c, LSMS_ERR_ARG, "nrhs must be >= 0");
  const int ns = c->ns;
  int rc;
  if ((rc = need_finite(c, p_plus, (size_t)nrhs * ns, "P+"))) return rc;
  if ((rc = need_finite(c, q_minus, (size_t)nrhs * ns, "Q-"))) return rc;
  std::vector<cplx> pq((size_t)nrhs * 2 * ns);
  for (int r = 0; r < nrhs; ++r) {
    std::memcpy(static_cast<void*>(pq.data() + (size_t)r * 2 * ns), p_plus + (size_t)r * ns * 2, ns * sizeof(cplx));
    std::memcpy(static_cast<void*>(pq.data() + (size_t)r * 2 * ns + ns), q_minus + (size_t)r * ns * 2, ns * sizeof(cplx));
  }
  if ((rc = copy_in(c, c->ws_pq, (const double*)pq.data(), pq.size()))) return rc;
  if ((rc = ensure(c, c->ws_sig, pq.size() * sizeof(double2)))) return rc;
  launch_node_stage(ns, c->P, nrhs, nullptr, nullptr, (const double2*)c->ws_pq.ptr, c->d_refl, nullptr,
                    nullptr, (double2*)c->ws_sig.ptr, nullptr, c->stream);
  if ((rc = check_cuda(c, "reflect"))) return rc;
  if ((rc = copy_out(c, (double*)pq.data(), c->ws_sig.ptr, pq.size()))) return rc;
  for (int r = 0; r < nrhs; ++r) {
    std::memcpy(s_plus + (size_t)r * ns * 2, pq.data() + (size_t)r * 2 * ns, ns * sizeof(cplx));
    std::memcpy(s_minus + (size_t)r * ns * 2, pq.data() + (size_t)r * 2 * ns + ns, ns * sizeof(cplx));
  }
  return LSMS_OK;
}

extern "C" int lsms_disaggregate(lsms_ctx* c, int nrhs, const double* s_plus, const double* s_minus,
                                 double* alpha, int precision) {
  int rc;
  if ((rc = need_particles(c))) return rc;
  if (is_batch(c)) return fail(c, LSMS_ERR_ARG, "not available on a layout batch");
  if (nrhs < 0) return fail(c, LSMS_ERR_ARG, "nrhs must be >= 0");
  const int ns = c->ns, P = c->P;
  const size_t len = (size_t)nrhs * c->n * P;
  if (len == 0) return LSMS_OK;
  if ((rc = need_finite(c, s_plus, (size_t)nrhs * ns, "sigma+"))) return rc;
  if ((rc = need_finite(c, s_minus, (size_t)nrhs * ns, "sigma-"))) return rc;
  std::vector<cplx> sg((size_t)nrhs * 2 * ns);
  const std::vector<cplx> ph = shift_phase(c, 1.0);
  const cplx* sp = reinterpret_cast<const cplx*>(s_plus);
  const cplx* sm = reinterpret_cast<const cplx*>(s_minus);
  for (int r = 0; r < nrhs; ++r)
    for (int v = 0; v < ns; ++v) {
      sg[(size_t)r * 2 * ns + v] = sp[(size_t)r * ns + v] * ph[v];
      sg[(size_t)r * 2 * ns + ns + v] = sm[(size_t)r * ns + v] * ph[v];
    }
  if ((rc = copy_in(c, c->ws_sig, (const double*)sg.data(), sg.size()))) return rc;
  if ((rc = ensure(c, c->ws_v, (size_t)nrhs * 2 * ns * P * sizeof(double2)))) return rc;
  if ((rc = ensure(c, c->ws_alpha, len * sizeof(double2)))) return rc;
  launch_sigma_to_v(ns, P, nrhs, (const double2*)c->ws_sig.ptr, c->d_udis, (double2*)c->ws_v.ptr, c->stream);
  cudaMemsetAsync(c->ws_alpha.ptr, 0, len * sizeof(double2), c->stream);
  if (precision == LSMS_MIXED) {
    if ((rc = disaggregate_mixed(c, nrhs, (const double2*)c->ws_v.ptr, (double2*)c->ws_alpha.ptr, c->stream))) return rc;
  } else {
    launch_zgemm_rows(c->d_edis, c->n, 2 * ns, (const double2*)c->ws_v.ptr, (double2*)c->ws_alpha.ptr, P, nrhs, c->stream);
  }
  if ((rc = check_cuda(c, "disaggregate"))) return rc;
  if ((rc = copy_out(c, alpha, c->ws_alpha.ptr, len))) return rc;
  return precision == LSMS_MIXED ? mixed_check(c) : LSMS_OK;
}

// a_inc of line sources on the device: [nsrc][N][P] into `out`.
int incident_device(lsms_ctx* c, int nsrc, const double* d_src, double2* out, cudaStream_t st) {
  int rc;
  const int ns = c->ns, P = c->P;
  if ((rc = ensure(c, c->ws_sig, (size_t)nsrc * 2 * ns * sizeof(double2)))) return rc;
  if ((rc = ensure(c, c->ws_v, (size_t)nsrc * 2 * ns * P * sizeof(double2)))) return rc;
  launch_incident_sigma(ns, nsrc, d_src, c->xc, c->d_lam, c->d_g1, c->d_inc, (double2*)c->ws_sig.ptr, st);
  launch_sigma_to_v(ns, P, nsrc, (const double2*)c->ws_sig.ptr, c->d_udis, (double2*)c->ws_v.ptr, st);
  cudaMemsetAsync(out, 0, (size_t)nsrc * c->n * P * sizeof(double2), st);
  launch_zgemm_rows(c->d_edis, c->n, 2 * ns, (const double2*)c->ws_v.ptr, out, P, nsrc, st);
  return check_cuda(c, "incident");
}

int validate_sources(lsms_ctx* c, int nsrc, const double* xy) {
  if (nsrc < 0 || (nsrc > 0 && !xy)) return fail(c, LSMS_ERR_ARG, "bad source array");
  for (int s = 0; s < nsrc; ++s)
    if (!std::isfinite(xy[2 * s]) || !std::isfinite(xy[2 * s + 1]) || !(xy[2 * s + 1] > 0.0))
      return fail(c, LSMS_ERR_ARG, "sources must be finite and lie in the top layer (y > 0)");
  return LSMS_OK;
}

extern "C" int lsms_incident(lsms_ctx* c, int nsrc, const double* src_xy, double* a_inc) {
  int rc;
  if ((rc = need_particles(c))) return rc;
  if (is_batch(c)) return fail(c, LSMS_ERR_ARG, "not available on a layout batch");
  if ((rc = validate_sources(c, nsrc, src_xy))) return rc;
  const size_t len = (size_t)nsrc * c->n * c->P;
  if (len == 0) return LSMS_OK;
  if ((rc = ensure(c, c->ws_aux, (size_t)nsrc * 2 * sizeof(double)))) return rc;
  cudaMemcpyAsync(c->ws_aux.ptr, src_xy, (size_t)nsrc * 2 * sizeof(double), cudaMemcpyHostToDevice, c->stream);
  if ((rc = ensure(c, c->ws_alpha, len * sizeof(double2)))) return rc;
  if ((rc = incident_device(c, nsrc, (const double*)c->ws_aux.ptr, (double2*)c->ws_alpha.ptr, c->stream))) return rc;
  return copy_out(c, a_inc, c->ws_alpha.ptr, len);
}

// ---------------------------------------------------------------------------------------------
// field
// ---------------------------------------------------------------------------------------------
extern "C" int lsms_eval_field(lsms_ctx* c, int src_index, int ntgt, const double* tgt, int which,
                               double* out) {
  int rc;
  if ((rc = need_particles(c))) return rc;
  if (is_batch(c)) return batch_eval_field(c, src_index, ntgt, tgt, which, out);
  if (src_index < 0 || src_index >= c->n_src) return fail(c, LSMS_ERR_STATE, "no solution for that source: call lsms_solve first");
  if (which < LSMS_FIELD_TOTAL || which > LSMS_FIELD_PARTICLE) return fail(c, LSMS_ERR_ARG, "bad field selector");
  if (ntgt < 0 || (ntgt > 0 && (!tgt || !out))) return fail(c, LSMS_ERR_ARG, "bad target array");
  for (int t = 0; t < ntgt; ++t)
    if (!std::isfinite(tgt[2 * t]) || !std::isfinite(tgt[2 * t + 1]) || !(tgt[2 * t + 1] > 0.0))
      return fail(c, LSMS_ERR_ARG, "targets must lie in the top layer (y > 0)");
  if (ntgt == 0) return LSMS_OK;
  const int ns = c->ns, P = c->P;
  if ((rc = ensure(c, c->ws_g, (size_t)2 * ns * P * sizeof(double2)))) return rc;
  if ((rc = ensure(c, c->ws_pq, (size_t)2 * ns * sizeof(double2)))) return rc;
  if ((rc = ensure(c, c->ws_aux, (size_t)(2 * ntgt + 2) * sizeof(double) + (size_t)ntgt * sizeof(double2)))) return rc;
  double* d_tgt = (double*)c->ws_aux.ptr;
  double* d_src = d_tgt + 2 * ntgt;
  double2* d_out = (double2*)(d_src + 2);
  cudaMemcpyAsync(d_tgt, tgt, (size_t)2 * ntgt * sizeof(double), cudaMemcpyHostToDevice, c->stream);
  cudaMemcpyAsync(d_src, &c->src_xy[2 * src_index], 2 * sizeof(double), cudaMemcpyHostToDevice, c->stream);
  const double2* pq = nullptr;
  if (c->n > 0) {
    double2* G = (double2*)c->ws_g.ptr;
    cudaMemsetAsync(G, 0, (size_t)2 * ns * P * sizeof(double2), c->stream);
    const double2* beta = (const double2*)c->sol.ptr + (size_t)src_index * c->n * P;
    launch_zgemm_rows(c->d_eagg, 2 * ns, c->n, beta, G, P, 1, c->stream);
    launch_node_stage(ns, P, 1, G, c->d_fagg, nullptr, nullptr, nullptr, (double2*)c->ws_pq.ptr,
                      nullptr, nullptr, c->stream);
    pq = (const double2*)c->ws_pq.ptr;
  }
  launch_field(ns, ntgt, d_tgt, c->xc, c->d_lam, c->d_g1, c->d_field, pq, d_src, c->k1, which, d_out,
               c->stream);
  if ((rc = check_cuda(c, "eval_field"))) return rc;
  return copy_out(c, out, d_out, ntgt);
}

// ---------------------------------------------------------------------------------------------
// getters
// ---------------------------------------------------------------------------------------------
extern "C" int lsms_get_contour(const lsms_ctx* c, double* nodes, double* weights) {
  if (!c) return LSMS_ERR_ARG;
  if (nodes) std::memcpy(nodes, c->nodes.lam.data(), c->ns * sizeof(cplx));
  if (weights) std::memcpy(weights, c->nodes.wt.data(), c->ns * sizeof(cplx));
  return LSMS_OK;
}
extern "C" int lsms_get_scattering(const lsms_ctx* c, double* s) {
  if (!c || !s) return LSMS_ERR_ARG;
  if (c->dense) {
    for (int q = 0; q < c->P; ++q) std::memcpy(s + 2 * q, &c->smat[(size_t)q * c->P + q], sizeof(cplx));
  } else {
    std::memcpy(s, c->S.data(), c->P * sizeof(cplx));
  }
  return LSMS_OK;
}
// Replace the diagonal scattering matrix (absorbing or perfectly conducting discs, Sec. 3.1) in
// place: the host copy and the device table [S_n; |H_n(k2 R)| S_n] read by the combine and the
// right-hand side; NULL restores the Mie diagonal of the context's kp.
extern "C" int lsms_set_scattering_diagonal(lsms_ctx* c, const double* s) {
  if (!c) return LSMS_ERR_ARG;
  const int P = c->P;
  std::vector<cplx> S(P);
  if (s) {
    std::memcpy(static_cast<void*>(S.data()), s, P * sizeof(cplx));
    for (const cplx& v : S)
      if (!std::isfinite(v.real()) || !std::isfinite(v.imag()))
        return fail(c, LSMS_ERR_ARG, "set_scattering_diagonal: non-finite entry");
  } else {
    S = mie_diagonal(c->p, c->k2, c->kp, c->R);
  }
  cudaStreamSynchronize(c->stream);
  if (c->side) cudaStreamSynchronize(c->side);
  batch_clear_graphs(c);
  std::vector<cplx> s_out(2 * P);
  for (int q = 0; q < P; ++q) {
    s_out[q] = S[q];
    s_out[P + q] = c->hscale[q] * S[q];
  }
  if (cudaMemcpy(c->d_scale_out, s_out.data(), s_out.size() * sizeof(cplx), cudaMemcpyHostToDevice) != cudaSuccess)
    return check_cuda(c, "set_scattering_diagonal");
  c->S = S;
  c->custom_diag = s != nullptr;
  for (lsms_ctx* k : c->kids) {
    const int rc = lsms_set_scattering_diagonal(k, s);
    if (rc) return fail(c, rc, std::string("set_scattering_diagonal: ") + k->err);
  }
  return LSMS_OK;
}

extern "C" int lsms_num_nodes(const lsms_ctx* c) { return c ? c->ns : LSMS_ERR_ARG; }
extern "C" int lsms_num_particles(const lsms_ctx* c) { return c ? c->n : LSMS_ERR_ARG; }

extern "C" int lsms_set_timing(lsms_ctx* c, int enable) {
  if (!c) return LSMS_ERR_ARG;
  if (enable && !c->ev[0]) {
    for (int i = 0; i < 3; ++i)
      if (cudaEventCreate(&c->ev[i]) != cudaSuccess) return check_cuda(c, "cudaEventCreate");
  }
  c->timing = enable ? 1 : 0;
  return LSMS_OK;
}

extern "C" int lsms_last_timing(lsms_ctx* c, double* ms_translate, double* ms_reflect,
                                int* launches) {
  if (!c) return LSMS_ERR_ARG;
  if (!c->timing) return fail(c, LSMS_ERR_STATE, "timing is off: call lsms_set_timing(ctx, 1)");
  float a = 0.f, b = 0.f;
  if (cudaEventSynchronize(c->ev[2]) != cudaSuccess) return check_cuda(c, "cudaEventSynchronize");
  cudaEventElapsedTime(&a, c->ev[0], c->ev[1]);
  cudaEventElapsedTime(&b, c->ev[1], c->ev[2]);
  if (ms_translate) *ms_translate = a;
  if (ms_reflect) *ms_reflect = b;
  if (launches) *launches = c->last_launches;
  return check_cuda(c, "lsms_last_timing");
}

extern "C" int lsms_build_contour(const lsms_contour* contour, double k1, double k2, double k3,
                                  double* nodes, double* weights) {
  if (!contour || !nodes || !weights) return fail(nullptr, LSMS_ERR_ARG, "NULL argument");
  std::vector<cplx> lam, wt;
  std::string err;
  const int rc = build_contour(*contour, {k1, k2, k3}, lam, wt, err);
  if (rc) return fail(nullptr, rc, err);
  std::memcpy(nodes, lam.data(), lam.size() * sizeof(cplx));
  std::memcpy(weights, wt.data(), wt.size() * sizeof(cplx));
  return LSMS_OK;
}

extern "C" int lsms_build_contour_stack(const lsms_contour* contour, int n_layers, const double* k,
                                        double* nodes, double* weights) {
  if (!contour || !k || !nodes || !weights || n_layers < 3)
    return fail(nullptr, LSMS_ERR_ARG, "need n_layers >= 3 and non-NULL arguments");
  for (int j = 0; j < n_layers; ++j)
    if (!std::isfinite(k[j]) || !(k[j] > 0.0)) return fail(nullptr, LSMS_ERR_ARG, "wavenumbers must be finite and > 0");
  std::vector<cplx> lam, wt;
  std::string err;
  const int rc = build_contour(*contour, std::vector<double>(k, k + n_layers), lam, wt, err);
  if (rc) return fail(nullptr, rc, err);
  std::memcpy(nodes, lam.data(), lam.size() * sizeof(cplx));
  std::memcpy(weights, wt.data(), wt.size() * sizeof(cplx));
  return LSMS_OK;
}

extern "C" int lsms_layer_response(int n_layers, const double* k, const double* thickness, int particle_layer,
                                   int n, const double* lam, double* out) {
  if (n_layers < 3 || !k || !thickness || particle_layer < 2 || particle_layer > n_layers - 1 || n < 0 ||
      (n > 0 && (!lam || !out)))
    return fail(nullptr, LSMS_ERR_ARG, "layer_response: need n_layers >= 3, 2 <= particle_layer <= n_layers - 1");
  lsms_ctx tmp;
  tmp.layer = particle_layer;
  for (int j = 0; j < n_layers; ++j) {
    const cplx kj(k[2 * j], k[2 * j + 1]);
    if (!std::isfinite(kj.real()) || !std::isfinite(kj.imag()) || !(kj.real() > 0.0) || !(kj.imag() >= 0.0))
      return fail(nullptr, LSMS_ERR_ARG, "layer_response: wavenumbers need Re k > 0, Im k >= 0");
    tmp.kc.push_back(kj);
    tmp.ks.push_back(kj.real());
  }
  for (int j = 0; j < n_layers - 2; ++j) {
    if (!std::isfinite(thickness[j]) || !(thickness[j] > 0.0))
      return fail(nullptr, LSMS_ERR_ARG, "layer_response: thicknesses must be finite and > 0");
    tmp.ds.push_back(thickness[j]);
  }
  std::vector<cplx> g;
  cplx r[4][3];
  for (int v = 0; v < n; ++v) {
    layer_response(&tmp, cplx(lam[2 * v], lam[2 * v + 1]), g, r);
    for (int u = 0; u < 4; ++u)
      for (int s = 0; s < 3; ++s) {
        out[2 * ((size_t)v * 12 + u * 3 + s)] = r[u][s].real();
        out[2 * ((size_t)v * 12 + u * 3 + s) + 1] = r[u][s].imag();
      }
  }
  return LSMS_OK;
}

extern "C" int lsms_scattering_diagonal(int p, double k2, double kp, double radius, double* s) {
  if (p < 0 || p > LSMS_MAX_P || !s || !(k2 > 0) || !(kp > 0) || !(radius > 0))
    return fail(nullptr, LSMS_ERR_ARG, "bad arguments");
  std::vector<cplx> S = mie_diagonal(p, k2, kp, radius);
  std::memcpy(s, S.data(), S.size() * sizeof(cplx));
  return LSMS_OK;
}

extern "C" int lsms_check_geometry(double d, double radius, int n, const double* xy) {
  if (!(d > 0) || !(radius > 0) || n < 0 || (n > 0 && !xy)) return fail(nullptr, LSMS_ERR_ARG, "bad arguments");
  lsms_ctx tmp;
  tmp.d = d;
  tmp.R = radius;
  std::string err;
  const int rc = validate_geometry(&tmp, n, xy, err);
  if (rc) return fail(nullptr, rc, err);
  return LSMS_OK;
}

extern "C" const char* lsms_last_error(const lsms_ctx* c) {
  return c ? c->err.c_str() : g_create_err.c_str();
}
