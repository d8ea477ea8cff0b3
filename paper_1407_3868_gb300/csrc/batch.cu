// Batches of independent layouts (a design sweep over particle configurations, Sec. 1 and Sec. 6 of
// the paper: the solver is meant to run for "a sequence of configurations as part of a design or
// optimization process").
//
// lsms_set_layouts turns a context into a batch: one child context per layout, sharing the medium,
// the discretisation and the precision.  A batched operator application is one CUDA graph: a fork
// from the caller's stream into one branch per layout (each child's kernels on its own stream) and
// a join; the graph is captured on the first application with a given (x, y, flags) and replayed
// afterwards.  A batched solve runs the layouts' solves (each a graph-captured device GMRES) from a
// small host thread pool, largest layout first, so that the GPU works on many layouts at once.
// lsms_autotune picks the FP32 translation's tile shape and source-split factor by timing candidates,
// and for a batch how finely the one-launch translation of all layouts splits its sources.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <numeric>
#include <thread>
#include <vector>

#include "lsms_internal.h"
#include "lsms_ops.h"

bool is_batch(const lsms_ctx* c) { return c && !c->kids.empty(); }

void batch_clear_graphs(lsms_ctx* c) {
  for (auto& g : c->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  c->graphs.clear();
}

void batch_free(lsms_ctx* c) {
  batch_clear_graphs(c);
  batch_translation_free(c);
  for (cudaEvent_t e : c->kid_ev)
    if (e) cudaEventDestroy(e);
  c->kid_ev.clear();
  for (lsms_ctx* k : c->kids) lsms_destroy(k);
  c->kids.clear();
  c->kid_off.clear();
}

extern "C" int lsms_set_layouts(lsms_ctx* c, int n_layouts, const int* counts, const double* xy) {
  if (!c) return LSMS_ERR_ARG;
  if (n_layouts < 1 || !counts) return ctx_fail(c, LSMS_ERR_ARG, "set_layouts: need n_layouts >= 1 and counts");
  long long total = 0;
  for (int l = 0; l < n_layouts; ++l) {
    if (counts[l] < 0) return ctx_fail(c, LSMS_ERR_ARG, "set_layouts: negative disc count");
    total += counts[l];
  }
  if (total > 0 && !xy) return ctx_fail(c, LSMS_ERR_ARG, "set_layouts: centres are NULL");
  cudaStreamSynchronize(c->stream);
  batch_free(c);
  c->n = -1;
  c->n_src = 0;
  long long off = 0;
  for (int l = 0; l < n_layouts; ++l) {
    lsms_ctx* k = nullptr;
    int rc = create_stack(c->kc, c->ds, c->layer, c->kp, c->R, c->p, &c->contour, c->precision, &k);
    if (rc) {
      const std::string m = lsms_last_error(nullptr);
      batch_free(c);
      return ctx_fail(c, rc, "set_layouts: layout " + std::to_string(l) + ": " + m);
    }
    k->use_graphs = c->use_graphs;
    k->split_mult = c->split_mult;
    k->f32_shape = c->f32_shape;
    k->fmm.box_width = c->fmm.box_width;
    k->fmm.order_req = c->fmm.order_req;
    k->fmm.scope = c->fmm.scope;
    c->kids.push_back(k);
    if (c->custom_diag && (rc = lsms_set_scattering_diagonal(k, reinterpret_cast<const double*>(c->S.data())))) {
      const std::string m = k->err;
      batch_free(c);
      return ctx_fail(c, rc, "set_layouts: layout " + std::to_string(l) + ": " + m);
    }
    if (c->dense && (rc = lsms_set_scattering_matrix(k, reinterpret_cast<const double*>(c->smat.data())))) {
      const std::string m = k->err;
      batch_free(c);
      return ctx_fail(c, rc, "set_layouts: layout " + std::to_string(l) + ": " + m);
    }
    c->kid_off.push_back(off);
    rc = lsms_set_particles(k, counts[l], xy + 2 * off);
    if (rc) {
      const std::string m = k->err;
      batch_free(c);
      return ctx_fail(c, rc, "set_layouts: layout " + std::to_string(l) + ": " + m);
    }
    off += counts[l];
  }
  c->kid_off.push_back(off);
  c->kid_ev.assign(n_layouts + 1, nullptr);
  for (auto& e : c->kid_ev)
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      batch_free(c);
      return check_cuda(c, "set_layouts events");
    }
  c->n = (int)total;
  int rc = batch_translation_setup(c);
  if (rc) {
    const std::string m = c->err;
    batch_free(c);
    c->n = -1;
    return ctx_fail(c, rc, m);
  }
  return LSMS_OK;
}

extern "C" int lsms_num_layouts(const lsms_ctx* c) {
  if (!c) return LSMS_ERR_ARG;
  return is_batch(c) ? (int)c->kids.size() : 1;
}

// The layouts' mixed all-pairs translations run as one launch over all layouts (one right-hand
// side, every layout translating all pairs in FP32 for this application).
static bool use_batch_translation(const lsms_ctx* c, int flags) {
  if (!c->bt_ready || !(flags & LSMS_APPLY_MIXED) || (flags & LSMS_APPLY_NO_TRANSLATION)) return false;
  for (const lsms_ctx* k : c->kids)
    if (k->fmm.ready && (k->fmm.scope == 0 || (flags & LSMS_APPLY_RESIDUAL_INTERNAL))) return false;
  return true;
}

// Fork from st into every layout's stream, apply, join back into st.  With the batched translation
// the parent computes every layout's translation on st beside the layouts' reflected couplings; each
// layout waits for it before it adds its reflection and combines.
static int fork_join_apply(lsms_ctx* c, const double2* x, double2* y, int flags, cudaStream_t st) {
  const int nl = (int)c->kids.size();
  cudaEvent_t fork = c->kid_ev[nl];
  cudaEventRecord(fork, st);
  const bool bt = use_batch_translation(c, flags);
  double2* alpha_all = nullptr;
  if (bt) {
    const long long len = c->kid_off.back() * c->P;
    int rc;
    if ((rc = ensure(c, c->ws_xs, len * sizeof(double2)))) return rc;
    if ((rc = ensure(c, c->ws_alpha, len * sizeof(double2)))) return rc;
    double2* xs = (double2*)c->ws_xs.ptr;
    alpha_all = (double2*)c->ws_alpha.ptr;
    const int mode = (flags & LSMS_APPLY_SCALED) ? 1 : 0;
    launch_scale_in(x, c->d_scale_in + mode * c->P, xs, 1, (int)c->kid_off.back(), c->P, st);
    if ((rc = translate_mixed_batch(c, xs, alpha_all, st))) return rc;
    cudaEventRecord(c->bt_ev, st);
  }
  for (int l = 0; l < nl; ++l) {
    lsms_ctx* k = c->kids[l];
    const long long o = c->kid_off[l] * c->P;
    cudaStreamWaitEvent(k->stream, fork, 0);
    const int timing = k->timing;
    k->timing = 0;
    k->alpha_given = bt ? alpha_all + o : nullptr;
    k->alpha_ready = bt ? c->bt_ev : nullptr;
    const int rc = apply_device(k, 1, x + o, y + o, bt ? (flags | LSMS_APPLY_TRANSLATION_GIVEN) : flags,
                                k->stream);
    k->alpha_given = nullptr;
    k->alpha_ready = nullptr;
    k->timing = timing;
    if (rc) return ctx_fail(c, rc, "layout " + std::to_string(l) + ": " + k->err);
    cudaEventRecord(c->kid_ev[l], k->stream);
    cudaStreamWaitEvent(st, c->kid_ev[l], 0);
  }
  return LSMS_OK;
}

// y = x - S (T + R) x for every layout (x, y: [sum N_l][P] on the device), one graph launch.
int batch_apply(lsms_ctx* c, int nrhs, const double2* x, double2* y, int flags, cudaStream_t st) {
  if (nrhs != 1) return ctx_fail(c, LSMS_ERR_ARG, "a layout batch takes one coefficient vector per layout");
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) == cudaSuccess && cap == cudaStreamCaptureStatusActive)
    return fork_join_apply(c, x, y, flags, st);     // recorded into the graph being captured
  for (auto& g : c->graphs)
    if (g.x == x && g.y == y && g.flags == flags) {
      if (cudaGraphLaunch(g.exec, st) != cudaSuccess) return check_cuda(c, "batched apply graph");
      return LSMS_OK;
    }
  // first application with these buffers: run it directly (this also sizes every workspace), then
  // capture the same fork/join for the next calls
  int rc = fork_join_apply(c, x, y, flags, st);
  if (rc) return rc;
  if (!c->use_graphs || c->graphs.size() >= 16) return check_cuda(c, "batched apply");
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
    const int crc = fork_join_apply(c, x, y, flags, st);
    const cudaError_t e = cudaStreamEndCapture(st, &graph);
    if (crc == LSMS_OK && e == cudaSuccess && graph && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess)
      exec = nullptr;
    if (graph) cudaGraphDestroy(graph);
  }
  cudaGetLastError();
  c->err.clear();
  if (exec) c->graphs.push_back({x, y, flags, exec});
  return LSMS_OK;
}

int batch_mixed_check(lsms_ctx* c) {
  for (lsms_ctx* k : c->kids) {
    const int rc = mixed_check(k);
    if (rc) return ctx_fail(c, rc, k->err);
  }
  return LSMS_OK;
}

// Every layout's solve (source l, or the one source for all), concurrently from a thread pool
// (largest layouts first), each layout on its own stream with its own per-step CUDA graphs.  A
// lockstep variant (the layouts as the systems of one batched GMRES, one captured graph per Arnoldi
// step over all layouts) took 37.6 s instead of 31.5 s on the 128-layout sweep: every step applies
// the operator to layouts that have already converged, and the per-layout solves overlap better.
int batch_solve(lsms_ctx* c, int nsrc, const double* src_xy, double tol, int maxiter, const double* x0,
                double* beta_out, lsms_solve_info* info) {
  const int nl = (int)c->kids.size();
  if (nsrc != 1 && nsrc != nl)
    return ctx_fail(c, LSMS_ERR_ARG, "a layout batch takes one source, or one source per layout");
  if ((c->n_src = 0), validate_sources(c, nsrc, src_xy)) return LSMS_ERR_ARG;
  std::vector<int> order(nl), rc(nl, LSMS_OK);
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(), [&](int a, int b) { return c->kids[a]->n > c->kids[b]->n; });
  std::vector<lsms_solve_info> inf(nl);
  for (auto& i : inf) std::memset(&i, 0, sizeof(i));
  std::atomic<int> next{0};
  const int P = c->P;
  auto work = [&]() {
    for (;;) {
      const int t = next.fetch_add(1);
      if (t >= nl) break;
      const int l = order[t];
      lsms_ctx* k = c->kids[l];
      const double* s = nsrc == 1 ? src_xy : src_xy + 2 * l;
      const long long o = c->kid_off[l] * P * 2;
      rc[l] = lsms_solve(k, 1, s, tol, maxiter, x0 ? x0 + o : nullptr, beta_out ? beta_out + o : nullptr, &inf[l]);
    }
  };
  unsigned hw = std::thread::hardware_concurrency();
  const int nt = std::max(1, std::min(nl, (int)std::min(hw ? hw : 4u, 16u)));
  std::vector<std::thread> pool;
  for (int i = 1; i < nt; ++i) pool.emplace_back(work);
  work();
  for (auto& th : pool) th.join();
  int status = LSMS_OK;
  for (int l = 0; l < nl; ++l) {
    if (rc[l] == LSMS_OK) continue;
    if (status == LSMS_OK || (status == LSMS_ERR_NOT_CONVERGED && rc[l] != LSMS_ERR_NOT_CONVERGED)) {
      status = rc[l];
      ctx_fail(c, rc[l], "layout " + std::to_string(l) + ": " + c->kids[l]->err);
    }
  }
  if (info) {
    info->iters = info->outer_iters = 0;
    info->rel_res = info->rel_res_fp64 = 0.0;
    info->n_history = 0;
    for (int l = 0; l < nl; ++l) {
      info->iters = std::max(info->iters, inf[l].iters);
      info->outer_iters = std::max(info->outer_iters, inf[l].outer_iters);
      info->rel_res = std::max(info->rel_res, inf[l].rel_res);
      info->rel_res_fp64 = std::max(info->rel_res_fp64, inf[l].rel_res_fp64);
    }
  }
  if (status == LSMS_OK || status == LSMS_ERR_NOT_CONVERGED) c->n_src = nl;
  return status;
}

int batch_eval_field(lsms_ctx* c, int layout, int ntgt, const double* tgt, int which, double* out) {
  if (layout < 0 || layout >= (int)c->kids.size() || c->n_src == 0)
    return ctx_fail(c, LSMS_ERR_STATE, "no solution for that layout: call lsms_solve first");
  const int rc = lsms_eval_field(c->kids[layout], 0, ntgt, tgt, which, out);
  if (rc) return ctx_fail(c, rc, c->kids[layout]->err);
  return LSMS_OK;
}

// ---------------------------------------------------------------------------------------------
// autotuning of the FP32 translation's tile shape and source splits
// ---------------------------------------------------------------------------------------------
// Times the one-right-hand-side translation of c's layout in its three tile shapes (two lanes per
// target, 64 targets per CTA; four lanes per target, 32 per CTA; one sequence per unordered pair)
// under five split multipliers and keeps the fastest pair.
static int autotune_one(lsms_ctx* c, int* best_shape, double* best_mult) {
  *best_mult = c->split_mult;
  *best_shape = c->f32_shape;
  if (c->n <= 0) return LSMS_OK;
  const size_t len = (size_t)c->n * c->P;
  int rc;
  if ((rc = ensure(c, c->ws_xs, len * sizeof(double2)))) return rc;
  if ((rc = ensure(c, c->ws_alpha, len * sizeof(double2)))) return rc;
  cudaMemsetAsync(c->ws_xs.ptr, 0, len * sizeof(double2), c->stream);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const double cand[] = {0.5, 1.0, 1.5, 2.0, 3.0};
  float best = 1e30f;
  for (int shape = 0; shape < 3 && !rc; ++shape)
    for (double m : cand) {
      c->split_mult = m;
      c->f32_shape = shape;
      if ((rc = translate_mixed(c, 1, (const double2*)c->ws_xs.ptr, (double2*)c->ws_alpha.ptr, c->stream))) break;
      cudaEventRecord(e0, c->stream);
      for (int r = 0; r < 3; ++r)
        if ((rc = translate_mixed(c, 1, (const double2*)c->ws_xs.ptr, (double2*)c->ws_alpha.ptr, c->stream))) break;
      cudaEventRecord(e1, c->stream);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        *best_mult = m;
        *best_shape = shape;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->split_mult = *best_mult;
  c->f32_shape = *best_shape;
  if (rc) return rc;
  return check_cuda(c, "autotune");
}

extern "C" int lsms_autotune(lsms_ctx* c, double* split_mult) {
  if (!c) return LSMS_ERR_ARG;
  if (c->n < 0) return ctx_fail(c, LSMS_ERR_STATE, "call lsms_set_particles or lsms_set_layouts first");
  double m = c->split_mult;
  int shape = c->f32_shape;
  if (!is_batch(c)) {
    const int rc = autotune_one(c, &shape, &m);
    if (split_mult) *split_mult = m;
    return rc;
  }
  // one measurement per size bucket (powers of two), on the bucket's largest layout
  std::vector<int> bucket(c->kids.size());
  for (size_t l = 0; l < c->kids.size(); ++l)
    bucket[l] = c->kids[l]->n > 0 ? (int)std::ceil(std::log2((double)c->kids[l]->n)) : -1;
  std::vector<int> done;
  for (size_t l = 0; l < c->kids.size(); ++l) {
    const int b = bucket[l];
    if (b < 0 || std::find(done.begin(), done.end(), b) != done.end()) continue;
    size_t big = l;
    for (size_t j = l; j < c->kids.size(); ++j)
      if (bucket[j] == b && c->kids[j]->n > c->kids[big]->n) big = j;
    double mb = 1.0;
    int sb = 0;
    const int rc = autotune_one(c->kids[big], &sb, &mb);
    if (rc) return ctx_fail(c, rc, c->kids[big]->err);
    for (size_t j = 0; j < c->kids.size(); ++j)
      if (bucket[j] == b) {
        c->kids[j]->split_mult = mb;
        c->kids[j]->f32_shape = sb;
      }
    done.push_back(b);
    if (split_mult) *split_mult = mb;   // the last bucket's factor
  }
  // the one-launch translation of all layouts: how many times its work items cover the GPU
  if (c->bt_ready) {
    const size_t len = (size_t)c->kid_off.back() * c->P;
    int rc;
    if ((rc = ensure(c, c->ws_xs, len * sizeof(double2))) || (rc = ensure(c, c->ws_alpha, len * sizeof(double2))))
      return rc;
    cudaMemsetAsync(c->ws_xs.ptr, 0, len * sizeof(double2), c->stream);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    int best_w = c->bt_waves, best_s = c->bt_shape;
    for (int trial = 0; trial < 8 && !rc; ++trial) {
      const int sh = trial < 4 ? 2 : 0, w = 1 << (trial & 3);
      c->bt_shape = sh;
      c->bt_waves = w;
      if ((rc = batch_translation_items(c))) break;
      const double2* xs = (const double2*)c->ws_xs.ptr;
      double2* a = (double2*)c->ws_alpha.ptr;
      if ((rc = translate_mixed_batch(c, xs, a, c->stream))) break;
      cudaEventRecord(e0, c->stream);
      for (int r = 0; r < 3 && !rc; ++r) rc = translate_mixed_batch(c, xs, a, c->stream);
      cudaEventRecord(e1, c->stream);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rc) break;
      if (ms < best) {
        best = ms;
        best_w = w;
        best_s = sh;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->bt_waves = best_w;
    c->bt_shape = best_s;
    const int rc2 = batch_translation_items(c);
    if (rc) return rc;
    if (rc2) return rc2;
  }
  batch_clear_graphs(c);
  return LSMS_OK;
}

extern "C" int lsms_get_batch_translation(const lsms_ctx* c, int* waves, int* work_items) {
  if (!c) return LSMS_ERR_ARG;
  const bool on = is_batch(c) && c->bt_ready;
  if (waves) *waves = on ? c->bt_waves : 0;
  if (work_items) *work_items = on ? c->bt_ncta : 0;
  return LSMS_OK;
}

extern "C" int lsms_get_translation_tuning(const lsms_ctx* c, int layout, int* shape, double* split_mult) {
  if (!c) return LSMS_ERR_ARG;
  const lsms_ctx* k = c;
  if (is_batch(c)) {
    if (layout < 0 || layout >= (int)c->kids.size()) return LSMS_ERR_ARG;
    k = c->kids[layout];
  } else if (layout > 0) {
    return LSMS_ERR_ARG;
  }
  if (shape) *shape = k->f32_shape;
  if (split_mult) *split_mult = k->split_mult;
  return LSMS_OK;
}

extern "C" int lsms_set_translation_tuning(lsms_ctx* c, int layout, int shape, double split_mult) {
  if (!c) return LSMS_ERR_ARG;
  if (shape < 0 || shape > 2 || !std::isfinite(split_mult) || !(split_mult > 0.0) || split_mult > 64.0)
    return ctx_fail(c, LSMS_ERR_ARG, "set_translation_tuning: shape 0, 1 or 2 and 0 < split_mult <= 64");
  std::vector<lsms_ctx*> targets;
  if (!is_batch(c)) {
    if (layout > 0) return ctx_fail(c, LSMS_ERR_ARG, "set_translation_tuning: a single layout is layout 0 (or -1)");
    targets.push_back(c);
  } else if (layout < 0) {
    targets = c->kids;
  } else if (layout < (int)c->kids.size()) {
    targets.push_back(c->kids[layout]);
  } else {
    return ctx_fail(c, LSMS_ERR_ARG, "set_translation_tuning: layout out of range");
  }
  for (lsms_ctx* k : targets) {
    k->f32_shape = shape;
    k->split_mult = split_mult;
  }
  if (is_batch(c)) batch_clear_graphs(c);
  return LSMS_OK;
}
