// Operations shared by the translation units of liblsms (abi.cu, gmres.cu, mixed.cu).
#pragma once

#include <string>
#include <vector>

#include "lsms_internal.h"

int ctx_fail(lsms_ctx* c, int code, const std::string& msg);
// context for a stack of layers (kc top to bottom, Im k >= 0 and real in layer 1 and the particle
// layer; interior thicknesses ds; discs in `layer`)
int create_stack(const std::vector<cplx>& kc, const std::vector<double>& ds, int layer, double kp,
                 double radius, int p, const lsms_contour* contour, int precision, lsms_ctx** out);
int ensure(lsms_ctx* c, DevBuf& b, size_t bytes);
// Gaussian elimination with partial pivoting, a (n x n) x = b (n x nrhs), row-major; false if singular
bool solve_small(std::vector<cplx>& a, int n, std::vector<cplx>& b, int nrhs);
// box-compressed translation (fmm.cu)
int fmm_setup(lsms_ctx* c);
void fmm_free(lsms_ctx* c);
// mixed: the near field in FP32 (adjacent boxes) plus the FP32 near-pair kernel; else all FP64
int fmm_translate(lsms_ctx* c, int nrhs, const double2* xs, double2* alpha, bool mixed, cudaStream_t st);
// drop the captured batched applications (their kernels depend on the context's settings)
void batch_clear_graphs(lsms_ctx* c);
int check_cuda(lsms_ctx* c, const char* where);
int need_particles(lsms_ctx* c);
int validate_sources(lsms_ctx* c, int nsrc, const double* xy);

// y = x - s_out (T + R)(s_in x) on device buffers, flags LSMS_APPLY_*.
int apply_device(lsms_ctx* c, int nrhs, const double2* x, double2* y, int flags, cudaStream_t st);
// reflected coupling alpha += R xs, FP64
int reflection_f64(lsms_ctx* c, int nrhs, const double2* xs, double2* alpha, cudaStream_t st);
// a_inc for nsrc line sources (device source array), out [nsrc][N][P]
int incident_device(lsms_ctx* c, int nsrc, const double* d_src, double2* out, cudaStream_t st);

// mixed-precision contour contractions on the tensor cores (contour_tc.cu)
int tc_setup(lsms_ctx* c);            // BF16 planes of the layout's tables (after set_particles)
void tc_free(lsms_ctx* c);
int mixed_check(lsms_ctx* c);         // reads and clears the device error flag of the TC kernels
// the mixed reflected coupling split at its final add (run the stage on a side stream, add after a join)
int reflection_mixed_stage(lsms_ctx* c, int nrhs, const double2* xs, cudaStream_t st);
void reflection_mixed_add(lsms_ctx* c, int nrhs, double2* alpha, cudaStream_t st);
int* tc_err_flag(lsms_ctx* c);        // that flag (device), or null before tc_setup
int build_lowp_tables(lsms_ctx* c);
// alpha = T xs in FP32 arithmetic (sums of the per-split FP32 partials accumulated in FP64)
int translate_mixed(lsms_ctx* c, int nrhs, const double2* xs, double2* alpha, cudaStream_t st);
// the same for blocks of right-hand sides on the tensor cores, near pairs excluded (translate_tc.cu)
int translate_mixed_tc(lsms_ctx* c, int nrhs, const double2* xs, double2* alpha, cudaStream_t st);
// alpha += near-pair terms of T xs32 (FP64-accurate sequences, FP32 coefficients); for target rows
// row0 .. row0 + nrows - 1 (nrows < 0: to the last disc), alpha [nrhs][nrows][P]
void launch_translate_near(lsms_ctx* c, int nrhs, const float2* xs32, double2* alpha, cudaStream_t st,
                           int row0 = 0, int nrows = -1);
// alpha_rows = rows row0 .. row0 + nrows - 1 of T xs (xs: all discs), FP32 arithmetic, [nrhs][nrows][P]
int translate_mixed_rows(lsms_ctx* c, int nrhs, const double2* xs, double2* alpha_rows, int row0, int nrows,
                         cudaStream_t st);
int aggregate_mixed(lsms_ctx* c, int nrhs, const double2* xs, double2* G, cudaStream_t st);
int disaggregate_mixed(lsms_ctx* c, int nrhs, const double2* V, double2* alpha, cudaStream_t st);
int reflection_mixed(lsms_ctx* c, int nrhs, const double2* xs, double2* alpha, cudaStream_t st);

// batches of independent layouts (batch.cu)
bool is_batch(const lsms_ctx* c);
void batch_free(lsms_ctx* c);
int batch_apply(lsms_ctx* c, int nrhs, const double2* x, double2* y, int flags, cudaStream_t st);
int batch_solve(lsms_ctx* c, int nsrc, const double* src_xy, double tol, int maxiter, const double* x0,
                double* beta_out, lsms_solve_info* info);
int batch_eval_field(lsms_ctx* c, int layout, int ntgt, const double* tgt, int which, double* out);
int batch_mixed_check(lsms_ctx* c);

// The systems one GMRES run iterates in lockstep (gmres.cu): nb vectors packed in one slot of
// length `slot`, system b at elements off[b] .. off[b + 1] (device copy d_off).  The operator is
// applied to a whole slot with apply_nrhs right-hand sides: nb for the sources of one layout (equal
// lengths), 1 for the layouts of a batch (the batch operator covers every layout at once).
struct GmSys {
  int nb = 0;
  long long slot = 0, maxlen = 0;
  const long long* d_off = nullptr;
  int apply_nrhs = 0;
};
// Solve the scaled systems of s (rhs = D S a_inc; xs scaled unknowns, initial guesses if nonzero):
// FP64 GMRES, or FP64 refinement around mixed inner GMRES for a mixed context.  Per system: it
// iterations, rest residual estimate, rel64 FP64 relative residual; outer refinement steps.
int solve_systems(lsms_ctx* c, const GmSys& s, const double2* rhs, double2* xs, bool nonzero, double tol,
                  int maxiter, std::vector<int>& it, std::vector<double>& rest, std::vector<double>& rel64,
                  int* outer_out, double* hist, int hcap, int* nh, cudaStream_t st);

// small device helpers (gmres.cu)
void launch_diag_mul(const double2* x, const double2* s, double2* y, long long total, int P,
                     cudaStream_t st);
void launch_diag_scale(const double2* x, const double* s, double2* y, long long total, int P,
                       cudaStream_t st);

// The mixed all-pairs translation of every layout of a batch in one launch (mixed.cu): the tables
// (after lsms_set_layouts), and alpha of all layouts from their scaled coefficients xs.
int batch_translation_setup(lsms_ctx* c);
int batch_translation_items(lsms_ctx* c);   // the work items for c->bt_waves (setup and autotune)
void batch_translation_free(lsms_ctx* c);
int translate_mixed_batch(lsms_ctx* c, const double2* xs, double2* alpha, cudaStream_t st);
