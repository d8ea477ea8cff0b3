/*
 * lsms.h — C ABI of the GB300 layered-medium multi-particle scattering library (liblsms.so).
 *
 * Problem (Lai, Kobayashi, Greengard, "A fast solver for multi-particle scattering in a layered
 * medium"): 2-D TM scattering of the field of a line source in the top layer (y > 0, wavenumber
 * k1) of a three-layer medium by identical dielectric discs (radius R, wavenumber kp) placed in the
 * middle layer (-d < y < 0, k2) above the bottom half-space (y < -d, k3); Sec. 1, Sec. 5.
 *
 * Generalisations built on the same operator: any number of layers with the particles in any
 * interior one (lsms_create_stack), absorbing layers (lsms_create_stack_c), inclusions of any smooth
 * shape turned per particle (Sec. 4: lsms_inclusion_scattering_matrix, lsms_set_scattering_matrix,
 * lsms_set_orientations), perfectly conducting and absorbing particles
 * (lsms_pec_scattering_diagonal, lsms_scattering_diagonal_c, lsms_inclusion_scattering_matrix_c),
 * batches of layouts (lsms_set_layouts) and, for long layouts of many discs, the translation
 * through boxes (lsms_set_fmm).  The header is plain C99.
 *
 * Unknowns: the outgoing (Hankel) coefficients beta^j_n, n = -p..p, of every disc j
 * (Sec. 3.1 Eq. "out"; truncation Sec. 3.1 Remark).  P = 2p + 1.
 *
 * Conventions shared by every entry point
 *   - Every function returns an int status: LSMS_OK (0) or a negative lsms_status code.  Nothing
 *     throws across the ABI.  lsms_last_error() gives a message for the last failure.
 *   - Complex numbers are interleaved (re, im) float64 pairs: C99 double _Complex,
 *     std::complex<double> and torch.complex128 all share this layout.
 *   - Coefficient arrays are right-hand-side major, then disc, then order:
 *     element (r, j, n) of a [nrhs][N][P] array sits at complex index (r*N + j)*P + (n + p).
 *   - Host pointers are owned by the caller; the library copies inputs and writes outputs the
 *     caller allocated.  The context owns all device memory it allocates.  `*_dev` entry points
 *     take device pointers (e.g. torch tensors) plus a cudaStream_t passed as void*; they are
 *     asynchronous on that stream.  All other calls are synchronous on the host.
 *   - A context is not thread-safe: use one context per host thread.
 *   - Time dependence exp(-i w t): H_n = H_n^(1) is outgoing.
 */
#ifndef LSMS_H
#define LSMS_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lsms_ctx lsms_ctx;

typedef enum {
  LSMS_OK = 0,
  LSMS_ERR_ARG = -1,           /* invalid argument: non-finite or non-positive k, p < 0, ...   */
  LSMS_ERR_GEOMETRY = -2,      /* gap < 0.2 R between discs, or a disc not inside its layer    */
  LSMS_ERR_NOT_CONVERGED = -3, /* GMRES hit maxiter (the iterate is still returned)            */
  LSMS_ERR_NONFINITE = -4,     /* a NaN/Inf appeared in the iteration                          */
  LSMS_ERR_OOM = -5,           /* device allocation failed                                     */
  LSMS_ERR_CUDA = -6,          /* a CUDA runtime call failed                                   */
  LSMS_ERR_STATE = -7          /* call order: e.g. apply before set_particles                  */
} lsms_status;

typedef enum {
  LSMS_FP64 = 0,   /* every step in float64                                                    */
  LSMS_MIXED = 1   /* FP32 translation, split-BF16 tensor-core contour contractions, FP64 refinement */
} lsms_precision;

/* Discretised Sommerfeld contour (Sec. 5.1, Eq. "sommerseg"): Gamma3 = t + i b (t < 0),
 * Gamma2 = i s (s from b to -b), Gamma1 = t - i b (t > 0), truncated at |t| = t_max.
 * Gamma1 and Gamma3 each hold n1 = q*floor((n_nodes - q)/(2q)) Gauss-Legendre nodes in panels of
 * order q = panel_order, graded toward the branch points (every layer's Re k; breakpoints
 * k_i +- b*2^j, the deepest grading that fits, then the longest panel halved).  In a guided-mode
 * medium (an interior k above both half-spaces' k: poles of the layer response on the real axis
 * between them, a distance b below Gamma1) the panels are instead placed greedily, halving the one
 * with the largest length / (b + distance to the nearest branch point), a panel meeting the pole
 * band counting as distance 0.  panel_rule = 1 asks for that greedy placement in every medium: far
 * more accurate for layouts a few wavelengths wide at the same n_nodes (16 discs, p = 10, 1024
 * nodes: 4e-12 against 8e-7 of the converged contour integral), while the grading keeps GMRES
 * iteration counts low on layouts thousands of wavelengths wide (where b is small).  Gamma2 holds
 * the remaining n_nodes - 2*n1 nodes as one Gauss-Legendre rule.  Node order is Gamma3, Gamma2,
 * Gamma1.  Zero fields take defaults: b = 0.2, t_max = max k + 20 (Sec. 6), panel_order = 16,
 * panel_rule = 0 (graded, greedy in guided-mode media); panel_rule must be 0 or 1. */
typedef struct {
  int n_nodes;       /* N_S, required; must leave n1 >= panel_order                          */
  double b;          /* offset of Gamma1/Gamma3 from the real axis                            */
  double t_max;      /* truncation of Gamma1/Gamma3                                           */
  int panel_order;   /* Gauss-Legendre order of each Gamma1/Gamma3 panel                      */
  int panel_rule;    /* 0: graded (greedy in guided-mode media); 1: greedy in every medium     */
} lsms_contour;

/* Outcome of lsms_solve.  history (optional, caller-owned, history_cap doubles) receives the
 * relative residual estimate after every inner GMRES iteration. */
typedef struct {
  int iters;            /* GMRES iterations (summed over refinement steps)                       */
  int outer_iters;      /* refinement steps (1 for LSMS_FP64)                                     */
  double rel_res;       /* final GMRES residual estimate, scaled preconditioned system            */
  double rel_res_fp64;  /* ||rhs - A beta|| / ||rhs|| recomputed in FP64 at the end               */
  double* history;      /* in: buffer or NULL                                                     */
  int history_cap;      /* in: capacity of history                                               */
  int n_history;        /* out: entries written                                                   */
} lsms_solve_info;

/* Field selector of lsms_eval_field (all in the top layer, Sec. 5 Eq. "fullrep"). */
enum {
  LSMS_FIELD_TOTAL = 0,      /* u1 = G_{k1}(x, x0) + u1^s                                     */
  LSMS_FIELD_SCATTERED = 1,  /* u1^s = u1 - G (layer reflection and discs)                     */
  LSMS_FIELD_PARTICLE = 2    /* u1 - u1(no discs): the part due to the discs                   */
};

/* Flags of lsms_apply_ex / lsms_apply_dev. */
enum {
  LSMS_APPLY_SCALED = 1,        /* x, y in the scaled basis b_n = |H_n(k2 R)| beta_n           */
  LSMS_APPLY_MIXED = 2,         /* mixed-precision operator (FP32 translation, BF16x3 contour) */
  LSMS_APPLY_NO_TRANSLATION = 4,/* drop T (free-space Graf coupling)                           */
  LSMS_APPLY_NO_REFLECTION = 8, /* drop R (layer-reflected coupling)                           */
  LSMS_APPLY_ALPHA = 16         /* output alpha = (T + R) x instead of x - S alpha             */
};

/* lsms_create — medium, discs and discretisation (Sec. 1; Sec. 3.1 Eq. "linear"; Sec. 5.1).
 *   k1, k2, k3: real wavenumbers of the three layers (> 0, finite).  d: middle-layer thickness.
 *   kp: wavenumber inside the discs.  radius: disc radius R (0 < R < d/2).  p >= 0, p <= 15.
 *   contour: see lsms_contour (required).  precision: default precision of lsms_apply/lsms_solve.
 *   On success *out holds a new context (free with lsms_destroy).  Errors: LSMS_ERR_ARG. */
int lsms_create(double k1, double k2, double k3, double d, double kp, double radius, int p,
                const lsms_contour* contour, int precision, lsms_ctx** out);

/* lsms_create_stack — lsms_create for any number of layers (the generalisation named in Sec. 1;
 *   the interface conditions of Sec. 2 at every interface, Sec. 5.2 "sommerfeldsys" extended).
 *   k[n_layers]: wavenumbers top (layer 1, y > 0) to bottom (layer n_layers), > 0, finite.
 *   thickness[n_layers - 2]: thicknesses of the interior layers 2 .. n_layers - 1 (> 0); the
 *   interfaces are at y = 0, -thickness[0], -thickness[0] - thickness[1], ...
 *   particle_layer: the interior layer m (2 <= m <= n_layers - 1) holding the discs, radius < half
 *   its thickness.  Centres passed to lsms_set_particles are in the same global frame (layer 1 is
 *   y > 0); sources and field targets too.  lsms_aggregate / lsms_reflect / lsms_disaggregate
 *   densities refer to layer m (P+ at its top interface, Q- at its bottom one).  The contour is
 *   graded to every k_j.  lsms_create(k1, k2, k3, d, ...) is this call with n_layers = 3, m = 2.
 *   Errors: LSMS_ERR_ARG (*out = NULL). */
int lsms_create_stack(int n_layers, const double* k, const double* thickness, int particle_layer,
                      double kp, double radius, int p, const lsms_contour* contour, int precision,
                      lsms_ctx** out);

/* lsms_create_stack_c — lsms_create_stack with complex wavenumbers k[n_layers] (interleaved re, im):
 *   Im k > 0 makes a layer absorbing (a lossy substrate or film; gamma = -i sqrt(k^2 - lambda^2)
 *   keeps Re gamma >= 0 on the contour).  Re k > 0 and Im k >= 0 everywhere; layer 1 (sources,
 *   targets) and the particle layer must be lossless (Im k = 0).  The contour is graded to Re k.
 *   Errors as lsms_create_stack. */
int lsms_create_stack_c(int n_layers, const double* k, const double* thickness, int particle_layer,
                        double kp, double radius, int p, const lsms_contour* contour, int precision,
                        lsms_ctx** out);

/* lsms_set_particles — disc centres (Sec. 3.2; Sec. 5).  centres_xy: 2n doubles (x0,y0,x1,...).
 *   Every disc must lie strictly inside the middle layer, with gaps >= 0.2 R between discs
 *   (10% of the diameter: the well-separation assumption of Sec. 1); otherwise
 *   LSMS_ERR_GEOMETRY.  Builds the per-disc contour tables on the device. n may be 0. */
int lsms_set_particles(lsms_ctx* ctx, int n, const double* centres_xy);

/* lsms_apply — y = x - S (T + R) x: the preconditioned multiple-scattering operator
 *   (Sec. 3.2 "scattmatrix" and the remark after it; Sec. 5.4 Eq. "schur").  x, y: [nrhs][N][P]
 *   complex, host.  T: Graf translation (Lemma 3.1); R: layer-reflected coupling (Thm 5.2 ->
 *   Eq. "sommerfeldsys" -> Lemma 5.1).  Uses the context's precision.  x and y may alias. */
int lsms_apply(lsms_ctx* ctx, int nrhs, const double* x, double* y);

/* lsms_apply_ex — lsms_apply with LSMS_APPLY_* flags (host pointers). */
int lsms_apply_ex(lsms_ctx* ctx, int nrhs, const double* x, double* y, int flags);

/* lsms_apply_dev — lsms_apply_ex on device pointers, asynchronous on `stream` (cudaStream_t). */
int lsms_apply_dev(lsms_ctx* ctx, int nrhs, const double* x_dev, double* y_dev, int flags,
                   void* stream);

/* lsms_apply_rows_dev — the rows of lsms_apply_dev for the target discs row0 .. row1 - 1: the block
 *   of the operator one GPU owns when the discs are split among GPUs by rows (Sec. 3.2 Eq.
 *   "scattmatrix"; the paper names a parallel implementation as the next step, Sec. 7).
 *   x_dev: [nrhs][N][P] complex, every disc (the gathered coefficients); y_dev: [nrhs][row1 - row0][P]
 *   complex, written: y_l = x_l - S (T x + R x)_l.  The translation (Lemma 3.1) runs for the owned
 *   target rows against every source disc; the reflected coupling (Thm 5.2 -> Eq.
 *   "sommerfeldsys" -> Lemma 5.1) is formed from all of x and its rows taken, so the only exchange
 *   a split operator needs per application is the gathering of x.  Flags as lsms_apply_dev
 *   (mixed precision: FP32 translation of the rows, split-BF16 contour).  Not for layout batches,
 *   nor with the box translation in scope LSMS_FMM_ALL.  Asynchronous on `stream`.
 *   Errors: LSMS_ERR_ARG (rows outside 0 <= row0 <= row1 <= N), LSMS_ERR_STATE. */
int lsms_apply_rows_dev(lsms_ctx* ctx, int nrhs, int row0, int row1, const double* x_dev, double* y_dev,
                        int flags, void* stream);

/* lsms_translate — alpha^l = sum_{m != l} T^{lm} beta^m (Sec. 3.2 Lemma 3.1, Eq. "trans"), with
 *   T^{lm}[nu][n] = H_{n-nu}(k2 rho) exp(i (n - nu) phi), rho = |x_l - x_m|, phi = arg(x_l - x_m).
 *   beta, alpha: [nrhs][N][P] complex, host.  precision: LSMS_FP64 or LSMS_MIXED. */
int lsms_translate(lsms_ctx* ctx, int nrhs, const double* beta, double* alpha, int precision);

/* lsms_aggregate — multipole-to-Sommerfeld (Sec. 5.3 Theorem 5.2, Eq. "invfft"):
 *   P+(nu) = sum_j sum_n beta^j_n c_n w-(nu)^n exp(gamma2 y_j - i lambda x_j),
 *   Q-(nu) = sum_j sum_n beta^j_n c_n w+(nu)^n exp(-gamma2 (y_j + d) - i lambda x_j),
 *   c_n = 4 (-i)^{n+1}, w-+ = (lambda -+ gamma2)/k2.  beta: [nrhs][N][P]; p_plus, q_minus:
 *   [nrhs][N_S] complex, host. */
int lsms_aggregate(lsms_ctx* ctx, int nrhs, const double* beta, double* p_plus, double* q_minus,
                   int precision);

/* lsms_reflect — per-node layer response (Sec. 2 Eq. "sommerfeldsys" with the discs' terms on
 *   the right): sigma2+ = R_t (P + R_b e Q)/D, sigma2- = R_b (Q + R_t e P)/D, D = 1 - R_t R_b e^2,
 *   R_t = (g2-g1)/(g2+g1), R_b = (g2-g3)/(g2+g3), e = exp(-g2 d).  Arrays [nrhs][N_S], host. */
int lsms_reflect(lsms_ctx* ctx, int nrhs, const double* p_plus, const double* q_minus,
                 double* sigma_plus, double* sigma_minus);

/* lsms_disaggregate — Sommerfeld-to-local by Jacobi-Anger (Sec. 5.2.1 Lemma 5.1, Eq. "JA2"):
 *   alpha^i_m = (1/4pi) sum_nu (w_nu/gamma2) i^m [sigma2+ w-^m exp(gamma2 y_i + i lambda x_i)
 *               + sigma2- w+^m exp(-gamma2 (y_i + d) + i lambda x_i)].
 *   sigma_*: [nrhs][N_S]; alpha: [nrhs][N][P], host. */
int lsms_disaggregate(lsms_ctx* ctx, int nrhs, const double* sigma_plus, const double* sigma_minus,
                      double* alpha, int precision);

/* lsms_incident — local expansion a_inc on every disc of the particle-free layered field of line
 *   sources src_xy (2 n_src doubles, y > 0): Eq. "sommerfeldsys" with the incident right-hand
 *   side, then Lemma 5.1.  a_inc: [n_src][N][P], host.  The right-hand side of the disc system is
 *   S a_inc (Sec. 5.4). */
int lsms_incident(lsms_ctx* ctx, int n_src, const double* src_xy, double* a_inc);

/* lsms_get_contour — the contour nodes lambda_nu and weights w_nu (d lambda included), N_S complex
 *   each, host.  lsms_get_scattering — the disc scattering matrix diagonal S_n (P complex). */
int lsms_get_contour(const lsms_ctx* ctx, double* nodes, double* weights);
int lsms_get_scattering(const lsms_ctx* ctx, double* s_diag);
int lsms_num_nodes(const lsms_ctx* ctx);
int lsms_num_particles(const lsms_ctx* ctx);

/* lsms_solve — beta for each source from (I - S(T + R)) beta = S a_inc (Sec. 3.2 GMRES,
 *   Sec. 5.4 Eq. "schur").  GMRES runs on the device on the scaled system (b = |H_n(k2R)| beta):
 *   x0 = 0 (or x0 if given, unscaled [n_src][N][P]), stop when the residual estimate divided by
 *   ||rhs|| <= tol or after maxiter iterations, 0 < maxiter <= 4096 (then LSMS_ERR_NOT_CONVERGED
 *   with the iterate in beta_out).  GMRES is not restarted: its basis holds maxiter + 1 vectors
 *   of N P complex numbers in device memory.  LSMS_MIXED: inner GMRES on the mixed operator inside an FP64 refinement loop.
 *   beta_out: [n_src][N][P] (may be NULL).  The solution is kept in the context for
 *   lsms_eval_field.  Several sources are solved together: one batched GMRES per source in
 *   lockstep, each step one multi-right-hand-side application of the operator.  info may be NULL;
 *   it reports the most iterations any source needed, the worst residuals and, for one source,
 *   the residual history. */
int lsms_solve(lsms_ctx* ctx, int n_src, const double* src_xy, double tol, int maxiter,
               const double* x0, double* beta_out, lsms_solve_info* info);

/* lsms_eval_field — field in the top layer at n_tgt points (2 n_tgt doubles, y > 0) for source
 *   src_index of the last lsms_solve (Sec. 2 Eq. "layer1", Sec. 5 Eq. "fullrep"):
 *   u1^s(x) = (1/4pi) sum_nu w_nu sigma1(nu) exp(-gamma1 y + i lambda x)/gamma1,
 *   sigma1 = R11 I + tau21 (P+ + e sigma2-).  which: LSMS_FIELD_*.  out: n_tgt complex, host. */
int lsms_eval_field(lsms_ctx* ctx, int src_index, int n_tgt, const double* tgt_xy, int which,
                    double* out);

/* lsms_set_layouts — a batch of independent layouts (a design sweep over particle
 *   configurations; Sec. 1: the solver serves "a sequence of configurations as part of a design or
 *   optimization process").  counts[l] discs for layout l; centres_xy holds every layout's centres
 *   one after the other (2 sum counts doubles), each checked as in lsms_set_particles.  After this
 *   call the context is a batch: coefficient arrays are the layouts' [N_l][P] arrays one after the
 *   other (one right-hand side per layout); lsms_apply / lsms_apply_dev apply every layout's
 *   operator, as one CUDA graph launch after the first call with the same buffers and flags;
 *   lsms_solve takes one source, or one per layout, and solves every layout (concurrently);
 *   lsms_eval_field's src_index selects the layout.  The per-step entry points (lsms_translate,
 *   ...) return LSMS_ERR_ARG on a batch.  lsms_set_particles turns the batch back into one layout.
 * lsms_num_layouts — layouts of the context (1 unless it is a batch). */
int lsms_set_layouts(lsms_ctx* ctx, int n_layouts, const int* counts, const double* centres_xy);
int lsms_num_layouts(const lsms_ctx* ctx);

/* lsms_autotune — time the one-right-hand-side FP32 translation on the current layout (or on the
 *   largest layout of every power-of-two size bucket of a batch, applied to the whole bucket) in its
 *   three tile shapes (0: two lanes per target disc, 64 targets per CTA; 1: four lanes per target,
 *   32 per CTA, twice the CTAs for small layouts; 2: one Hankel sequence per unordered disc pair,
 *   contracted into both discs' outputs, h_s(m <- l) = (-1)^s h_s(l <- m) (Sec. 3.2 Lemma 3.1),
 *   FP32 atomic sums; the default) under five split multipliers (0.5 .. 3: the source splits of
 *   shapes 0 and 1, the length of shape 2's block runs), and keep the fastest pair; *split_mult
 *   (may be NULL) receives the (last bucket's) factor.  For a batch it then times the one-launch
 *   translation of all layouts (used by the batched mixed application) in its two kernels (one
 *   sequence per unordered pair, the default; two lanes per target) with the work items covering
 *   the GPU 1, 2, 4 or 8 times, and keeps the fastest.
 *   No counterpart in the paper: a tuning step of this implementation.
 * lsms_get_translation_tuning / lsms_set_translation_tuning — the (shape, split multiplier) of
 *   layout `layout` (0 or -1 for a single layout; for a batch its layout index, -1 in the setter:
 *   every layout), e.g. to store the tuning and apply it again without timing.  shape 0, 1 or 2,
 *   0 < split_mult <= 64.  A layout batch's one-launch translation keeps its own kernel choice
 *   (lsms_autotune).  Errors: LSMS_ERR_ARG. */
int lsms_autotune(lsms_ctx* ctx, double* split_mult);
int lsms_get_translation_tuning(const lsms_ctx* ctx, int layout, int* shape, double* split_mult);
int lsms_set_translation_tuning(lsms_ctx* ctx, int layout, int shape, double split_mult);
/* lsms_get_batch_translation — for a layout batch, the one-launch translation of all layouts: how
 *   many times its work items (layout, CTA of two warps over runs of 16 x 16 disc blocks; or layout,
 *   tile of 64 target discs, source split) cover the GPU (4 until lsms_autotune picks) and their
 *   number; (0, 0) for a single layout or when the batch has none.
 *   NULL outputs are skipped.  Errors: LSMS_ERR_ARG (NULL ctx). */
int lsms_get_batch_translation(const lsms_ctx* ctx, int* waves, int* work_items);

/* lsms_set_tc_translation — mixed-precision translations of at least min_rhs right-hand sides at
 *   once (a block of sources, Sec. 3.2 Lemma 3.1 applied to every column) run on the tensor cores:
 *   per disc pair the (P x P) Toeplitz block times the (P x R) coefficient block as split-BF16
 *   tcgen05 MMAs accumulated in FP32 in tensor memory, drained into the FP64 result every `flush`
 *   source discs (fewer discs per FP32 accumulation: closer to the FP32 CUDA-core path's accuracy,
 *   more drains).  min_rhs = 0: never (the default is 48); flush = 0 keeps the current value (the
 *   default is 32).  Orders p < 6 always use the CUDA-core path.  Applies to the layouts of a batch
 *   too.  LSMS_ERR_ARG for negative arguments.  No counterpart in the paper. */
int lsms_set_tc_translation(lsms_ctx* ctx, int min_rhs, int flush);

/* lsms_set_timing — enable (1) or disable (0) CUDA-event timing of the operator's parts.  While
 *   enabled, every operator application records events on its stream around the translation
 *   (Lemma 3.1) and around the reflected coupling (Thm 5.2 -> Eq. "sommerfeldsys" -> Lemma 5.1).
 * lsms_last_timing — waits for the last application's events and returns the two durations in
 *   milliseconds and the number of kernels that application launched (any pointer may be NULL).
 *   LSMS_ERR_STATE when timing is off. */
int lsms_set_timing(lsms_ctx* ctx, int enable);
int lsms_last_timing(lsms_ctx* ctx, double* ms_translate, double* ms_reflect, int* launches);

/* lsms_translate_mixed_noalloc — the FP32 translation of lsms_translate(..., LSMS_MIXED) for
 *   callers that cannot allocate device memory: code that must live inside a memory budget owned
 *   by someone else (a framework's pooled allocator, a pre-sized arena) or a latency-critical loop
 *   where cudaMalloc/cudaFree, which may synchronise the device, are not allowed.  It needs no
 *   context and calls no allocating routine; its scratch is a fixed 16 MiB device array inside
 *   the library, which every GPU that loads the library keeps until the process exits.  The paper
 *   has no counterpart: it is a packaging of Lemma 3.1's operator, not a step of the method.
 *   n discs, order p (0..15), middle-layer wavenumber k2 > 0, nrhs coefficient vectors.
 *   centres_xy: device, 2n doubles; beta: device [nrhs][n][P] complex; alpha: device
 *   [nrhs][n][P] complex, written.  Asynchronous on `stream` (a cudaStream_t).  Sizes with
 *   16 n + 16 nrhs n (2p+1) bytes above 16 MiB (n above about 35000 at p = 14, nrhs = 1) are
 *   rejected with LSMS_ERR_ARG.  The first call on each device looks up the scratch array's
 *   device address (cudaGetSymbolAddress); make that first call before any stream capture.
 *   Every call shares the one scratch array, which keeps the last call's contents, so calls
 *   that overlap on the GPU (different streams, or different host threads) race: serialise them.
 *   Errors are reported by lsms_last_error(NULL). */
int lsms_translate_mixed_noalloc(int n, int p, double k2, int nrhs, const double* centres_xy,
                                 const double* beta, double* alpha, void* stream);

/* Inclusions of any smooth shape (Sec. 4; Sec. 4.1 "The scattering matrix").
 *
 * lsms_set_scattering_matrix — replace the disc's Mie diagonal by a dense prototype matrix:
 *   s: [P][P] complex (row l = outgoing order, column n = incoming order, orders -p..p), the
 *   outgoing coefficients beta_l of the prototype for the incoming wave J_n(k2 r) e^{i n theta}
 *   (e.g. from lsms_inclusion_scattering_matrix).  Every particle j then scatters with
 *   S_j[l][n] = e^{-i l theta_j} S[l][n] e^{i n theta_j} (theta_j from lsms_set_orientations, else 0)
 *   in lsms_apply*, lsms_solve and the batched forms.  The radius given at creation is the
 *   enclosing disc's: each inclusion must lie inside it, and the geometry rules of
 *   lsms_set_particles apply to the enclosing discs.  s = NULL restores the Mie diagonal.
 *   Copied; may be called before or after lsms_set_particles / lsms_set_layouts.
 *   Errors: LSMS_ERR_ARG (non-finite entry), LSMS_ERR_OOM.
 * lsms_set_orientations — rotation angles theta_j (radians, counterclockwise) of the n particles
 *   (n = lsms_num_particles; for a batch of layouts, all layouts' particles in order).  NULL: all
 *   zero.  lsms_set_particles / lsms_set_layouts reset them to zero.  Errors: LSMS_ERR_ARG (n or a
 *   non-finite angle), LSMS_ERR_STATE (no particles yet).
 * lsms_get_scattering_matrix — the prototype matrix in use ([P][P] complex; the Mie diagonal as a
 *   diagonal matrix unless one was set).  lsms_get_scattering returns its diagonal. */
int lsms_set_scattering_matrix(lsms_ctx* ctx, const double* s);
int lsms_set_orientations(lsms_ctx* ctx, int n, const double* theta);
int lsms_get_scattering_matrix(const lsms_ctx* ctx, double* s);

/* lsms_inclusion_scattering_matrix — host only, no context.  The scattering matrix of a homogeneous
 *   inclusion (wavenumber kp) in the layer of wavenumber k2 (Sec. 4): Muller's second-kind system
 *   (Eqs. "intg1", "intg2") for the unknowns mu, sigma of u^s = S^{k2} sigma + D^{k2} mu outside,
 *   u = S^{kp} sigma + D^{kp} mu inside, solved by Nystrom discretisation with Kress's product rule
 *   for the logarithmic singularities of the difference kernels (spectrally accurate for smooth
 *   boundaries; the paper uses Alpert's hybrid Gauss-trapezoidal rule) for the 2p+1 incoming waves
 *   J_n(k2 r) e^{i n theta}; beta_l from Graf's theorem (Sec. 4.1).
 *   curve: [n_pts][6] doubles x, y, x', y', x'', y'' at t_j = 2 pi j / n_pts of a smooth closed
 *   curve run counterclockwise, coordinates relative to the enclosing disc's centre; n_pts even,
 *   8 <= n_pts <= 4096 (about 256 gives 1e-13 for the shapes of Sec. 6); radius: the enclosing
 *   disc's.  s_out: [P][P] complex as for lsms_set_scattering_matrix.  O(n_pts^3) host work,
 *   spread over the host's threads (assembly by rows, blocked LU with a parallel trailing update:
 *   1.5 s at 1024 points on 8 cores).
 *   Errors: LSMS_ERR_ARG (arguments, a clockwise or degenerate curve, a singular system),
 *   LSMS_ERR_GEOMETRY (a point outside the enclosing disc or at its centre). */
int lsms_inclusion_scattering_matrix(int p, double k2, double kp, double radius, int n_pts,
                                     const double* curve, double* s_out);
/* lsms_inclusion_scattering_matrix_c — the same for an absorbing inclusion: complex interior
 *   wavenumber kp = kp_re + i kp_im (kp_re >= 0, kp_im >= 0; the layer k2 stays real) in the
 *   interior kernels of Muller's system, their J_0, J_1, Y_0, Y_1 at complex argument from
 *   Miller's backward recurrence and Neumann's expansions.  The product rule's log part grows like
 *   exp(Im kp r) along the curve, so accuracy falls off as about 1e-16 exp(2 Im kp R): kp_im * 2R
 *   must be <= 12 (1e-10 or better), and |kp| * 2R <= 1e4.  kp_im = 0 is
 *   lsms_inclusion_scattering_matrix.
 *   Errors: as above, LSMS_ERR_ARG also for a loss beyond that bound. */
int lsms_inclusion_scattering_matrix_c(int p, double k2, double kp_re, double kp_im, double radius, int n_pts,
                                       const double* curve, double* s_out);

/* lsms_pec_scattering_diagonal — host only.  S_n = -J_n(k2 R) / H_n(k2 R), n = -p..p, of a perfectly
 *   conducting disc (Sec. 3.1, remark after Definition 3.1: the total field vanishes on the
 *   boundary); pass diag(S) to lsms_set_scattering_matrix.  s_diag: 2p + 1 complex.
 *   Errors: LSMS_ERR_ARG. */
int lsms_pec_scattering_diagonal(int p, double k2, double radius, double* s_diag);

/* lsms_scattering_diagonal_c — host only.  S_n, n = -p..p, of an absorbing dielectric disc: the
 *   mode system of Sec. 3.1 Eq. "linear" with a complex interior wavenumber kp = kp_re + i kp_im
 *   (kp_re >= 0, kp_im >= 0: a lossy or conducting interior; the layer k2 stays real), solved
 *   through the logarithmic derivative J_n'(kp R) / J_n(kp R), which stays finite where J_n(kp R)
 *   overflows.  kp_im = 0 gives lsms_scattering_diagonal.  As kp_im grows the disc tends to the
 *   perfectly conducting one (lsms_pec_scattering_diagonal).  Pass diag(S) to
 *   lsms_set_scattering_matrix.  s_diag: 2p + 1 complex.  Errors: LSMS_ERR_ARG (also for
 *   |kp| R > 1e5). */
int lsms_scattering_diagonal_c(int p, double k2, double kp_re, double kp_im, double radius, double* s_diag);

/* lsms_set_scattering_diagonal — replace the discs' diagonal scattering matrix S_n, n = -p..p
 *   (s_diag: 2p + 1 complex; Sec. 3.1), e.g. by lsms_scattering_diagonal_c (absorbing discs) or
 *   lsms_pec_scattering_diagonal (perfectly conducting discs), keeping the diagonal combine (a
 *   dense matrix from lsms_set_scattering_matrix, while set, takes precedence).  NULL restores the
 *   Mie diagonal of the kp given at creation.  Applies to every layout of lsms_set_layouts, now and
 *   later.  Errors: LSMS_ERR_ARG (NULL ctx, a non-finite entry), LSMS_ERR_CUDA. */
int lsms_set_scattering_diagonal(lsms_ctx* ctx, const double* s_diag);

/* lsms_set_fmm — translate through boxes for long layouts of many discs (the FMM acceleration named
 *   in Sec. 3.2; the multipole shifts of Sec. 5.3).  Discs are grouped into boxes of width
 *   box_width along x (centres at the disc layer's mid-height); pairs in the same or adjacent boxes
 *   are translated directly; farther pairs through box expansions of order `order`: Graf shifts
 *   disc -> box (H -> H) and box -> disc (J -> J), and Lemma 3.1 between boxes two or more apart,
 *   evaluated for all boxes at once as a cyclic convolution over (box offset, order difference)
 *   with the library's own FFTs.  Used by lsms_apply*, lsms_translate and lsms_solve in both precisions (FP32 shifts,
 *   convolution and near field in mixed precision, FP64 otherwise), in place of the all-pairs and
 *   the tensor-core block translations.
 *   order = 0: ceil(k2 r_box) + 32 with r_box = hypot(box_width, d) / 2 (about 1e-12 relative
 *   in the scaled norm).  box_width <= 0 turns it off (all-pairs translation).  box_width must be
 *   at least the disc layer's thickness d (boxes two apart are then well separated); order in
 *   [p, 400].  The tables follow each lsms_set_particles / lsms_set_layouts (one set per layout).
 *   Errors: LSMS_ERR_ARG (also more than 131072 boxes), LSMS_ERR_OOM, LSMS_ERR_CUDA.
 * lsms_get_fmm — number of boxes and the order in use (0, 0 when off or before particles).
 * lsms_fmm_stats — ordered disc pairs translated directly (adjacent boxes), and, when timing is on
 *   (lsms_set_timing), the device milliseconds of the last box translation's far part (shifts,
 *   FFT convolution) and near part; waits for that translation.  NULL outputs are skipped. */
int lsms_set_fmm(lsms_ctx* ctx, double box_width, int order);
/* lsms_set_fmm_scope — where the box translation of lsms_set_fmm is used.  LSMS_FMM_ALL (the
 *   default): every translation.  LSMS_FMM_RESIDUAL: only the FP64 residuals r = rhs - A beta of the
 *   mixed-precision refinement (lsms_solve on an LSMS_MIXED context), the step that checks the
 *   solution; every other application (the inner mixed GMRES, lsms_apply*, lsms_translate) keeps
 *   the all-pairs translation.  The solve then refines against the box operator, whose translation
 *   differs from all pairs by the truncation of the box expansions (about 1e-12 relative at the
 *   default order), far below a refinement tolerance of 1e-8.  Applies to the layouts of a batch.
 *   Errors: LSMS_ERR_ARG. */
enum { LSMS_FMM_ALL = 0, LSMS_FMM_RESIDUAL = 1 };
int lsms_set_fmm_scope(lsms_ctx* ctx, int scope);
int lsms_get_fmm(const lsms_ctx* ctx, int* n_boxes, int* order);
int lsms_fmm_stats(lsms_ctx* ctx, long long* near_pairs, double* far_ms, double* near_ms);

/* Host-only helpers: no GPU needed, no context.
 * lsms_build_contour — the nodes and weights lsms_create would use for `contour` (see
 *   lsms_contour; Sec. 5.1 Eq. "sommerseg"); nodes, weights: contour->n_nodes complex each.
 * lsms_scattering_diagonal — S_n, n = -p..p, of a dielectric disc (Sec. 3.1 Eq. "linear").
 * lsms_check_geometry — LSMS_OK when n discs of radius R (centres_xy, 2n doubles) lie strictly
 *   inside the layer -d < y < 0 with gaps >= 0.2 R (10% of the diameter, the well-separation
 *   assumption of Sec. 1), else LSMS_ERR_GEOMETRY (or LSMS_ERR_ARG for non-finite input). */
int lsms_build_contour(const lsms_contour* contour, double k1, double k2, double k3, double* nodes,
                       double* weights);
/* lsms_build_contour_stack — the contour lsms_create_stack / lsms_create_stack_c would use: k holds
 *   the n_layers wavenumbers top to bottom (their real parts for an absorbing stack). */
int lsms_build_contour_stack(const lsms_contour* contour, int n_layers, const double* k, double* nodes,
                             double* weights);
/* lsms_layer_response — host only.  The interface conditions of Sec. 2 at every interface of a
 *   stack (complex k[n_layers] interleaved, thicknesses of layers 2 .. n_layers - 1, discs in
 *   particle_layer), solved at n complex nodes lam for a unit incident density I in layer 1, a unit
 *   upgoing particle density P at the top of the particle layer and a unit downgoing Q at its
 *   bottom.  out: [n][4][3] complex; row u = sigma_1, s_m^+, s_m^-, sigma_L; column s = I, P, Q (the
 *   per-node tables every context precomputes).  NaN entries where the system is singular. */
int lsms_layer_response(int n_layers, const double* k, const double* thickness, int particle_layer, int n,
                        const double* lam, double* out);
int lsms_scattering_diagonal(int p, double k2, double kp, double radius, double* s_diag);
int lsms_check_geometry(double d, double radius, int n, const double* centres_xy);

/* lsms_last_error — message of the last failure on ctx (or of lsms_create when ctx is NULL).
 *   The string is owned by the library and valid until the next call on ctx. */
const char* lsms_last_error(const lsms_ctx* ctx);

/* lsms_destroy — free the context and all its device memory.  NULL is ignored. */
void lsms_destroy(lsms_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* LSMS_H */
