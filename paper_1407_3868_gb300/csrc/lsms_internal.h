// Internal declarations of liblsms: the context, host-side setup and kernel launchers.
#pragma once

#include <cuda_runtime.h>

#include <complex>
#include <string>
#include <vector>

#include "lsms.h"

using cplx = std::complex<double>;

#define LSMS_MAX_P 15          // P = 2p + 1 <= 31 fits one warp of lanes over orders
// internal apply flag (above the public LSMS_APPLY_* bits): the FP64 residual of the mixed
// refinement, which takes the box translation when its scope is LSMS_FMM_RESIDUAL
#define LSMS_APPLY_RESIDUAL_INTERNAL (1 << 12)
// child of a layout batch: the translation of this application was computed for every layout at
// once by the parent (alpha_given, ready at the event alpha_ready); skip it and add to it
#define LSMS_APPLY_TRANSLATION_GIVEN (1 << 13)

// ------------------------------------------------------------------------------------------
// Device buffer owned by a context (grown on demand, never shrunk).
// ------------------------------------------------------------------------------------------
struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
};

// Per-node constants of the contour, FP64 (Sec. 2 Eq. "sommerfeldsys", Sec. 5.1).
struct NodeTables {
  std::vector<cplx> lam, wt;        // nodes and weights
  std::vector<cplx> g1, g2, g3;     // gamma_i(lambda)
  std::vector<cplx> refl;           // [ns][4]: a11 a12 a21 a22 of sigma2 = a * (P, Q)
  std::vector<cplx> inc;            // [ns][2]: sigma2+ = t1 I, sigma2- = t2 I (particle free)
  std::vector<cplx> field;          // [ns][4]: sigma_1 per unit I, P, Q; w/(4 pi gamma1)
  std::vector<cplx> fagg;           // [2 ns][P]: c_n w-^n (rows < ns), c_n w+^n (rows >= ns)
  std::vector<cplx> udis;           // [2 ns][P]: w/(4 pi g2) i^m w-^m, ... w+^m
};

// Box-compressed translation (fmm.cu): tables of the current layout.
struct FmmState {
  double box_width = 0.0;           // > 0: translation through boxes of this width
  int order_req = 0;                // requested box order (0: k2 r_box + 32)
  bool ready = false;
  int scope = 0;                    // 0: every translation; 1: only the FP64 refinement residuals
  bool far = false;                 // at least three boxes: a far field exists
  int order = 0, S = 0, nb = 0, n1 = 0, n2 = 0, dmin = 2;   // dmin: smallest offset in the FFT
  int logA = 0, logB = 0, logn2 = 0;   // n1 = 2^(logA + logB) (four-step split), n2 = 2^logn2
  double x0 = 0.0;
  int* d_perm = nullptr;            // [n] discs sorted by box
  int* d_bstart = nullptr;          // [nb + 1]
  int* d_dbox = nullptr;            // [n] box of each disc
  int* d_sbox = nullptr;            // [n] box in sorted order
  double* d_scx = nullptr;          // [n] sorted centres (device frame)
  double* d_scy = nullptr;
  double2* d_tab = nullptr;         // [n][2S + 1] J_s(k r) e^{i s phi}
  double2* d_khat = nullptr;        // [n1][n2] transformed box kernel / (n1 n2)
  double2* d_grid = nullptr;        // [n1][2Q + 1] work array (spectrum along the boxes)
  double2* d_bq = nullptr;          // [nb][2Q + 1] box coefficients B_i(q)
  double2* d_acc = nullptr;         // [nb][2Q + 1] local expansions A_i(nu)
  double2* d_hd = nullptr;          // [2 (dmin - 2)][4Q + 1] kernels of the direct offsets
  double2* d_twn = nullptr;         // [n1] e^{-2 pi i u / n1}
  double2* d_tw2 = nullptr;         // [n2] e^{-2 pi i u / n2}
  int* d_cptr = nullptr;            // [n + 1] mixed near field: pairs in the same or adjacent box by
  int* d_csrc = nullptr;            //   target in box order, source disc of each pair
  float2* d_cseq = nullptr;         // [pairs][4p + 2] their Hankel sequences (FP64-built, stored FP32)
  float2* d_tab32 = nullptr;        // FP32 copies of the shift tables, the transformed kernel, the
  float2* d_khat32 = nullptr;       // work array, the box coefficients and expansions, the
  float2* d_grid32 = nullptr;       // direct-offset kernels and the twiddles (mixed-precision far
  float2* d_bq32 = nullptr;         // field)
  float2* d_acc32 = nullptr;
  float2* d_hd32 = nullptr;
  float2* d_twn32 = nullptr;
  float2* d_tw232 = nullptr;
  DevBuf ws;                        // FP32 copies and partial sums of the mixed near field
  long long near_pairs = 0;         // ordered pairs translated directly
  bool timed = false;               // the last translation recorded the events
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};   // far start, near start, near end (timing)
};

struct lsms_ctx {
  // medium and discretisation: layers ks[0] (top) .. ks[L-1] (bottom), interior thicknesses
  // ds[0..L-3]; the discs lie in layer `layer` (1-based, 2 <= layer <= L-1), whose top interface is
  // `depth` below y = 0.  k1 = ks[0], k2 = ks[layer-1] (the disc layer), k3 = ks[L-1], d = its
  // thickness.  Disc centres are kept in the disc layer's own frame (top interface at y = 0).
  std::vector<double> ks, ds;       // ks: real parts of kc (the contour's branch points)
  std::vector<cplx> kc;             // wavenumbers (Im k > 0: an absorbing layer)
  int layer = 2;
  double depth = 0.0;
  double k1 = 0, k2 = 0, k3 = 0, d = 0, kp = 0, R = 0;
  int p = 0, P = 0, precision = 0;
  lsms_contour contour{};
  int ns = 0;
  NodeTables nodes;
  std::vector<cplx> S;              // Mie diagonal, P (or the caller's, custom_diag)
  bool custom_diag = false;         // S set by lsms_set_scattering_diagonal
  // inclusions of another shape (Sec. 4.1): a dense prototype matrix S[l][n] and per-particle angles
  bool dense = false;
  std::vector<cplx> smat;           // [P][P]
  double2* d_smt = nullptr;         // [2][P][P] transposed ([n][l]): S, diag(|H_l(k2 R)|) S
  DevBuf theta_buf;                 // [N] rotation angles (valid when has_theta)
  bool has_theta = false;
  FmmState fmm;
  // side stream of the mixed operator: the reflected coupling runs beside the translation
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  std::vector<double> hscale;       // |H_n(k2 R)|, P

  // discs
  int n = -1;                       // -1: set_particles not called yet
  double xc = 0.0;                  // x shift applied on the device (layout midpoint)
  std::vector<double> cx, cy;       // centres as given

  // device copies of the constant tables
  double2* d_lam = nullptr;         // [ns]
  double2* d_g1 = nullptr;          // [ns]
  double2* d_g2 = nullptr;          // [ns]
  double2* d_refl = nullptr;        // [ns][4]
  double2* d_inc = nullptr;         // [ns][2]
  double2* d_field = nullptr;       // [ns][4]
  double2* d_fagg = nullptr;        // [2ns][P]
  double2* d_udis = nullptr;        // [2ns][P]
  double* d_scale_in = nullptr;     // [2][P]: 1 (unscaled), 1/|H_n| (scaled)
  double* d_hscale = nullptr;       // [P]: |H_n(k2 R)|
  double2* d_scale_out = nullptr;   // [2][P]: S_n, |H_n| S_n

  // per-layout device data
  double* d_cx = nullptr;           // centred x, [n]
  double* d_cy = nullptr;           // [n]
  double2* d_eagg = nullptr;        // [2ns][n]: exp(g2 y - i l x) rows, then exp(-g2 (y+d) - i l x)
  double2* d_edis = nullptr;        // [n][2ns]: exp(g2 y + i l x), then exp(-g2 (y+d) + i l x)
  // low-precision copies for the mixed path (split BF16 hi/lo planes, see mixed.cu)
  void* d_eagg_lp = nullptr;
  void* d_edis_lp = nullptr;
  void* d_lp_misc = nullptr;
  DevBuf ws_lp;
  void* tc = nullptr;               // tensor-core path state (contour_tc.cu)
  // near pairs (k2 rho < 25) of the mixed translation: CSR by target, FP64-accurate sequences
  int near_nnz = 0;
  double near_r2 = 0.0;             // squared distance threshold
  int* d_near_ptr = nullptr;        // [n + 1]
  int* d_near_idx = nullptr;        // [nnz]
  void* d_near_h = nullptr;         // float4 [nnz]: H_0, H_1 of each near pair (FP64-built)

  // workspaces
  DevBuf ws_x, ws_y, ws_xs, ws_alpha, ws_g, ws_v, ws_pq, ws_sig, ws_aux;
  DevBuf ws_rows;                   // the target rows of a row-range application (lsms_apply_rows_dev)
  DevBuf gm_v, gm_h, gm_small, gm_x, gm_r, gm_w, gm_b, gm_mask, gm_off;
  double* h_pinned = nullptr;       // small pinned host scratch for residual polling
  cudaEvent_t gm_ev[8] = {};        // events of the GMRES residual ring
  void* gm_ring = nullptr;          // host-mapped ring of per-system GMRES states
  void* gm_ring_dev = nullptr;      // its device address
  size_t gm_ring_bytes = 0;
  int use_graphs = 1;               // capture each GMRES step as a CUDA graph
  DevBuf gm_loop;                   // device state of the graph-resident GMRES loop (gmres.cu)
  bool refine_stagnated = false;    // the last mixed solve stopped refining on stagnation
  double split_mult = 1.0;          // source splits of the FP32 translation (autotuned)
  int f32_shape = 2;                // FP32 translation tile shape (autotuned): 0 = two lanes per target,
                                    // 16 targets per warp; 1 = four lanes per target, 8 per warp;
                                    // 2 = one sequence per unordered pair (both directions)
  int tc_min_rhs = 48;              // mixed translations of >= this many right-hand sides (p >= 6)
                                    // run on the tensor cores; 0 = never
  int tc_flush = 32;                // source discs summed per FP32 tensor-memory accumulation
  DevBuf ws_tcb;                    // BF16 coefficient images of the tensor-core translation

  // a batch of independent layouts (lsms_set_layouts): one child context per layout
  std::vector<lsms_ctx*> kids;
  std::vector<long long> kid_off;   // first disc of every layout, and the total at the end
  struct GraphEntry {
    const void* x;
    void* y;
    int flags;
    cudaGraphExec_t exec;
  };
  std::vector<GraphEntry> graphs;   // captured batched applications
  std::vector<cudaEvent_t> kid_ev;  // join events (one per layout) and a fork event at the end
  // the mixed all-pairs translation of every layout in one launch (mixed.cu, translate_mixed_batch)
  bool bt_ready = false;
  int bt_ncta = 0;                  // work items, largest layout first: (layout, target tile, source
                                    // split) of shape 0; (layout, CTA, blocks per CTA) of shape 2
  int bt_waves = 4;                 // the items cover the GPU about this many times (autotuned)
  int bt_shape = 2;                 // 0: two lanes per target (k_translate_f32_h2_batch); 2: one
                                    // sequence per unordered pair (k_translate_f32_sym_batch); autotuned
  void* d_bt_items = nullptr;       // int4 [bt_ncta]
  void* d_bt_lays = nullptr;        // longlong4 [layouts]: disc offset, discs, sources per split, part offset
  void* d_bt_cff = nullptr;         // float4 [total discs]: every layout's float-float centres
  int* d_bt_nptr = nullptr;         // near pairs of all layouts: CSR by disc [total + 1] (global indices)
  int* d_bt_nidx = nullptr;
  void* d_bt_ntab = nullptr;        // float4 [nnz]: H_0, H_1
  long long bt_part = 0;            // float2 partial sums of all layouts
  DevBuf ws_bt;                     // scaled coefficients (FP64, FP32), partial sums, translation
  cudaEvent_t bt_ev = nullptr;      // the batched translation is done
  double2* alpha_given = nullptr;   // child: its rows of the parent's batched translation
  cudaEvent_t alpha_ready = nullptr;

  cudaStream_t stream = nullptr;    // internal stream of the host-pointer entry points

  // optional timing of the operator's parts (CUDA events on the launching stream)
  int timing = 0;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  int last_launches = 0;            // kernels launched by the last operator application

  // solution of the last lsms_solve (device, unscaled beta), per source
  int n_src = 0;
  std::vector<double> src_xy;
  DevBuf sol;

  std::string err;
};

// ------------------------------------------------------------------------------------------
// Host setup (host_setup.cpp)
// ------------------------------------------------------------------------------------------
int build_contour(const lsms_contour& c, const std::vector<double>& ks, std::vector<cplx>& lam,
                  std::vector<cplx>& wt, std::string& err);
// Gamma1 panel breakpoints; band_hi > band_lo marks a guided-mode band; greedy: the length over
// distance rule even without a band
std::vector<double> contour_panel_breaks(int n_panels, const double* ks, int nk, double b,
                                         double t_max, double band_lo, double band_hi, bool greedy);
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w);
std::vector<cplx> mie_diagonal(int p, double k2, double kp, double R);
std::vector<double> hankel_scale(int p, double k2, double R);
cplx gamma_of(cplx lam, double k);
cplx gamma_of(cplx lam, cplx k);
void build_node_tables(lsms_ctx* c);
// the interface system of one node for unit I, P, Q (rows sigma_1, s_m^+, s_m^-, sigma_L)
void layer_response(const lsms_ctx* c, cplx lam, std::vector<cplx>& g, cplx r[4][3]);
int validate_geometry(const lsms_ctx* c, int n, const double* xy, std::string& err);

// ------------------------------------------------------------------------------------------
// Kernel launchers (kernels_f64.cu).  All arrays are device pointers; all launches are
// asynchronous on `st`.  Coefficient arrays are [nrhs][N][P] (complex as double2).
// ------------------------------------------------------------------------------------------
void launch_scale_in(const double2* x, const double* scale, double2* xs, int nrhs, int n, int P,
                     cudaStream_t st);
// target rows row0 .. row0 + nrows - 1 (nrows < 0: to the last disc); alpha: [nrhs][nrows][P]
void launch_translate_f64(const double* cx, const double* cy, int n, int p, double k,
                          const double2* xs, double2* alpha, int nrhs, cudaStream_t st, int row0 = 0,
                          int nrows = -1);
void launch_etables(const double* cx, const double* cy, int n, const double2* lam,
                    const double2* g2, int ns, double d, double2* eagg, double2* edis,
                    cudaStream_t st);
// C[r][m][n] += sum_k A[m][k] B[r][k][n];  C must be pre-zeroed (split-K uses atomics)
void launch_zgemm_rows(const double2* A, int M, int K, const double2* B, double2* C, int P,
                       int nrhs, cudaStream_t st);
// per node: P,Q from G (if G) else from pq_in; optional outputs pq_out, sig_out, V
void launch_node_stage(int ns, int P, int nrhs, const double2* G, const double2* fagg,
                       const double2* pq_in, const double2* refl, const double2* udis,
                       double2* pq_out, double2* sig_out, double2* V, cudaStream_t st);
// per node: sigma from given sigma arrays -> V (for lsms_disaggregate)
void launch_sigma_to_v(int ns, int P, int nrhs, const double2* sig, const double2* udis,
                       double2* V, cudaStream_t st);
// incident densities of line sources: sig [nsrc][2][ns]
void launch_incident_sigma(int ns, int nsrc, const double* src, double xc, const double2* lam,
                           const double2* g1, const double2* inc, double2* sig, cudaStream_t st);
// y = x - s_out * alpha   (or y = alpha if alpha_only)
// y = x - D(-theta_j) M D(theta_j) alpha per particle (x == nullptr: y = D(-theta) M D(theta) alpha);
// mt: [P][P] transposed, theta: [n] or nullptr (all zero); nrhs blocks of n particles.
void launch_scatter_dense(const double2* x, const double2* alpha, const double2* mt, const double* theta,
                          int nrhs, int n, int P, double2* y, cudaStream_t st);
void launch_combine(const double2* x, const double2* alpha, const double2* s_out, double2* y,
                    int nrhs, int n, int P, int alpha_only, cudaStream_t st);
// field in layer 1 at targets
void launch_field(int ns, int ntgt, const double* tgt, double xc, const double2* lam,
                  const double2* g1, const double2* fieldtab, const double2* pq, const double* src,
                  double k1, int which, double2* out, cudaStream_t st);
