// Internal declarations shared by the CUDA translation units of the KKT solver library.
// The public C ABI is include/kkt.h; nothing here is exported.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "kkt.h"

namespace kkt {

// Records a message for kkt_last_error() and returns `status`.
int set_error(int status, const std::string& msg);

#define KKT_CUDA_TRY(expr)                                                              \
  do {                                                                                  \
    cudaError_t e_ = (expr);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return ::kkt::set_error(KKT_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define KKT_TRY(expr)                 \
  do {                                \
    int s_ = (expr);                  \
    if (s_ < 0) return s_;            \
  } while (0)

// Tables of one orthonormal DST-I of length n-1 (n intervals), resident on the device.
struct DstPlan {
  int n = 0;          // intervals; the transform has n-1 points
  int logn = 0;       // log2(n) when n is a power of two, else -1 (direct transform)
  double* d_pre = nullptr;    // pairs c (sin(j pi / n) + 1/2), c (sin(j pi / n) - 1/2), j = 0..n/2,
                              // c = 1 / sqrt(2n) (pre-processing weights with the scale folded in)
  double2* d_tw = nullptr;    // exp(-2 pi i k / (n/2)), k = 0..n/2-1 (FFT twiddles)
  double2* d_post = nullptr;  // exp(-2 pi i k / n), k = 0..n/2 (real-FFT unpacking)
  double* d_sin = nullptr;    // direct transform: sqrt(2/n) sin(pi m / n), m = 0..2n-1
  int tile_lines = 0;         // lines per CTA tile (0: the size-based default; set by dst_autotune)
  bool lane_direct = false;   // one thread per line, direct sum (lines of at most 31 points;
                              // chosen by dst_autotune or kkt_set_dst_method)
};

// Time decomposition of Section 3 and the data of the Nicolaides coarse space (Eq 14).
struct TimeDecomp {
  int n_sub = 0;
  int max_len = 0;                    // max nodes of a subdomain (last - first + 1)
  std::vector<int> first, last;       // per subdomain: first/last time node (1-based)
  std::vector<int> ofirst, olast;     // per subdomain: owned node range (D_s)
  std::vector<int> owner;             // per node n (index n-1): owning subdomain (0-based)
  std::vector<double> phi;            // per node: the linear coarse function of its owner
  // per subdomain, 2x2 symmetric moment matrices (xx, xy, yy) of (1, phi) over owned nodes:
  // P0 = sum phi~ phi~^T, P1 = same over nodes >= 2, P2 = sum over owned neighbour pairs of
  // (phi~_n phi~_{n+1}^T + phi~_{n+1} phi~_n^T); the coarse block is (mu^2 P0 + P1 - mu P2)/h
  std::vector<double> P0, P1, P2;
};

// (G v)_s for one mode's coarse operator G = h S_0(mu) (Eq 14 and the operator after it): the
// 2 x 2 diagonal block mu^2 P0 + P1 - mu P2 from the subdomain's moments mom[9 s ..] and the
// couplings E_s = -mu a_s b_{s+1}^T with a_s = (1, phi(last owned node of s)),
// b_{s+1} = (1, phi(first owned node of s+1)). v holds the pairs (v_{2s}, v_{2s+1}).
template <typename TV>
__device__ __forceinline__ void coarse_op_apply_row(const double* __restrict__ mom, const double* __restrict__ phi,
                                                    const int* __restrict__ ofirst, const int* __restrict__ olast,
                                                    int n_sub, double mu, double mu2, const TV* v, int s,
                                                    double& e0, double& e1) {
  const double* M = mom + 9 * s;
  const double g00 = fma(mu2, M[0], M[3]) - mu * M[6];
  const double g01 = fma(mu2, M[1], M[4]) - mu * M[7];
  const double g11 = fma(mu2, M[2], M[5]) - mu * M[8];
  const double v0 = static_cast<double>(v[2 * s]), v1 = static_cast<double>(v[2 * s + 1]);
  e0 = g00 * v0 + g01 * v1;
  e1 = g01 * v0 + g11 * v1;
  if (s + 1 < n_sub) {   // E_s v_{s+1}
    const double a1 = __ldg(phi + __ldg(olast + s) - 1), b1 = __ldg(phi + __ldg(ofirst + s + 1) - 1);
    const double bv = static_cast<double>(v[2 * s + 2]) + b1 * static_cast<double>(v[2 * s + 3]);
    e0 -= mu * bv;
    e1 -= mu * a1 * bv;
  }
  if (s > 0) {           // E_{s-1}^T v_{s-1}
    const double a1 = __ldg(phi + __ldg(olast + s - 1) - 1), b1 = __ldg(phi + __ldg(ofirst + s) - 1);
    const double av = static_cast<double>(v[2 * s - 2]) + a1 * static_cast<double>(v[2 * s - 1]);
    e0 -= mu * av;
    e1 -= mu * b1 * av;
  }
}

// Device copy of TimeDecomp (one allocation).
struct DeviceDecomp {
  int n_sub = 0, max_len = 0, Nt = 0;
  int* first = nullptr;
  int* last = nullptr;
  int* ofirst = nullptr;
  int* olast = nullptr;
  int* owner = nullptr;
  double* phi = nullptr;
  double* moments = nullptr;   // [s][9]: P0 (3), P1 (3), P2 (3)
  float* phi_f = nullptr;      // phi in FP32 (the reduced-precision sweeps and restriction)
  void* base = nullptr;
};

// Tensor-core transform plan of the reduced-precision forms (square grids): the DST matrix Q
// and the slice stacks [Nt][P][P] the four transforms of an apply pass through.
struct TcPlan {
  int n = 0, P = 0, slices = 0, bf16 = 1, tile_n = 256;
  void* q = nullptr;       // Q, P x P, BF16 or FP32 (hi part)
  void* q_lo = nullptr;    // Q - Q_hi in the same type
  void* x0 = nullptr;      // packed input (hi part) / third transform output
  void* x0_lo = nullptr;   // lo part of the packed input
  void* x1 = nullptr;      // first transform output (hi part)
  void* x1_lo = nullptr;   // its lo part
  void* yin = nullptr;     // sweep output, input of the inverse transform (hi part)
  void* yin_lo = nullptr;  // its lo part
  float* rhat = nullptr;   // spectral coefficients [n][l][k], FP32
  int* err = nullptr;      // device flag: a pipeline wait timed out
  CUtensorMap map_q, map_q_lo, map_x0, map_x0_lo, map_x1, map_x1_lo, map_yin, map_yin_lo;
  size_t bytes = 0;
};

// FP64-accurate sine transform on the tensor cores (square grids, at most 255 points per line):
// every line and every column of the DST matrix is scaled by its own power of two and cut into
// kOzDigits balanced signed digits of kOzDigitBits bits, each digit plane exact in BF16;
// digit-plane products accumulate exactly in FP32 (tcgen05, TMEM) and are recombined in 64-bit
// integers.
constexpr int kOzDigits = 6;
constexpr int kOzDigitBits = 8;
struct OzPlan {
  int n = 0;            // intervals per direction (lines of n - 1 points)
  int M = 0;            // n - 1
  int P = 0;            // padded line length: 64, 128 or 256
  int N = 0;            // output columns per GEMM tile: 64, or 96 when P = 256
  int slices = 0;       // time slices (Nt)
  long long rows = 0;   // lines per pass: slices * M
  int rows_pad = 0;     // rows rounded up to the 128-row tile
  void* qs = nullptr;   // digit planes of Q: [kOzDigits][P][P] BF16, row c = output column, K contiguous
  int* qexp = nullptr;  // per column c: G_c with |Q[k][c]| < 2^G_c
  void* xs = nullptr;   // digit planes of the pass input: [kOzDigits][rows_pad][P] BF16
  int* xexp = nullptr;  // per row: E_r with |x| < 2^E_r
  double* tmp = nullptr;  // first pass output [slices][M][M] (transposed per slice)
  int* err = nullptr;   // device flag: a pipeline wait timed out
  CUtensorMap map_q, map_x;
  size_t bytes = 0;
};

struct Geometry {
  int nx, ny, Nt, n_sub, Mx, My;
  long long N, V;
  double T, nu, omega, Lx, Ly, dx, dy, dt, h;
  double a;        // diagonal shift of Jhat's block: 1 - jhat_sign * dt / sqrt(omega)
  double dtnu, cx, cy;   // dt nu, dt nu / dx^2, dt nu / dy^2
};


}  // namespace kkt

struct kkt_handle {
  kkt::Geometry g;
  kkt_options opt;
  int device = 0;
  int staging = KKT_STAGING_AUTO;   // how kkt_solve moves host vectors (enum kkt_staging)
  kkt::DstPlan dst_x, dst_y;
  kkt::TimeDecomp td;
  kkt::DeviceDecomp dd;
  double* d_lx = nullptr;      // lambda_x[k], k = 1..Mx (eigenvalues of the x second difference)
  double* d_ly = nullptr;
  double* d_lx_pad = nullptr;  // the same, zero-padded to the tensor-core transform size
  double* d_ly_pad = nullptr;
  kkt::TcPlan tc;              // reduced-precision transforms (allocated when such a precision is set)
  kkt::OzPlan oz;              // FP64 transforms on the tensor cores (kkt_set_dst_method TENSOR)
  bool dst_tensor = false;     // FP64 sine transforms by the tensor-core digit-plane GEMMs
  long long coarse_modes = 0;  // modes the coarse buffers are sized for
  // learned coarse correction
  kkt_mlp* mlp = nullptr;      // not owned
  int mlp_mode = 0;            // 0 learned with the guard, 1 no coarse on the learned modes, 2 network only
  int learn_k = 0;             // learned modes per direction
  double* learn_c = nullptr;   // [learn_k^2][2 n_sub] restricted right-hand sides
  double* learn_feat = nullptr;  // [learn_k^2][2]
  float* learn_x = nullptr;    // [learn_k^2][2 n_sub + 2] network input
  long long* learn_count = nullptr;  // device: kept, fallback
  // preconditioner workspace
  double* spec = nullptr;      // V doubles: spectral coefficients [n][l][k]
  double* spec2 = nullptr;     // V doubles
  double* coarse_c = nullptr;  // [n_sub][2][N] coarse coefficients
  double* coarse_w = nullptr;  // [n_sub][2][modes] eliminated coarse right-hand sides
  double* coarse_f = nullptr;  // [n_sub][3][N] block-Thomas factors D_s^{-1} (per configuration)
  double* coarse_f_pad = nullptr;  // the same over the padded modes of the mixed forms
  double* cr_factors = nullptr;    // cyclic-reduction factors, slot-major [slots(n_sub)][N] (FP64 path)
  size_t cr_factor_bytes = 0;
  double* vscratch = nullptr;  // sweep storage when a subdomain is too long for shared memory
  // Krylov workspace (allocated at the first solve)
  int kry_restart = 0;
  double* kV = nullptr;        // (restart+1) full vectors (3V each)
  double* kZw = nullptr;       // restart w-blocks (V each)
  double* kx = nullptr;        // staging for host x / f (3V each)
  double* kf = nullptr;
  double* ks_f = nullptr;      // spectral basis: sine-mode coefficients of f and x (3V each)
  double* ks_x = nullptr;
  double* red = nullptr;       // reduction partials
  double* red_out = nullptr;   // reduction results (device)
  double* h_red = nullptr;     // pinned host copy of reduction results
  double* dcoef = nullptr;     // device coefficient arrays for multi-axpy
  size_t bytes = 0;
};

namespace kkt {

// ---- instrumentation: counts every launch, times it with CUDA events when enabled -------
// flops / bytes: the launch's algorithmic work (what the method must compute and move), summed
// for the timed launches so that achieved rates can be read against a roofline.
void prof_begin(int cls, cudaStream_t st);
void prof_end(int cls, cudaStream_t st, double flops, double bytes);
struct ProfScope {
  int cls;
  cudaStream_t st;
  double flops, bytes;
  ProfScope(int c, cudaStream_t s, double f = 0.0, double b = 0.0) : cls(c), st(s), flops(f), bytes(b) {
    prof_begin(c, s);
  }
  ~ProfScope() { prof_end(cls, st, flops, bytes); }
};
// While a stream is captured into a CUDA graph, launches are tallied into a ProfCapture (not
// counted, not timed); every replay through prof_graph_launch then adds the tallied kernel
// launches to the counters and times the whole graph as one KKT_K_GRAPH launch.
struct ProfCapture {
  long long launches[KKT_K_COUNT] = {};
  double flops = 0.0, bytes = 0.0;
};
void prof_capture(ProfCapture* acc);   // nullptr ends the capture on this thread
int prof_graph_launch(cudaGraphExec_t g, const ProfCapture& acc, cudaStream_t st);

// ---- kernels launched from the C ABI (each defined in its own translation unit) ---------
int dst_plan_create(DstPlan& p, int n);
// Frees a handle's Krylov storage and host-buffer staging (reallocated by the next kkt_solve).
void release_krylov(kkt_handle* h);
// Times the candidate tile heights (8, 16, 32 lines) of the row and column passes on the
// handle's spectral buffers and keeps the fastest in dst_x / dst_y (at create).
int dst_autotune(kkt_handle* h);
int dst_set_method(kkt_handle* h, int method);
void dst_plan_destroy(DstPlan& p);
// orthonormal 2D DST-I of every slice: rows (along x) then columns (along y)
int dst2d(const kkt_handle* h, const double* in, double* out, cudaStream_t st);

// y = diag(ou, oz, ow) K (su u, sz z, sw w)
int launch_matvec(const kkt_handle* h, const double* u, double su, const double* z, double sz,
                  const double* w, double sw, double* y, cudaStream_t st, double ou = 1.0, double oz = 1.0,
                  double ow = 1.0);
// The matvec on sine-mode coefficients of all three blocks (same arguments as launch_matvec).
int launch_matvec_spectral(const kkt_handle* h, const double* u, double su, const double* z, double sz,
                  const double* w, double sw, double* y, cudaStream_t st, double ou = 1.0, double oz = 1.0,
                  double ow = 1.0);
int launch_build_rhs(const kkt_handle* h, const double* ut, const double* u0, double* f, cudaStream_t st);
int launch_scale(const double* x, double s, double* y, long long n, cudaStream_t st);
// yu = su xu and yz = sz xz in one launch (n elements each)
int launch_scale2(const double* xu, double su, double* yu, const double* xz, double sz, double* yz, long long n,
                  cudaStream_t st);
int launch_jhat_time(const kkt_handle* h, const double* in, double* out, int dir, double scale,
                     cudaStream_t st);

// Schur preconditioner in spectral space: in -> out, both [n][l][k] blocks (may alias)
int spectral_schur_precond(const kkt_handle* h, const double* rhat, double* yhat, double in_scale,
                           cudaStream_t st);
int spectral_coarse_only(const kkt_handle* h, const double* rhat, double* xhat, cudaStream_t st);
// learned coarse correction: y (network output, [learn_k^2][2 n_sub] FP32) -> cc of the learned modes
int spectral_learned_apply(const kkt_handle* h, bool padded, const float* y, cudaStream_t st);
// network pieces used by the preconditioner (kkt_mlp.cu)
int mlp_forward(kkt_mlp* m, const float* X, int B, int use_bf16, cudaStream_t st);
const float* mlp_output(const kkt_mlp* m);
int mlp_dims(const kkt_mlp* m, int* d_in, int* width, int* d_out);
int mlp_make_input(const double* c, const double* feat, long long S, int nc, float* X, cudaStream_t st);
const kkt_mlp_config& mlp_config(const kkt_mlp* m);
// per-mode block-Thomas factors of the coarse operator (depend on mu and the decomposition only)
// Computes (or frees) the cyclic reduction's factors for the handle's options: stored when the
// FP64 path's coarse solve is the cyclic reduction and they take at most 2 GB.
int spectral_cr_factor(kkt_handle* h);
int spectral_coarse_factor(const kkt_handle* h, bool padded, double* cf, cudaStream_t st);
// reduced-precision forms: FP32 spectral input (padded modes), output BF16 (bf16 != 0) or FP32
// (yhat_lo non-null: also the lo part, yhat + yhat_lo = the FP32 result)
int spectral_schur_precond_mixed(const kkt_handle* h, const float* rhat, double in_scale, void* yhat, void* yhat_lo,
                                 int bf16, cudaStream_t st);

// tensor-core transforms (kkt_tc_gemm.cu)
int tc_padded_size(int n);
int tc_plan_create(TcPlan& t, int n, int slices, int bf16);
void tc_plan_destroy(TcPlan& t);
// which_in: 0 = x0, 1 = x1, 2 = yin; out_mode: 0 BF16 / 1 FP32 padded slices, 2 FP64 valid x
// valid, 3 hi + lo pair (out, out_lo); split: the input and Q as hi + lo parts (3 products)
int tc_gemm(const TcPlan& t, int which_in, int out_mode, void* out, int valid, cudaStream_t st, bool split = false,
            void* out_lo = nullptr);
int tc_pack(const TcPlan& t, const double* in, int valid, cudaStream_t st);   // -> x0 (+ x0_lo)
int tc_check(const TcPlan& t, cudaStream_t st);
// FP64-accurate transforms on the tensor cores (kkt_tc_gemm.cu)
int oz_plan_create(OzPlan& o, int n, int slices);
void oz_plan_destroy(OzPlan& o);
int oz_dst2d(const OzPlan& o, const double* in, double* out, cudaStream_t st);   // both directions
int oz_check(const OzPlan& o, cudaStream_t st);   // reads and clears the timeout flag
long long oz_tiles(const OzPlan& o);               // output tiles of one GEMM pass
int tc_set_flag(const TcPlan& t);   // host-side write of the timeout flag (kkt_inject_tc_timeout)

// Krylov primitives (deterministic two-stage reductions; results in h->red_out on device)
int krylov_multidot(kkt_handle* h, const double* V, long long stride, int count, const double* w,
                    long long n, cudaStream_t st, double* out = nullptr);   // out (default red_out)[k] = <V_k, w>, [count] = <w,w>
int krylov_update_norm(kkt_handle* h, const double* V, long long stride, int count,
                       const double* coef_dev, double* w, long long n, cudaStream_t st);  // w -= sum c_k V_k; red_out[0] = <w,w>
int krylov_axpy_multi(const double* V, long long stride, int count, const double* coef_dev,
                      double* x, long long n, cudaStream_t st);  // x += sum c_k V_k
int krylov_norm2(kkt_handle* h, const double* x, long long n, cudaStream_t st);  // red_out[0]
// One modified Gram-Schmidt step over n elements: if Vk, w -= (dot[0] * s) Vk; then *out =
// <Vn, w> (Vn non-null) or <w, w> (Vn null), reduced deterministically.
int krylov_mgs_step(kkt_handle* h, const double* Vk, const double* dot, double s, const double* Vn, double* w,
                    long long n, double* out, cudaStream_t st);
// Basis vectors per block of the blocked MGS orthogonalisations (1: plain MGS or CGS2).
inline int orth_block(int orth) {
  return orth == KKT_ORTH_MGS2 ? 2 : orth == KKT_ORTH_MGS4 ? 4 : orth == KKT_ORTH_MGS8 ? 8 : 1;
}
// Blocked MGS step (block size bs = 2, 4 or 8): w -= sum_{a < na} (dot[a] s[a]) A_a with
// A_a = A + a stride, then out[0..nd) = <B_d, w> with B_d = Bv + d stride (nd > 0) or
// out[0] = <w, w> (nd = 0); na, nd in 0..bs.
int krylov_mgsb_step(kkt_handle* h, int bs, int na, const double* A, const double* dot, const double* s, int nd,
                     const double* Bv, long long stride, double* w, long long n, double* out, cudaStream_t st);
int krylov_partial_capacity();

// ---- batched forms: several instances per launch ---------------------------------------
// One tile launch of the DST line kernel (rows or columns of one instance).
struct DstLaunch {
  const double* in;
  double* out;
  int n, logn, M, ldt, tile_lines;
  int mode;                 // 0: lines are rows (along x), 1: lines are columns (along y)
  long long total_lines;    // rows mode: number of rows in the block
  int cols;                 // columns mode: columns per slice (the row length Mx)
  long long slice;          // columns mode: elements per slice
  int tiles_per_slice;      // columns mode
  const double* pre;
  const double2* tw;
  const double2* post;
  const double* sintab;
  int lane;                 // one thread per line (lines of at most 31 points), no tiles
  int fft_group;            // FFT path: lanes per line (32 / fft_group lines per warp)
  long long lines;          // lines of the launch (rows: total_lines; columns: slices x cols)
};

// Per-instance parameters of the spectral kernels (modes, decomposition, coarse buffers).
struct SpecParams {
  int Mx, Nt, n_sub;      // Mx: modes per spectral row (the padded size in the mixed forms)
  long long N;
  double a, dtnu, h, inv_h;
  const double* lx;
  const double* ly;
  const int* first;
  const int* last;
  const int* ofirst;
  const int* olast;
  const int* owner;
  const double* phi;
  const float* phi_f;
  const double* mom;
  const double* cf;    // coarse factors [s][3][N]: D_s^{-1} of the block-Thomas elimination
  int learn_k;         // modes k, l < learn_k also write their R_0 r to learn_c
  double* learn_c;
  int two_level;       // apply the coarse correction
  int multiplicative;  // subtract S-hat x_0 before the local solves
  int ras;             // local solves with R_s S-hat R_s^T (Eq 9) instead of RASQ's (Eq 13)
  int cyclic;          // coarse solve by cyclic reduction (else block Thomas)
  const double* crf;   // the cyclic reduction's stored factors (nullptr: eliminate in every solve)
  int cr_mpc;          // modes per CTA of the cyclic-reduction solve
};
SpecParams make_spec_params(const kkt_handle* h);

// One instance's share of a batched spectral phase: rhat -> yhat with the in-scale
// scale_base * scale_dev[scale_index] (the Krylov driver keeps 1 / eta per instance on the device).
struct SpecJob {
  SpecParams p;
  const double* rhat;
  double* yhat;
  double* cc;            // coarse coefficients [s][2][N]
  double* cy;            // eliminated coarse right-hand sides [s][2][N]
  double scale_base;
  int max_len;
  int scale_index;
};

// One instance's matvec: y = diag(du, dz, dw) K (su u, sz z, w) with su, sz = base * scale_dev[index].
struct MatvecJob {
  const double* u;
  const double* z;
  const double* w;
  double* y;
  int Mx, My, Nt;
  long long N, V;
  double uu, wc0, wcx, wcy, wn, zz, zw, uc0, ucx, ucy, up, wz;   // su-, sz-dependent terms at su = sz = 1
  int scale_index;
  // spectral basis: the stencil acts per sine mode as mu0 = 1 + dtnu (lx_k + ly_l); wc0, uc0 then
  // exclude the centre weight and wcx, wcy, ucx, ucy are unused
  int spectral;
  const double* lx;
  const double* ly;
  double dtnu;
};
// out = alpha * x + beta * y (elementwise; out may alias x or y)
int launch_axpby(double alpha, const double* x, double beta, const double* y, double* out, long long n,
                 cudaStream_t st);

// Device tables of one batched phase sequence (the launches of one captured graph).
struct DstJob {
  const kkt_handle* h;
  const double* in;
  double* out;
};

struct BatchSlot {
  int njobs = 0;
  // DST: [pass 0 fwd rows, 1 fwd cols, 2 inv rows, 3 inv cols] x dst_njobs (the instances whose
  // transforms run as line tiles; the others are in oz_jobs)
  int dst_njobs = 0;
  DstLaunch* dst = nullptr;
  long long* dst_prefix = nullptr;    // [4][njobs + 1]
  long long dst_total[4] = {0, 0, 0, 0};
  size_t dst_smem[4] = {0, 0, 0, 0};
  double dst_flops[4] = {0, 0, 0, 0}, dst_bytes[4] = {0, 0, 0, 0};
  SpecJob* spec = nullptr;
  long long* coarse_prefix = nullptr;   // blocks of 128 modes
  long long* sweep_prefix = nullptr;    // blocks of (modes / tb) x n_sub
  long long coarse_total = 0, sweep_total = 0;
  size_t sweep_smem = 0;
  // jobs are ordered by subdomain length: items [0, sweep_split) belong to short subdomains and
  // run in their own launch with sweep_smem_short, so long ones do not set everyone's occupancy
  long long sweep_split = 0;
  size_t sweep_smem_short = 0;
  int sweep_tb = 128;
  double coarse_flops = 0, coarse_bytes = 0, sweep_flops = 0, sweep_bytes = 0;
  // instances whose coarse solve is the cyclic reduction: their own job and item tables
  SpecJob* spec_cr = nullptr;
  long long* cr_prefix = nullptr;
  int cr_njobs = 0;
  long long cr_total = 0;
  size_t cr_smem = 0;
  MatvecJob* mv = nullptr;
  long long* mv_prefix = nullptr;
  long long mv_total = 0;
  double mv_V = 0;
  // instances large enough to fill the GPU alone whose transforms run on the tensor cores:
  // one 2D transform each, [0] forward, [1] inverse
  std::vector<DstJob> oz_jobs[2];
};

// Item lookup of the batched persistent kernels: item t belongs to job k with
// prefix[k] <= t < prefix[k+1]. Each block copies the prefix table (at most KKT_BATCH_MAX + 1
// entries) to shared memory once, so the per-item search costs no global-memory round trips.
__device__ __forceinline__ void batch_prefix_load(long long* sp, const long long* __restrict__ prefix, int nj) {
  for (int i = threadIdx.x; i <= nj; i += blockDim.x) sp[i] = prefix[i];
  __syncthreads();
}
__device__ __forceinline__ int batch_find(const long long* sp, int nj, long long t) {
  int lo = 0, hi = nj - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (sp[mid] <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Fill the DST tables of `slot` for passes `first_pass`, first_pass + 1 (forward rows/cols or
// inverse rows/cols) from jobs (synchronous copies); launch one pass from the tables.
int dst_batched_prepare(BatchSlot& slot, int first_pass, const DstJob* jobs, int njobs, int tile_lines);
int dst_batched_launch(const BatchSlot& slot, int pass, cudaStream_t st);
// True when the instance's 2D transforms run on the tensor cores and one of its GEMM passes has
// at least one tile per SM (a batch then transforms it alone rather than in the line tables).
bool dst_tensor_fills_gpu(const kkt_handle* h);
// spectral coarse + sweeps for all jobs of the slot (FP64), scale_dev: per-instance 1/eta
int spectral_batched_prepare(BatchSlot& slot, const SpecJob* jobs, int njobs);
int spectral_batched_launch(const BatchSlot& slot, const double* scale_dev, cudaStream_t st);
int matvec_batched_prepare(BatchSlot& slot, const MatvecJob* jobs, int njobs);
int matvec_batched_launch(const BatchSlot& slot, const double* scale_dev, cudaStream_t st);
void batch_slot_free(BatchSlot& slot);



}  // namespace kkt
