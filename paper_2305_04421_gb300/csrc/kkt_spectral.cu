// The two-level time-DD approximation of S-hat^{-1} (Section 3, Eqs 13-15) in the sine basis.
//
// After the 2D DST every operator of the preconditioner is diagonal in space: Jhat's block
// becomes the scalar mu_q = a + dt nu (lambda_x[k] + lambda_y[l]) for mode q = l*Mx + k, so
//   S-hat = T(mu)/h per mode, T = Jhat Jhat^T tridiagonal in time:
//           T_11 = mu^2, T_nn = 1 + mu^2 (n >= 2), T_{n,n+-1} = -mu.
// Per mode the kernels below carry out, in this order:
//   coarse_solve_kernel  R_0 r (sums over each subdomain's owned nodes against (1, phi)),
//                        then S_0 c' = R_0 r with S_0 = Z^T T Z / h, block tridiagonal with
//                        2x2 blocks (mu^2 P0 + P1 - mu P2)/h on the diagonal and the rank-one
//                        coupling -mu/h (1, phi_last(s)) (1, phi_first(s+1))^T between
//                        neighbours, solved by block Thomas elimination (S_0 is SPD);
//   sweep_kernel         x_0 = Z c', r' = r - T x_0 / h, then on each subdomain the forward
//                        sweep v_n = (r'_n + v_{n-1}) / mu with zero state before its first
//                        node (Jhat_s^{-1}, the extra node of Q_s carries zero), g = h v, and
//                        the backward sweep y_n = (g_n + y_{n+1}) / mu with zero terminal
//                        state (Jhat_s^{-T}); owned nodes receive y (+ x_0).
// The coarse time solve is FP64 in every form. In the reduced-precision forms the spectral
// coefficients arrive in FP32 (from the tensor-core transforms), the sweeps run in FP32 and
// write the type the inverse transform reads (BF16 or FP32); the residual r - S-hat x_0 is
// formed in FP64 before rounding.
#include <cuda_bf16.h>

#include <algorithm>
#include <vector>

#include "kkt_internal.cuh"

namespace kkt {
namespace {



// (q < 2^31: at most 1023^2 modes; a 32-bit division stays off the FP64 pipe)
__device__ __forceinline__ double mode_mu(const SpecParams& p, long long q) {
  const int l = static_cast<int>(q) / p.Mx;
  const int k = static_cast<int>(q) - l * p.Mx;
  return p.a + p.dtnu * (p.lx[k] + p.ly[l]);
}

template <typename TI>
__device__ __forceinline__ double load_d(const TI* p) {
  return static_cast<double>(__ldg(p));
}

template <typename TO>
__device__ __forceinline__ TO store_cast(double v) {
  return static_cast<TO>(v);
}
template <>
__device__ __forceinline__ __nv_bfloat16 store_cast<__nv_bfloat16>(double v) {
  return __double2bfloat16(v);
}

// hi + lo parts in the output type (for the split inverse transforms): hi = rounded value,
// lo = rounded remainder; TF32 operands read FP32 words, so hi is rounded to 10 mantissa bits
template <typename TO>
__device__ __forceinline__ void store_split(TO* hi, TO* lo, long long i, float v);
template <>
__device__ __forceinline__ void store_split<__nv_bfloat16>(__nv_bfloat16* hi, __nv_bfloat16* lo, long long i, float v) {
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  hi[i] = h;
  lo[i] = __float2bfloat16_rn(v - __bfloat162float(h));
}
template <>
__device__ __forceinline__ void store_split<float>(float* hi, float* lo, long long i, float v) {
  const float h = __uint_as_float((__float_as_uint(v) + 0x1000u) & 0xFFFFE000u);
  hi[i] = h;
  lo[i] = v - h;
}
template <>
__device__ __forceinline__ void store_split<double>(double* hi, double* lo, long long i, float v) {
  hi[i] = v;
  lo[i] = 0.0;
}

// Block-Thomas factorisation of the per-mode coarse operator h S_0 = Z_t^T T(mu) Z_t, which
// depends on mu and the decomposition only: run once per configuration. Diagonal blocks
// G_s = mu^2 P0 + P1 - mu P2; the coupling between s-1 and s is E = -mu a b^T with
// a = (1, phi_last(s-1)), b = (1, phi_first(s)); D_s = G_s - E^T D_{s-1}^{-1} E.
__global__ void coarse_factor_kernel(SpecParams p, double* __restrict__ cf) {
  const long long q = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= p.N) return;
  const long long N = p.N;
  const double mu = mode_mu(p, q), mu2 = mu * mu;
  double d00 = 0, d01 = 0, d11 = 0, a1_prev = 0.0;
  for (int s = 0; s < p.n_sub; ++s) {
    const double* M = p.mom + 9 * s;
    double g00 = fma(mu2, M[0], M[3]) - mu * M[6];
    double g01 = fma(mu2, M[1], M[4]) - mu * M[7];
    double g11 = fma(mu2, M[2], M[5]) - mu * M[8];
    if (s > 0) {
      const double b1 = __ldg(p.phi + __ldg(p.ofirst + s) - 1);
      const double t0 = d00 + d01 * a1_prev, t1 = d01 + d11 * a1_prev;   // D^{-1} a
      const double f = mu2 * (t0 + t1 * a1_prev);
      g00 -= f;
      g01 -= f * b1;
      g11 -= f * b1 * b1;
    }
    const double id = 1.0 / (g00 * g11 - g01 * g01);
    d00 = g11 * id;
    d01 = -g01 * id;
    d11 = g00 * id;
    double* F = cf + static_cast<long long>(s) * 3 * N + q;
    F[0] = d00;
    F[N] = d01;
    F[2 * N] = d11;
    a1_prev = __ldg(p.phi + __ldg(p.olast + s) - 1);
  }
}

// R_0 r of subdomain s for mode q: the sums of r over the subdomain's owned nodes against
// (1, phi_n), times in_scale. FP32 input (the reduced-precision forms) is summed in compensated
// FP32 and widened once per subdomain; FP64 input in FP64.
template <typename TI>
__device__ __forceinline__ void restrict_sub(const TI* __restrict__ rhat, double in_scale, const SpecParams& p,
                                             long long q, int s, double& c0, double& c1) {
  const long long N = p.N;
  const int o1 = __ldg(p.ofirst + s), o2 = __ldg(p.olast + s);
  if constexpr (sizeof(TI) == 4) {
    float s0 = 0.f, e0 = 0.f, s1 = 0.f, e1 = 0.f;
#pragma unroll 4
    for (int n = o1; n <= o2; ++n) {
      const float r = __ldg(rhat + static_cast<long long>(n - 1) * N + q);
      const float y0 = r - e0, t0 = s0 + y0;
      e0 = (t0 - s0) - y0;
      s0 = t0;
      const float y1 = fmaf(r, __ldg(p.phi_f + n - 1), -e1), t1 = s1 + y1;
      e1 = (t1 - s1) - y1;
      s1 = t1;
    }
    c0 = static_cast<double>(s0) * in_scale;
    c1 = static_cast<double>(s1) * in_scale;
  } else {
    c0 = 0.0;
    c1 = 0.0;
#pragma unroll 4
    for (int n = o1; n <= o2; ++n) {
      const double r = load_d(rhat + static_cast<long long>(n - 1) * N + q) * in_scale;
      c0 += r;
      c1 = fma(r, __ldg(p.phi + n - 1), c1);
    }
  }
}

// R_0 r and the block-Thomas substitutions with the precomputed factors; c' = h x.
template <typename TI>
__device__ void coarse_body(const TI* __restrict__ rhat, double in_scale, const SpecParams& p,
                            double* __restrict__ cc, double* __restrict__ cy, long long q) {
  const long long N = p.N;
  const double mu = mode_mu(p, q);
  double y0 = 0, y1 = 0, t0 = 0, t1 = 0;   // eliminated rhs of s-1 and D_{s-1}^{-1} a_{s-1}
  int learned = -1;                          // index among the learned modes, if any
  if (p.learn_k > 0) {
    const int l = static_cast<int>(q) / p.Mx, k = static_cast<int>(q) - l * p.Mx;
    if (k < p.learn_k && l < p.learn_k) learned = static_cast<int>(l * p.learn_k + k);
  }
  for (int s = 0; s < p.n_sub; ++s) {
    double c0, c1;
    restrict_sub<TI>(rhat, in_scale, p, q, s, c0, c1);
    const int o1 = __ldg(p.ofirst + s), o2 = __ldg(p.olast + s);
    if (learned >= 0) {
      p.learn_c[(learned * p.n_sub + s) * 2LL] = c0;
      p.learn_c[(learned * p.n_sub + s) * 2LL + 1] = c1;
    }
    if (s > 0) {
      // y_s = c_s - E^T D^{-1} y_{s-1} = c_s + mu b (a^T D^{-1} y_{s-1})
      const double b1 = __ldg(p.phi + o1 - 1);
      const double aDy = t0 * y0 + t1 * y1;
      c0 += mu * aDy;
      c1 += mu * b1 * aDy;
    }
    y0 = c0;
    y1 = c1;
    cy[(2LL * s) * N + q] = y0;
    cy[(2LL * s + 1) * N + q] = y1;
    const double* F = p.cf + static_cast<long long>(s) * 3 * N + q;
    const double d00 = F[0], d01 = F[N], d11 = F[2 * N];
    const double a1 = __ldg(p.phi + o2 - 1);
    t0 = d00 + d01 * a1;
    t1 = d01 + d11 * a1;
  }
  // back substitution: x_s = D_s^{-1} (y_s - E_s x_{s+1}) = D_s^{-1} (y_s + mu a_s (b_{s+1}^T x_{s+1}))
  double x0 = 0, x1 = 0;
  for (int s = p.n_sub - 1; s >= 0; --s) {
    const double* F = p.cf + static_cast<long long>(s) * 3 * N + q;
    const double d00 = F[0], d01 = F[N], d11 = F[2 * N];
    double z0 = cy[(2LL * s) * N + q], z1 = cy[(2LL * s + 1) * N + q];
    if (s + 1 < p.n_sub) {
      const double a1 = __ldg(p.phi + __ldg(p.olast + s) - 1);
      const double b1 = __ldg(p.phi + __ldg(p.ofirst + s + 1) - 1);
      const double bx = x0 + b1 * x1;
      z0 += mu * bx;
      z1 += mu * a1 * bx;
    }
    x0 = d00 * z0 + d01 * z1;
    x1 = d01 * z0 + d11 * z1;
    cc[(2LL * s) * N + q] = p.h * x0;
    cc[(2LL * s + 1) * N + q] = p.h * x1;
  }
}

template <typename TI>
__global__ void coarse_solve_kernel(const TI* __restrict__ rhat, double in_scale, SpecParams p,
                                    double* __restrict__ cc, double* __restrict__ cy) {
  const long long q = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q < p.N) coarse_body<TI>(rhat, in_scale, p, cc, cy, q);
}

// Multilevel solve of the same per-mode coarse system (Z_t^T T(mu) Z_t) x = R_0 r by block
// cyclic reduction. Block s (subdomain s) has the symmetric diagonal block
// D_s = mu^2 P0 + P1 - mu P2 and the coupling U_s = -mu a_s b_{s+1}^T to block s+1
// (a_s = (1, phi_last(s)), b_{s+1} = (1, phi_first(s+1))); row s reads
//   U_{s-1}^T x_{s-1} + D_s x_s + U_s x_{s+1} = c_s.
// Level l works on the blocks whose index is a multiple of 2^l. Each even-positioned block j
// takes in its odd-positioned neighbours o1 < j < o2 (the Schur complement onto the even
// blocks, again symmetric block tridiagonal):
//   D_j <- D_j - U_o1^T D_o1^-1 U_o1 - U_j D_o2^-1 U_j^T
//   c_j <- c_j - U_o1^T D_o1^-1 c_o1 - U_j D_o2^-1 c_o2
//   U_j <- -U_j D_o2^-1 U_o2             (its coupling to the next even block)
// and the old U_j is kept as o2's left coupling. Each odd block's D is inverted once, in
// place, before its neighbours use it. After ceil(log2 N_D) levels block 0 is alone; the way
// back solves, level by level, x_o = D_o^-1 (c_o - L_o^T x_left - U_o x_right) with the values
// the block had when it was eliminated. c' = h x as in block Thomas.
//
// A CTA holds `mpc` modes in shared memory, 13 doubles per block and mode: D (3, D^-1 once
// the block is eliminated), U (4), L (4), c (2, overwritten by x). Thread t serves mode t % mpc (consecutive threads read
// consecutive modes) and, with the other blockDim.x / mpc threads of that mode, strides over
// its subdomains and eliminations. Threads past the last mode only join the barriers.
constexpr int kCrThreads = 256;
constexpr int kCrFields = 13;
// AUTO on the FP64 path: the cyclic reduction with stored factors whenever those factors take at
// most kCyclicAutoFactorBytes, else block Thomas. Measured on GB300 (kkt_coarse_apply) the stored-
// factor cyclic solve is never slower than Thomas, from 225 modes (4.7x faster at N_D = 640) up
// to the benchmark's 65025 modes (equal there, 10.27 against 10.23 ms), and 9 % faster at 16129
// modes; above the cap the factors cost device memory (632 MB at 65025 modes, N_D = 64) for
// no measurable gain. The mixed forms' padded modes eliminate in every solve, so there AUTO keeps
// the crossover measured for that kernel: cyclic below kCyclicBelowModes modes (ahead by 3 % at
// 9025 modes with N_D = 64, Thomas ahead by 5 % at 16129 modes with N_D = 410).
constexpr long long kCyclicBelowModes = 12288;
constexpr double kCyclicAutoFactorBytes = 256.0 * 1024 * 1024;

__device__ __forceinline__ void sym_inv(double d00, double d01, double d11, double& i00, double& i01, double& i11) {
  const double id = 1.0 / (d00 * d11 - d01 * d01);
  i00 = d11 * id;
  i01 = -d01 * id;
  i11 = d00 * id;
}

// Modes per CTA of the cyclic-reduction solve: the largest power of two up to 32 whose blocks
// fit in 96 KB of shared memory (two CTAs per SM); 0 when one mode does not fit in 200 KB.
__host__ __device__ inline int cr_modes_per_cta(int n_sub) {
  const size_t per_mode = static_cast<size_t>(kCrFields) * n_sub * sizeof(double);
  if (per_mode > 200 * 1024) return 0;
  int mpc = 32;
  while (mpc > 1 && mpc * per_mode > 96 * 1024) mpc /= 2;
  return mpc;
}

// One CTA's group of modes (group * mpc ..): the whole solve, ending with c' in cc. Every thread
// of the block must call it (it synchronises the block).
template <typename TI>
__device__ void coarse_cr_body(const TI* __restrict__ rhat, double in_scale, const SpecParams& p, int mpc,
                               long long group, double* __restrict__ cc, double* __restrict__ cr_sm) {
  const int n = p.n_sub;
  const int m = threadIdx.x % mpc, w = threadIdx.x / mpc, W = blockDim.x / mpc;
  const long long q = group * mpc + m;
  const bool active = q < p.N;
  // field f of mode m: cr_sm[(f * mpc + m) * n + s]
  double* const F = cr_sm + static_cast<long long>(m) * n;
  const long long fs = static_cast<long long>(mpc) * n;   // stride between fields
  double *D00 = F, *D01 = F + fs, *D11 = F + 2 * fs;
  double *U00 = F + 3 * fs, *U01 = F + 4 * fs, *U10 = F + 5 * fs, *U11 = F + 6 * fs;
  double *L00 = F + 7 * fs, *L01 = F + 8 * fs, *L10 = F + 9 * fs, *L11 = F + 10 * fs;
  double *C0 = F + 11 * fs, *C1 = F + 12 * fs;

  const double mu = active ? mode_mu(p, q) : 1.0, mu2 = mu * mu;
  for (int s = w; s < n; s += W) {
    if (!active) continue;
    double c0, c1;
    restrict_sub<TI>(rhat, in_scale, p, q, s, c0, c1);
    C0[s] = c0;
    C1[s] = c1;
    const double* M = p.mom + 9 * s;
    D00[s] = fma(mu2, M[0], M[3]) - mu * M[6];
    D01[s] = fma(mu2, M[1], M[4]) - mu * M[7];
    D11[s] = fma(mu2, M[2], M[5]) - mu * M[8];
    double a1 = 0.0, b1 = 0.0, g = 0.0;
    if (s + 1 < n) {
      a1 = __ldg(p.phi + __ldg(p.olast + s) - 1);
      b1 = __ldg(p.phi + __ldg(p.ofirst + s + 1) - 1);
      g = -mu;
    }
    U00[s] = g;
    U01[s] = g * b1;
    U10[s] = g * a1;
    U11[s] = g * a1 * b1;
  }
  __syncthreads();

  int top = 1;   // first stride at which one block is left
  for (int st = 1; st < n; st *= 2) {
    const int cnt = (n + st - 1) / st;   // blocks of this level
    // the blocks eliminated at this level replace D by D^-1 (used by both neighbours and on
    // the way back)
    for (int e = w; 2 * e + 1 < cnt; e += W) {
      if (!active) continue;
      const int o = (2 * e + 1) * st;
      double i00, i01, i11;
      sym_inv(D00[o], D01[o], D11[o], i00, i01, i11);
      D00[o] = i00;
      D01[o] = i01;
      D11[o] = i11;
    }
    __syncthreads();
    for (int e = w; 2 * e < cnt; e += W) {
      if (!active) continue;
      const int k = 2 * e, j = k * st;
      double d00 = D00[j], d01 = D01[j], d11 = D11[j], c0 = C0[j], c1 = C1[j];
      if (k >= 1) {   // left neighbour o1: D_j -= U^T D_o1^-1 U, c_j -= U^T D_o1^-1 c_o1 (U = U_o1)
        const int o = j - st;
        const double i00 = D00[o], i01 = D01[o], i11 = D11[o];
        const double u00 = U00[o], u01 = U01[o], u10 = U10[o], u11 = U11[o];
        const double x00 = i00 * u00 + i01 * u10, x01 = i00 * u01 + i01 * u11;   // X = D^-1 U
        const double x10 = i01 * u00 + i11 * u10, x11 = i01 * u01 + i11 * u11;
        d00 -= u00 * x00 + u10 * x10;
        d01 -= u00 * x01 + u10 * x11;
        d11 -= u01 * x01 + u11 * x11;
        const double y0 = i00 * C0[o] + i01 * C1[o], y1 = i01 * C0[o] + i11 * C1[o];
        c0 -= u00 * y0 + u10 * y1;
        c1 -= u01 * y0 + u11 * y1;
      }
      if (k + 1 < cnt) {   // right neighbour o2: Y = U_j D_o2^-1
        const int o = j + st;
        const double i00 = D00[o], i01 = D01[o], i11 = D11[o];
        const double u00 = U00[j], u01 = U01[j], u10 = U10[j], u11 = U11[j];
        L00[o] = u00;
        L01[o] = u01;
        L10[o] = u10;
        L11[o] = u11;
        const double y00 = u00 * i00 + u01 * i01, y01 = u00 * i01 + u01 * i11;
        const double y10 = u10 * i00 + u11 * i01, y11 = u10 * i01 + u11 * i11;
        d00 -= y00 * u00 + y01 * u01;   // D_j -= Y U_j^T
        d01 -= y00 * u10 + y01 * u11;
        d11 -= y10 * u10 + y11 * u11;
        c0 -= y00 * C0[o] + y01 * C1[o];
        c1 -= y10 * C0[o] + y11 * C1[o];
        const double v00 = U00[o], v01 = U01[o], v10 = U10[o], v11 = U11[o];   // U_j <- -Y U_o2
        U00[j] = -(y00 * v00 + y01 * v10);
        U01[j] = -(y00 * v01 + y01 * v11);
        U10[j] = -(y10 * v00 + y11 * v10);
        U11[j] = -(y10 * v01 + y11 * v11);
      }
      D00[j] = d00;
      D01[j] = d01;
      D11[j] = d11;
      C0[j] = c0;
      C1[j] = c1;
    }
    __syncthreads();
    top = 2 * st;
  }

  if (active && w == 0) {   // the last block: x_0 = D_0^-1 c_0
    double i00, i01, i11;
    sym_inv(D00[0], D01[0], D11[0], i00, i01, i11);
    const double c0 = C0[0], c1 = C1[0];
    C0[0] = i00 * c0 + i01 * c1;
    C1[0] = i01 * c0 + i11 * c1;
  }
  __syncthreads();

  for (int st = top / 2; st >= 1; st /= 2) {
    const int cnt = (n + st - 1) / st;
    for (int e = w; 2 * e + 1 < cnt; e += W) {
      if (!active) continue;
      const int k = 2 * e + 1, o = k * st, left = o - st;
      const double xl0 = C0[left], xl1 = C1[left];
      double r0 = C0[o] - (L00[o] * xl0 + L10[o] * xl1);   // c_o - L^T x_left
      double r1 = C1[o] - (L01[o] * xl0 + L11[o] * xl1);
      if (k + 1 < cnt) {
        const int right = o + st;
        const double xr0 = C0[right], xr1 = C1[right];
        r0 -= U00[o] * xr0 + U01[o] * xr1;
        r1 -= U10[o] * xr0 + U11[o] * xr1;
      }
      const double i00 = D00[o], i01 = D01[o], i11 = D11[o];   // D_o^-1, stored at its level
      C0[o] = i00 * r0 + i01 * r1;
      C1[o] = i01 * r0 + i11 * r1;
    }
    __syncthreads();
  }

  const long long N = p.N;
  for (int s = w; s < n; s += W) {
    if (!active) continue;
    cc[(2LL * s) * N + q] = p.h * C0[s];
    cc[(2LL * s + 1) * N + q] = p.h * C1[s];
  }
}

template <typename TI>
__global__ void __launch_bounds__(kCrThreads) coarse_cr_kernel(const TI* __restrict__ rhat, double in_scale,
                                                                SpecParams p, int mpc, double* __restrict__ cc) {
  extern __shared__ __align__(16) double cr_sm[];
  coarse_cr_body<TI>(rhat, in_scale, p, mpc, blockIdx.x, cc, cr_sm);
}

// The cyclic reduction with its factors computed once per configuration. The matrices of every
// level depend only on mu and the decomposition, so coarse_cr_factor_kernel runs the forward
// elimination on them alone and stores, per mode (slot-major: F[slot * N + q]):
//   per block s (slots 11 s ..): D_s^-1 (3), P_s = D_s^-1 U_left^T (4), Q_s = D_s^-1 U_s (4)
//     for the block's own level (U_left the coupling of its left neighbour there);
//   per level l and kept block j = 2 e 2^l (slots 11 n + 8 (off_l + e) ..): A = U_o1^T D_o1^-1
//     and B = U_j D_o2^-1, with off_l the kept blocks of the levels below.
// A solve (coarse_crf_body) then moves only the right-hand side: c_j -= A c_o1 + B c_o2 on the
// way down, x_o = D_o^-1 c_o - P x_left - Q x_right on the way up: about 20 FMAs per block
// against about 80 with the elimination, and 2 doubles per block in shared memory.
__host__ __device__ inline long long cr_kept_total(int n) {
  long long K = 0;
  for (int st = 1; st < n; st *= 2) K += ((n + st - 1) / st + 1) / 2;
  return K;
}
__host__ __device__ inline long long cr_factor_slots(int n) { return 11LL * n + 8LL * cr_kept_total(n); }

__global__ void __launch_bounds__(kCrThreads) coarse_cr_factor_kernel(SpecParams p, int mpc, double* __restrict__ F) {
  extern __shared__ __align__(16) double cr_sm[];
  const int n = p.n_sub;
  const int m = threadIdx.x % mpc, w = threadIdx.x / mpc, W = blockDim.x / mpc;
  const long long N = p.N;
  const long long q = static_cast<long long>(blockIdx.x) * mpc + m;
  const bool active = q < N;
  double* const Fs = cr_sm + static_cast<long long>(m) * n;
  const long long fs = static_cast<long long>(mpc) * n;
  double *D00 = Fs, *D01 = Fs + fs, *D11 = Fs + 2 * fs;
  double *U00 = Fs + 3 * fs, *U01 = Fs + 4 * fs, *U10 = Fs + 5 * fs, *U11 = Fs + 6 * fs;
  const double mu = active ? mode_mu(p, q) : 1.0, mu2 = mu * mu;
  for (int s = w; s < n; s += W) {
    if (!active) continue;
    const double* M = p.mom + 9 * s;
    D00[s] = fma(mu2, M[0], M[3]) - mu * M[6];
    D01[s] = fma(mu2, M[1], M[4]) - mu * M[7];
    D11[s] = fma(mu2, M[2], M[5]) - mu * M[8];
    double a1 = 0.0, b1 = 0.0, g = 0.0;
    if (s + 1 < n) {
      a1 = __ldg(p.phi + __ldg(p.olast + s) - 1);
      b1 = __ldg(p.phi + __ldg(p.ofirst + s + 1) - 1);
      g = -mu;
    }
    U00[s] = g;
    U01[s] = g * b1;
    U10[s] = g * a1;
    U11[s] = g * a1 * b1;
  }
  __syncthreads();
  long long off = 0;   // kept blocks of the levels below
  for (int st = 1; st < n; st *= 2) {
    const int cnt = (n + st - 1) / st;
    for (int e = w; 2 * e + 1 < cnt; e += W) {   // eliminated blocks: D^-1, P, Q
      if (!active) continue;
      const int k = 2 * e + 1, o = k * st, left = o - st;
      double i00, i01, i11;
      sym_inv(D00[o], D01[o], D11[o], i00, i01, i11);
      const double l00 = U00[left], l01 = U01[left], l10 = U10[left], l11 = U11[left];
      double q00 = 0, q01 = 0, q10 = 0, q11 = 0;
      if (k + 1 < cnt) {
        q00 = i00 * U00[o] + i01 * U10[o];
        q01 = i00 * U01[o] + i01 * U11[o];
        q10 = i01 * U00[o] + i11 * U10[o];
        q11 = i01 * U01[o] + i11 * U11[o];
      }
      double* B = F + 11LL * o * N + q;
      B[0] = i00;
      B[N] = i01;
      B[2 * N] = i11;
      B[3 * N] = i00 * l00 + i01 * l01;   // P = D^-1 U_left^T
      B[4 * N] = i00 * l10 + i01 * l11;
      B[5 * N] = i01 * l00 + i11 * l01;
      B[6 * N] = i01 * l10 + i11 * l11;
      B[7 * N] = q00;
      B[8 * N] = q01;
      B[9 * N] = q10;
      B[10 * N] = q11;
      D00[o] = i00;
      D01[o] = i01;
      D11[o] = i11;
    }
    __syncthreads();
    for (int e = w; 2 * e < cnt; e += W) {   // kept blocks: A, B, and the Schur update
      if (!active) continue;
      const int k = 2 * e, j = k * st;
      double d00 = D00[j], d01 = D01[j], d11 = D11[j];
      double a00 = 0, a01 = 0, a10 = 0, a11 = 0, b00 = 0, b01 = 0, b10 = 0, b11 = 0;
      if (k >= 1) {   // A = U_o1^T D_o1^-1; D_j -= A U_o1
        const int o = j - st;
        const double i00 = D00[o], i01 = D01[o], i11 = D11[o];
        const double u00 = U00[o], u01 = U01[o], u10 = U10[o], u11 = U11[o];
        a00 = u00 * i00 + u10 * i01;
        a01 = u00 * i01 + u10 * i11;
        a10 = u01 * i00 + u11 * i01;
        a11 = u01 * i01 + u11 * i11;
        d00 -= a00 * u00 + a01 * u10;
        d01 -= a00 * u01 + a01 * u11;
        d11 -= a10 * u01 + a11 * u11;
      }
      if (k + 1 < cnt) {   // B = U_j D_o2^-1; D_j -= B U_j^T; U_j <- -B U_o2
        const int o = j + st;
        const double i00 = D00[o], i01 = D01[o], i11 = D11[o];
        const double u00 = U00[j], u01 = U01[j], u10 = U10[j], u11 = U11[j];
        b00 = u00 * i00 + u01 * i01;
        b01 = u00 * i01 + u01 * i11;
        b10 = u10 * i00 + u11 * i01;
        b11 = u10 * i01 + u11 * i11;
        d00 -= b00 * u00 + b01 * u01;
        d01 -= b00 * u10 + b01 * u11;
        d11 -= b10 * u10 + b11 * u11;
        const double v00 = U00[o], v01 = U01[o], v10 = U10[o], v11 = U11[o];
        U00[j] = -(b00 * v00 + b01 * v10);
        U01[j] = -(b00 * v01 + b01 * v11);
        U10[j] = -(b10 * v00 + b11 * v10);
        U11[j] = -(b10 * v01 + b11 * v11);
      }
      D00[j] = d00;
      D01[j] = d01;
      D11[j] = d11;
      double* A = F + (11LL * n + 8 * (off + e)) * N + q;
      A[0] = a00;
      A[N] = a01;
      A[2 * N] = a10;
      A[3 * N] = a11;
      A[4 * N] = b00;
      A[5 * N] = b01;
      A[6 * N] = b10;
      A[7 * N] = b11;
    }
    __syncthreads();
    off += (cnt + 1) / 2;
  }
  if (active && w == 0) {   // the last block
    double i00, i01, i11;
    sym_inv(D00[0], D01[0], D11[0], i00, i01, i11);
    F[q] = i00;
    F[N + q] = i01;
    F[2 * N + q] = i11;
  }
}

// A solve with the stored factors: R_0 r, the right-hand side down the levels, back up, c' = h x.
// Shared memory: c (2 doubles per block and mode, overwritten by x).
template <typename TI>
__device__ void coarse_crf_body(const TI* __restrict__ rhat, double in_scale, const SpecParams& p, int mpc,
                                long long group, double* __restrict__ cc, double* __restrict__ cr_sm) {
  const int n = p.n_sub;
  const int m = threadIdx.x % mpc, w = threadIdx.x / mpc, W = blockDim.x / mpc;
  const long long N = p.N;
  const long long q = group * mpc + m;
  const bool active = q < N;
  double* const C0 = cr_sm + static_cast<long long>(m) * n;
  double* const C1 = C0 + static_cast<long long>(mpc) * n;
  const double* __restrict__ F = p.crf;
  for (int s = w; s < n; s += W) {
    if (!active) continue;
    double c0, c1;
    restrict_sub<TI>(rhat, in_scale, p, q, s, c0, c1);
    C0[s] = c0;
    C1[s] = c1;
  }
  __syncthreads();
  long long off = 0;
  int top = 1;
  for (int st = 1; st < n; st *= 2) {
    const int cnt = (n + st - 1) / st;
    for (int e = w; 2 * e < cnt; e += W) {
      if (!active) continue;
      const int k = 2 * e, j = k * st;
      const double* A = F + (11LL * n + 8 * (off + e)) * N + q;
      double c0 = C0[j], c1 = C1[j];
      if (k >= 1) {
        const double y0 = C0[j - st], y1 = C1[j - st];
        c0 -= A[0] * y0 + A[N] * y1;
        c1 -= A[2 * N] * y0 + A[3 * N] * y1;
      }
      if (k + 1 < cnt) {
        const double y0 = C0[j + st], y1 = C1[j + st];
        c0 -= A[4 * N] * y0 + A[5 * N] * y1;
        c1 -= A[6 * N] * y0 + A[7 * N] * y1;
      }
      C0[j] = c0;
      C1[j] = c1;
    }
    __syncthreads();
    off += (cnt + 1) / 2;
    top = 2 * st;
  }
  if (active && w == 0) {
    const double c0 = C0[0], c1 = C1[0];
    C0[0] = F[q] * c0 + F[N + q] * c1;
    C1[0] = F[N + q] * c0 + F[2 * N + q] * c1;
  }
  __syncthreads();
  for (int st = top / 2; st >= 1; st /= 2) {
    const int cnt = (n + st - 1) / st;
    for (int e = w; 2 * e + 1 < cnt; e += W) {
      if (!active) continue;
      const int k = 2 * e + 1, o = k * st;
      const double* B = F + 11LL * o * N + q;
      const double c0 = C0[o], c1 = C1[o], xl0 = C0[o - st], xl1 = C1[o - st];
      double x0 = B[0] * c0 + B[N] * c1 - (B[3 * N] * xl0 + B[4 * N] * xl1);
      double x1 = B[N] * c0 + B[2 * N] * c1 - (B[5 * N] * xl0 + B[6 * N] * xl1);
      if (k + 1 < cnt) {
        const double xr0 = C0[o + st], xr1 = C1[o + st];
        x0 -= B[7 * N] * xr0 + B[8 * N] * xr1;
        x1 -= B[9 * N] * xr0 + B[10 * N] * xr1;
      }
      C0[o] = x0;
      C1[o] = x1;
    }
    __syncthreads();
  }
  for (int s = w; s < n; s += W) {
    if (!active) continue;
    cc[(2LL * s) * N + q] = p.h * C0[s];
    cc[(2LL * s + 1) * N + q] = p.h * C1[s];
  }
}

template <typename TI>
__global__ void __launch_bounds__(kCrThreads) coarse_crf_kernel(const TI* __restrict__ rhat, double in_scale,
                                                                 SpecParams p, int mpc, double* __restrict__ cc) {
  extern __shared__ __align__(16) double cr_sm[];
  coarse_crf_body<TI>(rhat, in_scale, p, mpc, blockIdx.x, cc, cr_sm);
}

// Learned coarse correction of one mode: the network's direction d, scaled by the
// minimal-residual step alpha = (G d)^T c / ||G d||^2 on the mode's coarse operator G = h S_0(mu)
// (the scale that minimises the coarse residual along d, the quantity training minimises).
// mode 0: kept when ||c - alpha G d||^2 <= ||c||^2 / 4, else the exact solve's result stays;
// mode 1: no coarse correction on the learned modes (the ablation); mode 2: always kept (the
// network alone; counts[1] then tallies the corrections the guard would have rejected). One
// warp per learned mode: lanes stride over the subdomains (coalesced reads of d and c) and the
// sums are reduced with shuffles.
__device__ __forceinline__ double warp_sum_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void learned_apply_kernel(SpecParams p, const float* __restrict__ y, int mode, double* __restrict__ cc,
                                     long long* __restrict__ counts) {
  const int w = static_cast<int>((static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  const int K = p.learn_k;
  if (w >= K * K) return;   // uniform per warp
  const int k = w % K, l = w / K;
  const long long q = static_cast<long long>(l) * p.Mx + k, N = p.N;
  if (mode == 1) {
    for (int s = lane; s < p.n_sub; s += 32) {
      cc[(2LL * s) * N + q] = 0.0;
      cc[(2LL * s + 1) * N + q] = 0.0;
    }
    return;
  }
  const double mu = mode_mu(p, q), mu2 = mu * mu;
  const float* d = y + static_cast<long long>(w) * 2 * p.n_sub;
  const double* c = p.learn_c + static_cast<long long>(w) * 2 * p.n_sub;
  double gg = 0, gc = 0, cc2 = 0;
  for (int s = lane; s < p.n_sub; s += 32) {
    double e0, e1;
    coarse_op_apply_row(p.mom, p.phi, p.ofirst, p.olast, p.n_sub, mu, mu2, d, s, e0, e1);
    gg += e0 * e0 + e1 * e1;
    gc += e0 * c[2 * s] + e1 * c[2 * s + 1];
    cc2 += c[2 * s] * c[2 * s] + c[2 * s + 1] * c[2 * s + 1];
  }
  gg = warp_sum_d(gg);
  gc = warp_sum_d(gc);
  cc2 = warp_sum_d(cc2);
  const bool degenerate = !(gg > 0.0);
  const double alpha = degenerate ? 0.0 : gc / gg;
  double res2 = cc2;
  if (!degenerate) {
    res2 = 0;
    for (int s = lane; s < p.n_sub; s += 32) {
      double e0, e1;
      coarse_op_apply_row(p.mom, p.phi, p.ofirst, p.olast, p.n_sub, mu, mu2, d, s, e0, e1);
      const double r0 = c[2 * s] - alpha * e0, r1 = c[2 * s + 1] - alpha * e1;
      res2 += r0 * r0 + r1 * r1;
    }
    res2 = warp_sum_d(res2);
  }
  const bool guard_ok = !degenerate && res2 <= 0.25 * cc2;
  if (mode == 0 && !guard_ok) {
    if (lane == 0) atomicAdd(reinterpret_cast<unsigned long long*>(counts + 1), 1ull);
    return;
  }
  for (int s = lane; s < p.n_sub; s += 32) {
    cc[(2LL * s) * N + q] = p.h * alpha * d[2 * s];
    cc[(2LL * s + 1) * N + q] = p.h * alpha * d[2 * s + 1];
  }
  if (lane == 0) {
    atomicAdd(reinterpret_cast<unsigned long long*>(counts), 1ull);
    if (!guard_ok) atomicAdd(reinterpret_cast<unsigned long long*>(counts + 1), 1ull);
  }
}

// x_0 at node n (1-based), given the coarse pairs of the three subdomains around s.
template <typename TC>
__device__ __forceinline__ TC coarse_value(const SpecParams& p, int n, int s, const TC* c3) {
  if (n < 1 || n > p.Nt) return TC(0);
  const int o = __ldg(p.owner + n - 1) - s + 1;        // 0, 1, 2 for s-1, s, s+1
  if (o < 0 || o > 2) return TC(0);                     // cannot happen when every m_s >= 2
  // selects, not c3[2 * o]: a runtime index would put c3 in local memory
  const TC c0 = o == 0 ? c3[0] : (o == 1 ? c3[2] : c3[4]);
  const TC c1 = o == 0 ? c3[1] : (o == 1 ? c3[3] : c3[5]);
  // FP32 sweeps read phi in FP32: an FP64 load and conversion per node would run on the
  // FP64 pipe, which the reduced-precision forms keep for the coarse solve
  if constexpr (sizeof(TC) == 4) return c0 + c1 * __ldg(p.phi_f + n - 1);
  return c0 + c1 * static_cast<TC>(__ldg(p.phi + n - 1));
}

template <typename TI, typename TC, typename TO>
__device__ void sweep_body(const TI* __restrict__ rhat, double in_scale, TO* __restrict__ yhat,
                           TO* __restrict__ yhat_lo, const SpecParams& p, const double* __restrict__ cc,
                           TC* __restrict__ vglobal, int max_len, long long q, int s, TC* vs_smem) {
  const long long N = p.N;
  const double mud = mode_mu(p, q);
  const TC mu = static_cast<TC>(mud), mu2 = mu * mu;
  const TC inv_mu = TC(1) / mu;   // (FP32 reciprocal in the reduced-precision sweeps)
  const TC hc = static_cast<TC>(p.h), inv_h = static_cast<TC>(p.inv_h), scale = static_cast<TC>(in_scale);
  const int first = __ldg(p.first + s), last = __ldg(p.last + s);
  const int o1 = __ldg(p.ofirst + s), o2 = __ldg(p.olast + s);
  TC* vs;
  long long vstride;
  if (vglobal) {   // (RAS stores two values per node: the scratch holds 2 max_len per mode)
    vs = vglobal + static_cast<long long>(s) * (p.ras ? 2 : 1) * max_len * N + q;
    vstride = N;
  } else {
    vs = vs_smem + threadIdx.x;
    vstride = blockDim.x;
  }
  TC c3[6] = {0, 0, 0, 0, 0, 0};
  if (p.two_level) {
    for (int o = 0; o < 3; ++o) {
      const int so = s - 1 + o;
      if (so >= 0 && so < p.n_sub) {
        c3[2 * o] = static_cast<TC>(cc[(2LL * so) * N + q]);
        c3[2 * o + 1] = static_cast<TC>(cc[(2LL * so + 1) * N + q]);
      }
    }
  }
  TC xm = 0, xc = 0, xp = 0;   // x_0 at n-1, n, n+1
  if (p.ras) {
    // RAS (Eq 9): the local Schur complement R_s S-hat R_s^T = T_s / h, T_s tridiagonal in time
    // over the subdomain's nodes (diagonal mu^2 at the global first node, mu^2 + 1 elsewhere,
    // off-diagonals -mu); T_s y = h r by the Thomas algorithm: forward elimination
    // m_n = b_n - mu^2 / m_n-1, d'_n = (h r_n + mu d'_n-1) / m_n (stored with 1 / m_n), then
    // y_n = d'_n + (mu / m_n) y_n+1. It differs from RASQ's (R_s Jhat R_s^T) (R_s Jhat R_s^T)^T
    // only in the first node's diagonal.
    TC* ws = vs + static_cast<long long>(max_len) * vstride;
    if (p.two_level) {
      xm = coarse_value<TC>(p, first - 1, s, c3);
      xc = coarse_value<TC>(p, first, s, c3);
    }
    TC dp = 0, im = 0;
    for (int n = first; n <= last; ++n) {
      TC r = static_cast<TC>(__ldg(rhat + static_cast<long long>(n - 1) * N + q)) * scale;
      if (p.two_level) {
        xp = coarse_value<TC>(p, n + 1, s, c3);
        if (p.multiplicative) {
          const TC tx = (n >= 2 ? mu2 + TC(1) : mu2) * xc - mu * (xm + xp);
          r = fma(-tx, inv_h, r);
        }
        xm = xc;
        xc = xp;
      }
      const TC bd = n >= 2 ? mu2 + TC(1) : mu2;
      const TC mth = n == first ? bd : fma(-mu2, im, bd);
      im = TC(1) / mth;
      dp = fma(hc, r, mu * dp) * im;
      vs[static_cast<long long>(n - first) * vstride] = dp;
      ws[static_cast<long long>(n - first) * vstride] = im;
    }
    TC y = 0;
    for (int n = last; n >= first; --n) {
      const long long i = static_cast<long long>(n - first) * vstride;
      y = fma(mu * ws[i], y, vs[i]);
      if (n >= o1 && n <= o2) {
        TC out = y;
        if (p.two_level) out += coarse_value<TC>(p, n, s, c3);
        const long long o = static_cast<long long>(n - 1) * N + q;
        if (yhat_lo)
          store_split<TO>(yhat, yhat_lo, o, static_cast<float>(out));
        else
          yhat[o] = store_cast<TO>(static_cast<double>(out));
      }
    }
    return;
  }
  // forward sweep over the subdomain's nodes
  if (p.two_level) {
    xm = coarse_value<TC>(p, first - 1, s, c3);
    xc = coarse_value<TC>(p, first, s, c3);
  }
  TC v = 0;
  for (int n = first; n <= last; ++n) {
    TC r = static_cast<TC>(__ldg(rhat + static_cast<long long>(n - 1) * N + q)) * scale;
    if (p.two_level) {
      xp = coarse_value<TC>(p, n + 1, s, c3);
      if (p.multiplicative) {
        // r - (T x_0)_n / h, T_nn = mu^2 (+1 from n >= 2), T_{n,n+-1} = -mu
        const TC tx = (n >= 2 ? mu2 + TC(1) : mu2) * xc - mu * (xm + xp);
        r = fma(-tx, inv_h, r);
      }
      xm = xc;
      xc = xp;
    }
    v = (r + v) * inv_mu;
    vs[static_cast<long long>(n - first) * vstride] = v;
  }
  // backward sweep; keep owned nodes
  TC y = 0;
  for (int n = last; n >= first; --n) {
    y = fma(hc, vs[static_cast<long long>(n - first) * vstride], y) * inv_mu;
    if (n >= o1 && n <= o2) {
      TC out = y;
      if (p.two_level) out += coarse_value<TC>(p, n, s, c3);
      const long long o = static_cast<long long>(n - 1) * N + q;
      if (yhat_lo)
        store_split<TO>(yhat, yhat_lo, o, static_cast<float>(out));
      else
        yhat[o] = store_cast<TO>(static_cast<double>(out));
    }
  }
}

template <typename TI, typename TC, typename TO>
__global__ void sweep_kernel(const TI* __restrict__ rhat, double in_scale, TO* __restrict__ yhat,
                             TO* __restrict__ yhat_lo, SpecParams p, const double* __restrict__ cc,
                             TC* __restrict__ vglobal, int max_len) {
  extern __shared__ __align__(16) unsigned char vs_raw[];
  const long long q = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q < p.N)
    sweep_body<TI, TC, TO>(rhat, in_scale, yhat, yhat_lo, p, cc, vglobal, max_len, q, blockIdx.y,
                           reinterpret_cast<TC*>(vs_raw));
}


// Batched coarse solves: item = a block of 128 modes of one instance (FP64).
__global__ void coarse_batched(const SpecJob* __restrict__ jobs, const long long* __restrict__ prefix, int nj,
                               long long total, const double* __restrict__ scale_dev) {
  __shared__ long long sp[KKT_BATCH_MAX + 1];
  batch_prefix_load(sp, prefix, nj);
  for (long long t = blockIdx.x; t < total; t += gridDim.x) {
    const int k = batch_find(sp, nj, t);
    const SpecJob J = jobs[k];   // (a register copy: the stores below cannot alias it)
    const long long q = (t - sp[k]) * blockDim.x + threadIdx.x;
    if (q < J.p.N && J.p.two_level)
      coarse_body<double>(J.rhat, J.scale_base * scale_dev[J.scale_index], J.p, J.cc, J.cy, q);
  }
}

// Batched cyclic-reduction coarse solves: item = a group of cr_mpc modes of one instance (FP64),
// with stored factors or the elimination in the solve; the dynamic shared memory fits the
// largest group of the launch.
__global__ void __launch_bounds__(kCrThreads) coarse_cr_batched(const SpecJob* __restrict__ jobs,
                                                                 const long long* __restrict__ prefix, int nj,
                                                                 long long total, const double* __restrict__ scale_dev) {
  extern __shared__ __align__(16) double cr_sm[];
  __shared__ long long sp[KKT_BATCH_MAX + 1];
  batch_prefix_load(sp, prefix, nj);
  for (long long t = blockIdx.x; t < total; t += gridDim.x) {
    const int k = batch_find(sp, nj, t);
    const SpecJob J = jobs[k];   // (a register copy: the stores below cannot alias it)
    const double scale = J.scale_base * scale_dev[J.scale_index];
    if (J.p.crf)
      coarse_crf_body<double>(J.rhat, scale, J.p, J.p.cr_mpc, t - sp[k], J.cc, cr_sm);
    else
      coarse_cr_body<double>(J.rhat, scale, J.p, J.p.cr_mpc, t - sp[k], J.cc, cr_sm);
    __syncthreads();   // the next item reuses the shared memory
  }
}

// Batched sweeps: item = (block of modes, subdomain) of one instance (FP64).
__global__ void sweep_batched(const SpecJob* __restrict__ jobs, const long long* __restrict__ prefix, int nj,
                              long long t_begin, long long t_end, const double* __restrict__ scale_dev) {
  extern __shared__ __align__(16) unsigned char vs_raw[];
  __shared__ long long sp[KKT_BATCH_MAX + 1];
  batch_prefix_load(sp, prefix, nj);
  for (long long t = t_begin + blockIdx.x; t < t_end; t += gridDim.x) {
    const int k = batch_find(sp, nj, t);
    const SpecJob J = jobs[k];   // (a register copy: the stores below cannot alias it)
    const long long local = t - sp[k];
    const long long mblocks = (J.p.N + blockDim.x - 1) / blockDim.x;
    const int s = static_cast<int>(local / mblocks);
    const long long q = (local % mblocks) * blockDim.x + threadIdx.x;
    if (q < J.p.N)
      sweep_body<double, double, double>(J.rhat, J.scale_base * scale_dev[J.scale_index], J.yhat, nullptr, J.p, J.cc,
                                         nullptr, J.max_len, q, s, reinterpret_cast<double*>(vs_raw));
  }
}

__global__ void prolong_kernel(SpecParams p, const double* __restrict__ cc, double* __restrict__ xhat) {
  const long long q = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int n = blockIdx.y + 1;
  if (q >= p.N) return;
  const int o = __ldg(p.owner + n - 1);
  xhat[static_cast<long long>(n - 1) * p.N + q] =
      cc[(2LL * o) * p.N + q] + cc[(2LL * o + 1) * p.N + q] * __ldg(p.phi + n - 1);
}

// Modes per CTA of the factored solve (2 doubles per block and mode in shared memory): up to 32,
// within 96 KB, and few enough that the modes still make two CTAs per SM.
int crf_modes_per_cta(int n_sub, long long N) {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 152;
  }
  const size_t per_mode = 2 * static_cast<size_t>(n_sub) * sizeof(double);
  int mpc = 32;
  while (mpc > 1 && (mpc * per_mode > 96 * 1024 || N / mpc < 2LL * sms)) mpc /= 2;
  return mpc;
}

bool use_cyclic(const kkt_handle* h, const SpecParams& p, bool padded) {
  if (p.learn_k > 0 || cr_modes_per_cta(p.n_sub) == 0) return false;
  if (h->opt.coarse_solve == KKT_COARSE_SOLVE_CYCLIC) return true;
  if (h->opt.coarse_solve != KKT_COARSE_SOLVE_AUTO) return false;
  if (padded) return p.N < kCyclicBelowModes;
  return static_cast<double>(cr_factor_slots(p.n_sub)) * p.N * sizeof(double) <= kCyclicAutoFactorBytes;
}

SpecParams make_params(const kkt_handle* h, bool padded) {  // (padded: the mixed forms' mode grid)
  SpecParams p;
  const Geometry& g = h->g;
  p.Mx = padded ? h->tc.P : g.Mx;
  p.Nt = g.Nt;
  p.n_sub = g.n_sub;
  p.N = padded ? static_cast<long long>(h->tc.P) * h->tc.P : g.N;
  p.a = g.a;
  p.dtnu = g.dtnu;
  p.h = g.h;
  p.inv_h = 1.0 / g.h;
  p.cf = padded ? h->coarse_f_pad : h->coarse_f;
  p.lx = padded ? h->d_lx_pad : h->d_lx;
  p.ly = padded ? h->d_ly_pad : h->d_ly;
  p.first = h->dd.first;
  p.last = h->dd.last;
  p.ofirst = h->dd.ofirst;
  p.olast = h->dd.olast;
  p.owner = h->dd.owner;
  p.phi = h->dd.phi;
  p.phi_f = h->dd.phi_f;
  p.mom = h->dd.moments;
  p.two_level = h->opt.coarse != KKT_COARSE_NONE;
  p.learn_k = (h->opt.coarse == KKT_COARSE_LEARNED && h->mlp) ? h->learn_k : 0;
  p.learn_c = h->learn_c;
  p.multiplicative = h->opt.variant == KKT_MULTIPLICATIVE;
  p.ras = h->opt.local == KKT_LOCAL_RAS;
  p.cyclic = p.two_level && use_cyclic(h, p, padded);
  p.crf = (!padded && p.cyclic) ? h->cr_factors : nullptr;
  p.cr_mpc = p.crf ? crf_modes_per_cta(p.n_sub, p.N) : cr_modes_per_cta(p.n_sub);
  return p;
}

template <typename TI>
int launch_coarse(const kkt_handle* h, const SpecParams& p, const TI* rhat, double in_scale, cudaStream_t st) {
  const double V = static_cast<double>(p.N) * p.Nt;
  if (p.cyclic && p.crf) {
    const int mpc = p.cr_mpc;
    const size_t smem = 2 * static_cast<size_t>(p.n_sub) * mpc * sizeof(double);
    KKT_CUDA_TRY(cudaFuncSetAttribute(coarse_crf_kernel<TI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      static_cast<int>(smem)));
    // restriction: 2 flops per node; right-hand side down and back up: about 20 FMAs per block,
    // reading 19 stored factors per block
    ProfScope ps(KKT_K_COARSE, st, 2.0 * V + 40.0 * p.n_sub * p.N, V * sizeof(TI) + (16.0 + 152.0) * p.n_sub * p.N);
    const long long nb = (p.N + mpc - 1) / mpc;
    coarse_crf_kernel<TI><<<static_cast<unsigned>(nb), kCrThreads, smem, st>>>(rhat, in_scale, p, mpc, h->coarse_c);
    KKT_CUDA_TRY(cudaGetLastError());
    return KKT_OK;
  }
  if (p.cyclic) {
    const int mpc = cr_modes_per_cta(p.n_sub);
    const size_t smem = static_cast<size_t>(kCrFields) * p.n_sub * mpc * sizeof(double);
    KKT_CUDA_TRY(cudaFuncSetAttribute(coarse_cr_kernel<TI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      static_cast<int>(smem)));
    // restriction: 2 flops per node; reduction and substitution: ~80 flops per block (one 2 x 2
    // inverse, the block products with both neighbours, one back-substitution)
    ProfScope ps(KKT_K_COARSE, st, 2.0 * V + 80.0 * p.n_sub * p.N, V * sizeof(TI) + 16.0 * p.n_sub * p.N);
    const long long nb = (p.N + mpc - 1) / mpc;
    coarse_cr_kernel<TI><<<static_cast<unsigned>(nb), kCrThreads, smem, st>>>(rhat, in_scale, p, mpc, h->coarse_c);
    KKT_CUDA_TRY(cudaGetLastError());
    return KKT_OK;
  }
  const int tb = 128;
  const long long nb = (p.N + tb - 1) / tb;
  // restriction: 2 flops per node; substitutions: ~26 flops per subdomain; reads the coefficients
  // once, the factors twice, writes and reads the eliminated right-hand sides
  ProfScope ps(KKT_K_COARSE, st, 2.0 * V + 26.0 * p.n_sub * p.N, V * sizeof(TI) + 12.0 * 8.0 * p.n_sub * p.N);
  coarse_solve_kernel<TI><<<static_cast<unsigned>(nb), tb, 0, st>>>(rhat, in_scale, p, h->coarse_c, h->coarse_w);
  KKT_CUDA_TRY(cudaGetLastError());
  return KKT_OK;
}

template <typename TI, typename TC, typename TO>
int launch_sweeps(const kkt_handle* h, const SpecParams& p, const TI* rhat, double in_scale, TO* yhat,
                  cudaStream_t st, bool padded, TO* yhat_lo = nullptr) {
  if (static_cast<const void*>(rhat) == static_cast<const void*>(yhat))
    return set_error(KKT_ERR_INVALID_ARG, "spectral sweep needs distinct buffers");
  if (p.two_level) KKT_TRY(launch_coarse<TI>(h, p, rhat, in_scale, st));
  if (p.learn_k > 0) {
    // learned coarse directions for the lowest modes, then the Galerkin step and the guard
    const long long nl = static_cast<long long>(p.learn_k) * p.learn_k;
    KKT_TRY(mlp_make_input(h->learn_c, h->learn_feat, nl, 2 * p.n_sub, h->learn_x, st));
    KKT_TRY(mlp_forward(h->mlp, h->learn_x, static_cast<int>(nl), 1, st));
    KKT_TRY(spectral_learned_apply(h, padded, mlp_output(h->mlp), st));
  }
  // sweep storage: shared memory when a subdomain's nodes fit, else the global scratch
  const size_t limit = 200 * 1024;
  const size_t words = p.ras ? 2 : 1;   // values stored per node and mode
  int tb = 0;
  for (int cand : {128, 64, 32})
    if (words * h->td.max_len * cand * sizeof(TC) <= limit) {
      tb = cand;
      break;
    }
  size_t smem = 0;
  TC* vglob = nullptr;
  if (tb) {
    smem = words * h->td.max_len * tb * sizeof(TC);
  } else {
    tb = 128;
    vglob = reinterpret_cast<TC*>(h->vscratch);
    if (!vglob) return set_error(KKT_ERR_INVALID_ARG, "sweep scratch missing");
  }
  dim3 grid(static_cast<unsigned>((p.N + tb - 1) / tb), static_cast<unsigned>(p.n_sub));
  auto kern = sweep_kernel<TI, TC, TO>;
  if (smem > 0)
    KKT_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
  // per mode and subdomain node: residual update (8 flops) + forward and backward steps (4)
  const double visits = static_cast<double>(p.N) * (p.Nt + p.n_sub);
  ProfScope ps(KKT_K_SWEEP, st, 12.0 * visits, visits * sizeof(TI) + static_cast<double>(p.N) * p.Nt * sizeof(TO));
  kern<<<grid, tb, smem, st>>>(rhat, in_scale, yhat, yhat_lo, p, h->coarse_c, vglob, h->td.max_len);
  KKT_CUDA_TRY(cudaGetLastError());
  return KKT_OK;
}

}  // namespace

int spectral_schur_precond(const kkt_handle* h, const double* rhat, double* yhat, double in_scale,
                           cudaStream_t st) {
  SpecParams p = make_params(h, false);
  return launch_sweeps<double, double, double>(h, p, rhat, in_scale, yhat, st, false);
}

int spectral_schur_precond_mixed(const kkt_handle* h, const float* rhat, double in_scale, void* yhat, void* yhat_lo,
                                 int bf16, cudaStream_t st) {
  SpecParams p = make_params(h, true);
  if (bf16)
    return launch_sweeps<float, float, __nv_bfloat16>(h, p, rhat, in_scale, static_cast<__nv_bfloat16*>(yhat), st,
                                                      true, static_cast<__nv_bfloat16*>(yhat_lo));
  return launch_sweeps<float, float, float>(h, p, rhat, in_scale, static_cast<float*>(yhat), st, true,
                                            static_cast<float*>(yhat_lo));
}

int spectral_learned_apply(const kkt_handle* h, bool padded, const float* y, cudaStream_t st) {
  SpecParams p = make_params(h, padded);
  const int n = p.learn_k * p.learn_k;
  if (n == 0) return KKT_OK;
  ProfScope ps(KKT_K_COARSE, st, 40.0 * n * p.n_sub, 40.0 * n * p.n_sub);
  learned_apply_kernel<<<static_cast<unsigned>((32LL * n + 127) / 128), 128, 0, st>>>(p, y, h->mlp_mode, h->coarse_c,
                                                                                       h->learn_count);
  KKT_CUDA_TRY(cudaGetLastError());
  return KKT_OK;
}

SpecParams make_spec_params(const kkt_handle* h) { return make_params(h, false); }

int spectral_batched_prepare(BatchSlot& slot, const SpecJob* jobs, int nj) {
  if (nj < 1 || nj > KKT_BATCH_MAX) return set_error(KKT_ERR_INVALID_ARG, "batched jobs out of range");
  slot.njobs = nj;
  const int tb = slot.sweep_tb > 0 ? slot.sweep_tb : 128;
  // order by subdomain length; subdomains of at most kShort nodes form the first group
  constexpr int kShort = 40;
  std::vector<SpecJob> js(jobs, jobs + nj);
  std::stable_sort(js.begin(), js.end(), [](const SpecJob& a, const SpecJob& b) { return a.max_len < b.max_len; });
  jobs = js.data();
  std::vector<long long> cp(nj + 1, 0), sp(nj + 1, 0);
  int max_len = 0, short_len = 0, n_short = 0;
  double cf = 0, cb = 0, sf = 0, sb = 0;
  for (int k = 0; k < nj; ++k) {
    const SpecParams& p = jobs[k].p;
    if (jobs[k].max_len <= kShort) {
      short_len = std::max(short_len, jobs[k].max_len);
      n_short = k + 1;
    }
    cp[k + 1] = cp[k] + (p.two_level && !p.cyclic ? (p.N + 127) / 128 : 0);
    sp[k + 1] = sp[k] + ((p.N + tb - 1) / tb) * p.n_sub;
    max_len = std::max(max_len, jobs[k].max_len);
    const double V = static_cast<double>(p.N) * p.Nt, visits = static_cast<double>(p.N) * (p.Nt + p.n_sub);
    if (p.two_level) {
      cf += 2.0 * V + (p.cyclic ? (p.crf ? 40.0 : 80.0) : 26.0) * p.n_sub * p.N;
      cb += 8.0 * V + (p.cyclic ? (p.crf ? 168.0 : 16.0) : 12.0 * 8.0) * p.n_sub * p.N;
    }
    sf += 12.0 * visits;
    sb += 8.0 * visits + 8.0 * V;
  }
  int words = 1;
  for (int k = 0; k < nj; ++k) words = std::max(words, jobs[k].p.ras ? 2 : 1);
  if (static_cast<size_t>(words) * max_len * tb * sizeof(double) > 200 * 1024)
    return set_error(KKT_ERR_UNSUPPORTED, "batched sweeps: a subdomain is too long for shared memory");
  if (!slot.spec) {
    KKT_CUDA_TRY(cudaMalloc(&slot.spec, KKT_BATCH_MAX * sizeof(SpecJob)));
    KKT_CUDA_TRY(cudaMalloc(&slot.coarse_prefix, (KKT_BATCH_MAX + 1) * sizeof(long long)));
    KKT_CUDA_TRY(cudaMalloc(&slot.sweep_prefix, (KKT_BATCH_MAX + 1) * sizeof(long long)));
  }
  KKT_CUDA_TRY(cudaMemcpy(slot.spec, jobs, nj * sizeof(SpecJob), cudaMemcpyHostToDevice));
  // the instances whose coarse solve is the cyclic reduction, with their own item table
  std::vector<SpecJob> cr;
  std::vector<long long> crp(1, 0);
  size_t cr_smem = 0;
  for (int k = 0; k < nj; ++k) {
    const SpecParams& p = jobs[k].p;
    if (!p.two_level || !p.cyclic) continue;
    cr.push_back(jobs[k]);
    // the instances share the launch, so pack modes as densely as shared memory allows
    // (cr_modes_per_cta, within 96 KB for the elimination's 13 doubles per block) rather than
    // spreading one instance's modes over the SMs
    const int mpc = cr_modes_per_cta(p.n_sub);
    cr.back().p.cr_mpc = mpc;
    crp.push_back(crp.back() + (p.N + mpc - 1) / mpc);
    const size_t fields = p.crf ? 2 : kCrFields;
    cr_smem = std::max(cr_smem, fields * p.n_sub * mpc * sizeof(double));
  }
  slot.cr_njobs = static_cast<int>(cr.size());
  slot.cr_total = crp.back();
  slot.cr_smem = cr_smem;
  if (!cr.empty()) {
    if (!slot.spec_cr) {
      KKT_CUDA_TRY(cudaMalloc(&slot.spec_cr, KKT_BATCH_MAX * sizeof(SpecJob)));
      KKT_CUDA_TRY(cudaMalloc(&slot.cr_prefix, (KKT_BATCH_MAX + 1) * sizeof(long long)));
    }
    KKT_CUDA_TRY(cudaMemcpy(slot.spec_cr, cr.data(), cr.size() * sizeof(SpecJob), cudaMemcpyHostToDevice));
    KKT_CUDA_TRY(cudaMemcpy(slot.cr_prefix, crp.data(), crp.size() * sizeof(long long), cudaMemcpyHostToDevice));
  }
  KKT_CUDA_TRY(cudaMemcpy(slot.coarse_prefix, cp.data(), (nj + 1) * sizeof(long long), cudaMemcpyHostToDevice));
  KKT_CUDA_TRY(cudaMemcpy(slot.sweep_prefix, sp.data(), (nj + 1) * sizeof(long long), cudaMemcpyHostToDevice));
  slot.coarse_total = cp[nj];
  slot.sweep_total = sp[nj];
  slot.sweep_tb = tb;
  slot.sweep_smem = static_cast<size_t>(words) * max_len * tb * sizeof(double);
  slot.sweep_split = (n_short > 0 && n_short < nj) ? sp[n_short] : 0;
  slot.sweep_smem_short = static_cast<size_t>(words) * short_len * tb * sizeof(double);
  slot.coarse_flops = cf;
  slot.coarse_bytes = cb;
  slot.sweep_flops = sf;
  slot.sweep_bytes = sb;
  return KKT_OK;
}

int spectral_batched_launch(const BatchSlot& slot, const double* scale_dev, cudaStream_t st) {
  int dev = 0, sms = 0;
  KKT_CUDA_TRY(cudaGetDevice(&dev));
  KKT_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (slot.coarse_total > 0 || slot.cr_total > 0) {
    ProfScope ps(KKT_K_COARSE, st, slot.coarse_flops, slot.coarse_bytes);
    if (slot.coarse_total > 0) {
      const long long grid = std::min<long long>(slot.coarse_total, static_cast<long long>(sms) * 16);
      coarse_batched<<<static_cast<unsigned>(grid), 128, 0, st>>>(slot.spec, slot.coarse_prefix, slot.njobs,
                                                                  slot.coarse_total, scale_dev);
      KKT_CUDA_TRY(cudaGetLastError());
    }
    if (slot.cr_total > 0) {
      KKT_CUDA_TRY(cudaFuncSetAttribute(coarse_cr_batched, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        static_cast<int>(slot.cr_smem)));
      int per_sm = 0;
      KKT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, coarse_cr_batched, kCrThreads, slot.cr_smem));
      const long long grid = std::min<long long>(slot.cr_total, static_cast<long long>(sms) * std::max(per_sm, 1));
      coarse_cr_batched<<<static_cast<unsigned>(grid), kCrThreads, slot.cr_smem, st>>>(
          slot.spec_cr, slot.cr_prefix, slot.cr_njobs, slot.cr_total, scale_dev);
      KKT_CUDA_TRY(cudaGetLastError());
    }
  }
  if (slot.sweep_total > 0) {
    KKT_CUDA_TRY(cudaFuncSetAttribute(sweep_batched, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      static_cast<int>(slot.sweep_smem)));
    auto launch = [&](long long t0, long long t1, size_t smem) -> int {
      int per_sm = 0;
      KKT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_batched, slot.sweep_tb, smem));
      const long long grid = std::min<long long>(t1 - t0, static_cast<long long>(sms) * std::max(per_sm, 1));
      sweep_batched<<<static_cast<unsigned>(grid), slot.sweep_tb, smem, st>>>(slot.spec, slot.sweep_prefix,
                                                                            slot.njobs, t0, t1, scale_dev);
      KKT_CUDA_TRY(cudaGetLastError());
      return KKT_OK;
    };
    ProfScope ps(KKT_K_SWEEP, st, slot.sweep_flops, slot.sweep_bytes);
    if (slot.sweep_split > 0) {   // short subdomains, then long ones
      KKT_TRY(launch(0, slot.sweep_split, slot.sweep_smem_short));
      KKT_TRY(launch(slot.sweep_split, slot.sweep_total, slot.sweep_smem));
    } else {
      KKT_TRY(launch(0, slot.sweep_total, slot.sweep_smem));
    }
  }
  return KKT_OK;
}

int spectral_cr_factor(kkt_handle* h) {
  SpecParams p = make_params(h, false);
  const long long slots = cr_factor_slots(p.n_sub);
  const double bytes = static_cast<double>(slots) * p.N * sizeof(double);
  if (!p.cyclic || bytes > 2.0 * 1024 * 1024 * 1024) {
    if (h->cr_factors) {
      cudaFree(h->cr_factors);
      h->bytes -= h->cr_factor_bytes;
      h->cr_factors = nullptr;
      h->cr_factor_bytes = 0;
    }
    return KKT_OK;
  }
  if (h->cr_factor_bytes != static_cast<size_t>(bytes)) {
    if (h->cr_factors) {
      cudaFree(h->cr_factors);
      h->bytes -= h->cr_factor_bytes;
      h->cr_factors = nullptr;
      h->cr_factor_bytes = 0;
    }
    KKT_CUDA_TRY(cudaMalloc(&h->cr_factors, static_cast<size_t>(bytes)));
    h->cr_factor_bytes = static_cast<size_t>(bytes);
    h->bytes += static_cast<size_t>(bytes);
  }
  const int mpc = cr_modes_per_cta(p.n_sub);
  const size_t smem = 7 * static_cast<size_t>(p.n_sub) * mpc * sizeof(double);
  KKT_CUDA_TRY(cudaFuncSetAttribute(coarse_cr_factor_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    static_cast<int>(smem)));
  const long long nb = (p.N + mpc - 1) / mpc;
  // Legacy default stream: the caller (configure) synchronises the device before any solve can
  // read these factors on the caller's stream.
  coarse_cr_factor_kernel<<<static_cast<unsigned>(nb), kCrThreads, smem, nullptr>>>(p, mpc, h->cr_factors);
  KKT_CUDA_TRY(cudaGetLastError());
  return KKT_OK;
}

int spectral_coarse_factor(const kkt_handle* h, bool padded, double* cf, cudaStream_t st) {
  SpecParams p = make_params(h, padded);
  const int tb = 128;
  const long long nb = (p.N + tb - 1) / tb;
  coarse_factor_kernel<<<static_cast<unsigned>(nb), tb, 0, st>>>(p, cf);
  KKT_CUDA_TRY(cudaGetLastError());
  return KKT_OK;
}

int spectral_coarse_only(const kkt_handle* h, const double* rhat, double* xhat, cudaStream_t st) {
  SpecParams p = make_params(h, false);
  KKT_TRY(launch_coarse<double>(h, p, rhat, 1.0, st));
  const int tb = 128;
  dim3 grid(static_cast<unsigned>((p.N + tb - 1) / tb), static_cast<unsigned>(p.Nt));
  ProfScope ps(KKT_K_SWEEP, st);
  prolong_kernel<<<grid, tb, 0, st>>>(p, h->coarse_c, xhat);
  KKT_CUDA_TRY(cudaGetLastError());
  return KKT_OK;
}

}  // namespace kkt
