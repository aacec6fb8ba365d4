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

#include "kkt_internal.cuh"

namespace kkt {
namespace {

struct SpecParams {
  int Mx, Nt, n_sub;      // Mx: modes per spectral row (the padded size in the mixed forms)
  long long N;
  double a, dtnu, h;
  const double* lx;
  const double* ly;
  const int* first;
  const int* last;
  const int* ofirst;
  const int* olast;
  const int* owner;
  const double* phi;
  const double* mom;
  int two_level;       // apply the coarse correction
  int multiplicative;  // subtract S-hat x_0 before the local solves
};

__device__ __forceinline__ double mode_mu(const SpecParams& p, long long q) {
  const long long l = q / p.Mx;
  const int k = static_cast<int>(q - l * p.Mx);
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

template <typename TI>
__global__ void coarse_solve_kernel(const TI* __restrict__ rhat, double in_scale, SpecParams p,
                                    double* __restrict__ cc, double* __restrict__ cw) {
  const long long q = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= p.N) return;
  const long long N = p.N;
  const double mu = mode_mu(p, q), mu2 = mu * mu;
  double d00 = 0, d01 = 0, d11 = 0, y0 = 0, y1 = 0;   // previous D^{-1} and eliminated rhs
  double a1_prev = 0.0;                              // phi at the last owned node of s-1
  for (int s = 0; s < p.n_sub; ++s) {
    double c0 = 0.0, c1 = 0.0;
    const int o1 = __ldg(p.ofirst + s), o2 = __ldg(p.olast + s);
#pragma unroll 4
    for (int n = o1; n <= o2; ++n) {
      const double r = load_d(rhat + static_cast<long long>(n - 1) * N + q) * in_scale;
      c0 += r;
      c1 = fma(r, __ldg(p.phi + n - 1), c1);
    }
    const double* M = p.mom + 9 * s;
    double g00 = fma(mu2, M[0], M[3]) - mu * M[6];
    double g01 = fma(mu2, M[1], M[4]) - mu * M[7];
    double g11 = fma(mu2, M[2], M[5]) - mu * M[8];
    if (s > 0) {
      const double b1 = __ldg(p.phi + o1 - 1);
      // E = -mu a b^T, a = (1, a1_prev), b = (1, b1): D -= E^T Dinv E, y = c - E^T Dinv y_prev
      const double t0 = d00 + d01 * a1_prev, t1 = d01 + d11 * a1_prev;   // Dinv a
      const double aDa = t0 + t1 * a1_prev;
      const double aDy = t0 * y0 + t1 * y1;
      const double f = mu2 * aDa;
      g00 -= f;
      g01 -= f * b1;
      g11 -= f * b1 * b1;
      c0 += mu * aDy;
      c1 += mu * b1 * aDy;
    }
    const double det = g00 * g11 - g01 * g01;
    const double id = 1.0 / det;
    d00 = g11 * id;
    d01 = -g01 * id;
    d11 = g00 * id;
    y0 = c0;
    y1 = c1;
    double* W = cw + static_cast<long long>(s) * 5 * N + q;
    W[0] = d00;
    W[N] = d01;
    W[2 * N] = d11;
    W[3 * N] = y0;
    W[4 * N] = y1;
    a1_prev = __ldg(p.phi + o2 - 1);
  }
  // back substitution; c' = h * x (S_0 = G/h)
  double x0 = d00 * y0 + d01 * y1, x1 = d01 * y0 + d11 * y1;
  {
    const int s = p.n_sub - 1;
    cc[(2LL * s) * N + q] = p.h * x0;
    cc[(2LL * s + 1) * N + q] = p.h * x1;
  }
  for (int s = p.n_sub - 2; s >= 0; --s) {
    const double* W = cw + static_cast<long long>(s) * 5 * N + q;
    const double e00 = W[0], e01 = W[N], e11 = W[2 * N], r0 = W[3 * N], r1 = W[4 * N];
    const double a1 = __ldg(p.phi + __ldg(p.olast + s) - 1);
    const double b1 = __ldg(p.phi + __ldg(p.ofirst + s + 1) - 1);
    const double bx = x0 + b1 * x1;                      // b^T x_{s+1}
    const double z0 = r0 + mu * bx, z1 = r1 + mu * a1 * bx;   // y - E x_{s+1}
    x0 = e00 * z0 + e01 * z1;
    x1 = e01 * z0 + e11 * z1;
    cc[(2LL * s) * N + q] = p.h * x0;
    cc[(2LL * s + 1) * N + q] = p.h * x1;
  }
}

// x_0 at node n (1-based), given the coarse pairs of the three subdomains around s.
__device__ __forceinline__ double coarse_value(const SpecParams& p, int n, int s, const double* c3) {
  if (n < 1 || n > p.Nt) return 0.0;
  const int o = __ldg(p.owner + n - 1) - s + 1;        // 0, 1, 2 for s-1, s, s+1
  if (o < 0 || o > 2) return 0.0;                       // cannot happen when every m_s >= 2
  return c3[2 * o] + c3[2 * o + 1] * __ldg(p.phi + n - 1);
}

template <typename TI, typename TC, typename TO>
__global__ void sweep_kernel(const TI* __restrict__ rhat, double in_scale, TO* __restrict__ yhat,
                             SpecParams p, const double* __restrict__ cc, TC* __restrict__ vglobal,
                             int max_len) {
  extern __shared__ __align__(16) unsigned char vs_raw[];
  TC* vs_smem = reinterpret_cast<TC*>(vs_raw);
  const long long q = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int s = blockIdx.y;
  if (q >= p.N) return;
  const long long N = p.N;
  const double mu = mode_mu(p, q), mu2 = mu * mu;
  const TC inv_mu = static_cast<TC>(1.0 / mu);
  const TC hc = static_cast<TC>(p.h);
  const int first = __ldg(p.first + s), last = __ldg(p.last + s);
  const int o1 = __ldg(p.ofirst + s), o2 = __ldg(p.olast + s);
  TC* vs;
  long long vstride;
  if (vglobal) {
    vs = vglobal + static_cast<long long>(s) * max_len * N + q;
    vstride = N;
  } else {
    vs = vs_smem + threadIdx.x;
    vstride = blockDim.x;
  }
  double c3[6] = {0, 0, 0, 0, 0, 0};
  if (p.two_level) {
    for (int o = 0; o < 3; ++o) {
      const int so = s - 1 + o;
      if (so >= 0 && so < p.n_sub) {
        c3[2 * o] = cc[(2LL * so) * N + q];
        c3[2 * o + 1] = cc[(2LL * so + 1) * N + q];
      }
    }
  }
  // forward sweep over the subdomain's nodes
  double xm = 0.0, xc = 0.0, xp = 0.0;   // x_0 at n-1, n, n+1
  if (p.two_level) {
    xm = coarse_value(p, first - 1, s, c3);
    xc = coarse_value(p, first, s, c3);
  }
  TC v = 0;
  for (int n = first; n <= last; ++n) {
    double r = load_d(rhat + static_cast<long long>(n - 1) * N + q) * in_scale;
    if (p.two_level) {
      xp = coarse_value(p, n + 1, s, c3);
      if (p.multiplicative) {
        const double tx = (n >= 2 ? mu2 + 1.0 : mu2) * xc - mu * (xm + xp);
        r -= tx / p.h;
      }
      xm = xc;
      xc = xp;
    }
    v = (static_cast<TC>(r) + v) * inv_mu;
    vs[static_cast<long long>(n - first) * vstride] = v;
  }
  // backward sweep; keep owned nodes
  TC y = 0;
  for (int n = last; n >= first; --n) {
    y = fma(hc, vs[static_cast<long long>(n - first) * vstride], y) * inv_mu;
    if (n >= o1 && n <= o2) {
      double out = static_cast<double>(y);
      if (p.two_level) out += coarse_value(p, n, s, c3);
      yhat[static_cast<long long>(n - 1) * N + q] = store_cast<TO>(out);
    }
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

SpecParams make_params(const kkt_handle* h, bool padded) {
  SpecParams p;
  const Geometry& g = h->g;
  p.Mx = padded ? h->tc.P : g.Mx;
  p.Nt = g.Nt;
  p.n_sub = g.n_sub;
  p.N = padded ? static_cast<long long>(h->tc.P) * h->tc.P : g.N;
  p.a = g.a;
  p.dtnu = g.dtnu;
  p.h = g.h;
  p.lx = padded ? h->d_lx_pad : h->d_lx;
  p.ly = padded ? h->d_ly_pad : h->d_ly;
  p.first = h->dd.first;
  p.last = h->dd.last;
  p.ofirst = h->dd.ofirst;
  p.olast = h->dd.olast;
  p.owner = h->dd.owner;
  p.phi = h->dd.phi;
  p.mom = h->dd.moments;
  p.two_level = h->opt.coarse == KKT_COARSE_EXACT;
  p.multiplicative = h->opt.variant == KKT_MULTIPLICATIVE;
  return p;
}

template <typename TI>
int launch_coarse(const kkt_handle* h, const SpecParams& p, const TI* rhat, double in_scale, cudaStream_t st) {
  const int tb = 128;
  const long long nb = (p.N + tb - 1) / tb;
  ProfScope ps(KKT_K_COARSE, st);
  coarse_solve_kernel<TI><<<static_cast<unsigned>(nb), tb, 0, st>>>(rhat, in_scale, p, h->coarse_c, h->coarse_w);
  KKT_CUDA_TRY(cudaGetLastError());
  return KKT_OK;
}

template <typename TI, typename TC, typename TO>
int launch_sweeps(const kkt_handle* h, const SpecParams& p, const TI* rhat, double in_scale, TO* yhat,
                  cudaStream_t st) {
  if (static_cast<const void*>(rhat) == static_cast<const void*>(yhat))
    return set_error(KKT_ERR_INVALID_ARG, "spectral sweep needs distinct buffers");
  if (p.two_level) KKT_TRY(launch_coarse<TI>(h, p, rhat, in_scale, st));
  // sweep storage: shared memory when a subdomain's nodes fit, else the global scratch
  const size_t limit = 200 * 1024;
  int tb = 0;
  for (int cand : {128, 64, 32})
    if (static_cast<size_t>(h->td.max_len) * cand * sizeof(TC) <= limit) {
      tb = cand;
      break;
    }
  size_t smem = 0;
  TC* vglob = nullptr;
  if (tb) {
    smem = static_cast<size_t>(h->td.max_len) * tb * sizeof(TC);
  } else {
    tb = 128;
    vglob = reinterpret_cast<TC*>(h->vscratch);
    if (!vglob) return set_error(KKT_ERR_INVALID_ARG, "sweep scratch missing");
  }
  dim3 grid(static_cast<unsigned>((p.N + tb - 1) / tb), static_cast<unsigned>(p.n_sub));
  auto kern = sweep_kernel<TI, TC, TO>;
  if (smem > 0)
    KKT_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
  ProfScope ps(KKT_K_SWEEP, st);
  kern<<<grid, tb, smem, st>>>(rhat, in_scale, yhat, p, h->coarse_c, vglob, h->td.max_len);
  KKT_CUDA_TRY(cudaGetLastError());
  return KKT_OK;
}

}  // namespace

int spectral_schur_precond(const kkt_handle* h, const double* rhat, double* yhat, double in_scale,
                           cudaStream_t st) {
  SpecParams p = make_params(h, false);
  return launch_sweeps<double, double, double>(h, p, rhat, in_scale, yhat, st);
}

int spectral_schur_precond_mixed(const kkt_handle* h, const float* rhat, void* yhat, int bf16, cudaStream_t st) {
  SpecParams p = make_params(h, true);
  if (bf16) return launch_sweeps<float, float, __nv_bfloat16>(h, p, rhat, 1.0, static_cast<__nv_bfloat16*>(yhat), st);
  return launch_sweeps<float, float, float>(h, p, rhat, 1.0, static_cast<float*>(yhat), st);
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
