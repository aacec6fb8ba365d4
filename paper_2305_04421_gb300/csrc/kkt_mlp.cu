// Learned coarse correction (not in the paper): a two-hidden-layer ReLU perceptron that maps a
// low sine mode's normalised coarse right-hand side R_0 r (Eq 14) and two features of the mode
// (log dt nu lambda, log dt / sqrt(omega)) to the direction of its coarse correction
// S_0^{-1} R_0 r. The magnitude along that direction comes from an exact one-dimensional
// minimal-residual step with the mode's coarse operator, so the correction never increases the
// coarse residual; a residual guard falls back to the exact coarse solve, which stays the
// reference the learned correction is measured against.
// FGMRES admits the resulting preconditioner because it tolerates a variable one.
//
// Training runs on the GPU with the kernels of this file: the coarse right-hand sides come
// from the method's restriction of seeded residual time series, the targets from the method's
// exact block-Thomas coarse solve. The network is fitted with Adam in two phases: first on the
// mean squared error to the unit target (a smooth start), then on the quantity the guard tests,
// the squared relative coarse residual ||c - alpha G d||^2 / ||c||^2 after the minimal-residual
// step (G = h S_0(mu) of the sample's mode), which weights the error of d by the coarse operator. All products are tiled FP32 CUDA-core GEMMs (the network is
// about 1.6 MFLOP per mode, far below any tensor-core bound); inference reads BF16 weights
// and accumulates in FP32.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
#include <vector>

#include "kkt_internal.cuh"

namespace kkt {
namespace {

// ---- GEMM: C[M x N] = op(A) op(B) (+ bias[n]) (relu), FP32 accumulate -------------------
// opA: 0 -> A[m][k] = A[m * lda + k], 1 -> A[m][k] = A[k * lda + m]
// opB: 0 -> B[k][n] = B[n * ldb + k] (B stored [N][K]), 1 -> B[k][n] = B[k * ldb + n]
constexpr int kBM = 64, kBN = 64, kBK = 16;

template <int OPA, int OPB, typename TB>
__global__ void __launch_bounds__(256) sgemm_kernel(int M, int N, int K, const float* __restrict__ A, int lda,
                                                    const TB* __restrict__ B, int ldb, const float* __restrict__ bias,
                                                    int relu, float* __restrict__ C, int ldc) {
  __shared__ float As[kBK][kBM + 4];
  __shared__ float Bs[kBK][kBN + 4];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * kBN;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += kBK) {
    for (int e = threadIdx.x; e < kBK * kBM; e += 256) {
      const int kk = OPA == 0 ? e % kBK : e / kBM;
      const int mm = OPA == 0 ? e / kBK : e % kBM;
      const int m = m0 + mm, k = k0 + kk;
      float v = 0.f;
      if (m < M && k < K) v = OPA == 0 ? A[static_cast<long long>(m) * lda + k] : A[static_cast<long long>(k) * lda + m];
      As[kk][mm] = v;
    }
    for (int e = threadIdx.x; e < kBK * kBN; e += 256) {
      const int kk = OPB == 0 ? e % kBK : e / kBN;
      const int nn = OPB == 0 ? e / kBK : e % kBN;
      const int n = n0 + nn, k = k0 + kk;
      float v = 0.f;
      if (n < N && k < K)
        v = static_cast<float>(OPB == 0 ? B[static_cast<long long>(n) * ldb + k] : B[static_cast<long long>(k) * ldb + n]);
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kBK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty * 4 + i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx * 4 + j;
      if (n >= N) continue;
      float v = acc[i][j];
      if (bias) v += bias[n];
      if (relu) v = fmaxf(v, 0.f);
      C[static_cast<long long>(m) * ldc + n] = v;
    }
  }
}

template <int OPA, int OPB, typename TB>
int gemm(int M, int N, int K, const float* A, int lda, const TB* B, int ldb, const float* bias, int relu, float* C,
         int ldc, cudaStream_t st) {
  dim3 grid((N + kBN - 1) / kBN, (M + kBM - 1) / kBM);
  ProfScope ps(KKT_K_MATVEC, st, 2.0 * M * N * K, 4.0 * (static_cast<double>(M) * K + static_cast<double>(N) * K + static_cast<double>(M) * N));
  sgemm_kernel<OPA, OPB, TB><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, bias, relu, C, ldc);
  KKT_CUDA_TRY(cudaGetLastError());
  return KKT_OK;
}

// dY = (Y - T) / B, partial sums of the squared error per block
__global__ void mse_grad_kernel(const float* __restrict__ Y, const float* __restrict__ T, float* __restrict__ dY,
                                long long n, float invB, double* __restrict__ part) {
  __shared__ double sh[256];
  double acc = 0.0;
  for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n; i += 256LL * gridDim.x) {
    const float d = Y[i] - T[i];
    dY[i] = d * invB;
    acc += static_cast<double>(d) * d;
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// dH *= (A > 0): back through the ReLU, A the pre-activation (here the activation itself)
__global__ void relu_back_kernel(float* __restrict__ dH, const float* __restrict__ H, long long n) {
  for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n; i += 256LL * gridDim.x)
    if (!(H[i] > 0.f)) dH[i] = 0.f;
}

// db[j] = sum_b dY[b][j]
__global__ void colsum_kernel(const float* __restrict__ dY, int B, int N, float* __restrict__ db) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  float s = 0.f;
  for (int b = 0; b < B; ++b) s += dY[static_cast<long long>(b) * N + j];
  db[j] = s;
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, long long n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
  for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n; i += 256LL * gridDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

__global__ void to_bf16_kernel(const float* __restrict__ x, __nv_bfloat16* __restrict__ y, long long n) {
  for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n; i += 256LL * gridDim.x) y[i] = __float2bfloat16_rn(x[i]);
}

unsigned grid_for(long long n) { return static_cast<unsigned>(std::min<long long>((n + 255) / 256, 4096)); }

// ---- coarse data for training: restriction + exact block-Thomas solve per sample ---------
struct DecompView {
  int n_sub, Nt;
  const int* ofirst;
  const int* olast;
  const double* phi;
  const double* mom;
};

// c = R_0 r for a time series r[n * S + i] (n = 0..Nt-1), x = (h S_0)^{-1} c with h S_0 the
// per-mode coarse operator for diagonal mu; per sample, D^{-1} and eliminated right-hand sides
// go to the scratch w[i][s][5].
__global__ void coarse_data_kernel(const double* __restrict__ r, const double* __restrict__ mu_arr, long long S,
                                   DecompView d, double* __restrict__ c_out, double* __restrict__ x_out,
                                   double* __restrict__ w) {
  const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (i >= S) return;
  const double mu = mu_arr[i], mu2 = mu * mu;
  double d00 = 0, d01 = 0, d11 = 0, y0 = 0, y1 = 0, a1_prev = 0;
  double* W = w + i * 5LL * d.n_sub;
  double* C = c_out + i * 2LL * d.n_sub;
  for (int s = 0; s < d.n_sub; ++s) {
    double c0 = 0, c1 = 0;
    for (int n = d.ofirst[s]; n <= d.olast[s]; ++n) {
      const double v = r[static_cast<long long>(n - 1) * S + i];
      c0 += v;
      c1 = fma(v, d.phi[n - 1], c1);
    }
    C[2 * s] = c0;
    C[2 * s + 1] = c1;
    const double* M = d.mom + 9 * s;
    double g00 = fma(mu2, M[0], M[3]) - mu * M[6];
    double g01 = fma(mu2, M[1], M[4]) - mu * M[7];
    double g11 = fma(mu2, M[2], M[5]) - mu * M[8];
    if (s > 0) {
      const double b1 = d.phi[d.ofirst[s] - 1];
      const double t0 = d00 + d01 * a1_prev, t1 = d01 + d11 * a1_prev;
      const double aDy = t0 * y0 + t1 * y1;
      const double f = mu2 * (t0 + t1 * a1_prev);
      g00 -= f;
      g01 -= f * b1;
      g11 -= f * b1 * b1;
      c0 += mu * aDy;
      c1 += mu * b1 * aDy;
    }
    const double id = 1.0 / (g00 * g11 - g01 * g01);
    d00 = g11 * id;
    d01 = -g01 * id;
    d11 = g00 * id;
    y0 = c0;
    y1 = c1;
    W[5 * s + 0] = d00;
    W[5 * s + 1] = d01;
    W[5 * s + 2] = d11;
    W[5 * s + 3] = y0;
    W[5 * s + 4] = y1;
    a1_prev = d.phi[d.olast[s] - 1];
  }
  double x0 = 0, x1 = 0;
  double* X = x_out + i * 2LL * d.n_sub;
  for (int s = d.n_sub - 1; s >= 0; --s) {
    double z0 = W[5 * s + 3], z1 = W[5 * s + 4];
    if (s + 1 < d.n_sub) {
      const double a1 = d.phi[d.olast[s] - 1];
      const double b1 = d.phi[d.ofirst[s + 1] - 1];
      const double bx = x0 + b1 * x1;
      z0 += mu * bx;
      z1 += mu * a1 * bx;
    }
    x0 = W[5 * s] * z0 + W[5 * s + 1] * z1;
    x1 = W[5 * s + 1] * z0 + W[5 * s + 2] * z1;
    X[2 * s] = x0;
    X[2 * s + 1] = x1;
  }
}

// network input [c / ||c||, f1, f2] and unit target x / ||x|| in FP32, one warp per sample
__global__ void make_xy_kernel(const double* __restrict__ c, const double* __restrict__ x,
                               const double* __restrict__ feat, long long S, int nc, float* __restrict__ X,
                               float* __restrict__ T) {
  const long long i = (blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= S) return;
  double sc = 0, sx = 0;
  for (int j = lane; j < nc; j += 32) {
    sc += c[i * nc + j] * c[i * nc + j];
    if (x) sx += x[i * nc + j] * x[i * nc + j];
  }
  for (int o = 16; o > 0; o >>= 1) {
    sc += __shfl_xor_sync(0xffffffffu, sc, o);
    sx += __shfl_xor_sync(0xffffffffu, sx, o);
  }
  const double ic = sc > 0 ? 1.0 / sqrt(sc) : 0.0, ix = sx > 0 ? 1.0 / sqrt(sx) : 0.0;
  for (int j = lane; j < nc; j += 32) {
    X[i * (nc + 2) + j] = static_cast<float>(c[i * nc + j] * ic);
    if (x) T[i * nc + j] = static_cast<float>(x[i * nc + j] * ix);
  }
  if (lane == 0) {
    X[i * (nc + 2) + nc] = static_cast<float>(feat[2 * i]);
    X[i * (nc + 2) + nc + 1] = static_cast<float>(feat[2 * i + 1]);
  }
}

// The decomposition of the training geometry as the coarse-operator helper reads it.
struct MlpDecomp {
  int n_sub;
  const int* ofirst;
  const int* olast;
  const double* phi;
  const double* mom;
};

// Coarse-residual loss of a batch, one warp per sample b: d = Y row b, c = the first nc entries
// of X row b (the normalised coarse right-hand side), G = G(mu_b):
//   g = G d, alpha = g^T c / g^T g, r = c - alpha g, loss_b = r^T r / c^T c,
//   dY_b = dloss_b/dd / B = -2 alpha G r / (c^T c B).
// Lanes stride over the subdomains; r is staged in scratch[b][nc] so that every lane can read
// its neighbours' pairs for G r (after __syncwarp, which orders the warp's memory accesses).
__global__ void resid_grad_kernel(const float* __restrict__ Y, const float* __restrict__ X, int ldx,
                                  const double* __restrict__ mu_arr, int B, int nc, MlpDecomp dd,
                                  double* __restrict__ scratch, float* __restrict__ dY, float invB,
                                  double* __restrict__ loss) {
  const int b = static_cast<int>((static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (b >= B) return;   // uniform per warp
  const float* d = Y + static_cast<long long>(b) * nc;
  const float* c = X + static_cast<long long>(b) * ldx;
  double* R = scratch + static_cast<long long>(b) * nc;
  const double mu = mu_arr[b], mu2 = mu * mu;
  double gg = 0, gc = 0, cc = 0;
  for (int s = lane; s < dd.n_sub; s += 32) {
    double e0, e1;
    coarse_op_apply_row(dd.mom, dd.phi, dd.ofirst, dd.olast, dd.n_sub, mu, mu2, d, s, e0, e1);
    const double c0 = c[2 * s], c1 = c[2 * s + 1];
    gg += e0 * e0 + e1 * e1;
    gc += e0 * c0 + e1 * c1;
    cc += c0 * c0 + c1 * c1;
  }
  for (int o = 16; o > 0; o >>= 1) {
    gg += __shfl_xor_sync(0xffffffffu, gg, o);
    gc += __shfl_xor_sync(0xffffffffu, gc, o);
    cc += __shfl_xor_sync(0xffffffffu, cc, o);
  }
  if (!(gg > 0.0) || !(cc > 0.0)) {   // d = 0 (or c = 0): loss 1, no gradient
    if (dY)
      for (int j = lane; j < nc; j += 32) dY[static_cast<long long>(b) * nc + j] = 0.f;
    if (lane == 0) loss[b] = 1.0;
    return;
  }
  const double alpha = gc / gg;
  double rr = 0;
  for (int s = lane; s < dd.n_sub; s += 32) {
    double e0, e1;
    coarse_op_apply_row(dd.mom, dd.phi, dd.ofirst, dd.olast, dd.n_sub, mu, mu2, d, s, e0, e1);
    const double r0 = c[2 * s] - alpha * e0, r1 = c[2 * s + 1] - alpha * e1;
    R[2 * s] = r0;
    R[2 * s + 1] = r1;
    rr += r0 * r0 + r1 * r1;
  }
  for (int o = 16; o > 0; o >>= 1) rr += __shfl_xor_sync(0xffffffffu, rr, o);
  if (lane == 0) loss[b] = rr / cc;
  if (!dY) return;
  __syncwarp();
  const double sc = -2.0 * alpha / cc * invB;
  for (int s = lane; s < dd.n_sub; s += 32) {
    double e0, e1;
    coarse_op_apply_row(dd.mom, dd.phi, dd.ofirst, dd.olast, dd.n_sub, mu, mu2, R, s, e0, e1);
    dY[static_cast<long long>(b) * nc + 2 * s] = static_cast<float>(sc * e0);
    dY[static_cast<long long>(b) * nc + 2 * s + 1] = static_cast<float>(sc * e1);
  }
}

}  // namespace
}  // namespace kkt

struct kkt_mlp {
  kkt_mlp_config cfg;
  int d_in = 0, H = 0, d_out = 0;
  long long nparam = 0;
  float* p = nullptr;        // FP32 master parameters: W1 b1 W2 b2 W3 b3
  __nv_bfloat16* pb = nullptr;  // BF16 copy used by inference
  float* g = nullptr;        // gradients (same layout)
  float* m = nullptr;        // Adam moments
  float* v = nullptr;
  int t = 0;                 // Adam step count
  int max_batch = 0;
  float* a1 = nullptr;       // activations [max_batch][H]
  float* a2 = nullptr;
  float* y = nullptr;        // [max_batch][d_out]
  float* dy = nullptr;
  float* dh2 = nullptr;
  float* dh1 = nullptr;
  double* part = nullptr;
  float lr = 1e-3f;
  // the training geometry's time decomposition (left partition of unity): owned node ranges
  // [2 n_sub] and phi [Nt] + moments [9 n_sub]
  int* dof = nullptr;
  double* dtab = nullptr;
  double* rscratch = nullptr;  // coarse-residual loss: r per sample [max_batch][2 n_sub]
  double* lossv = nullptr;     // per-sample loss [max_batch]
};

namespace kkt {
namespace {

struct ParamView {
  float *W1, *b1, *W2, *b2, *W3, *b3;
};

ParamView view(float* base, const kkt_mlp* m) {
  ParamView v;
  v.W1 = base;
  v.b1 = v.W1 + static_cast<long long>(m->H) * m->d_in;
  v.W2 = v.b1 + m->H;
  v.b2 = v.W2 + static_cast<long long>(m->H) * m->H;
  v.W3 = v.b2 + m->H;
  v.b3 = v.W3 + static_cast<long long>(m->d_out) * m->H;
  return v;
}

int ensure_batch(kkt_mlp* m, int B) {
  if (B <= m->max_batch) return KKT_OK;
  cudaFree(m->a1);
  cudaFree(m->a2);
  cudaFree(m->y);
  cudaFree(m->dy);
  cudaFree(m->dh2);
  cudaFree(m->dh1);
  cudaFree(m->rscratch);
  cudaFree(m->lossv);
  m->rscratch = nullptr;
  m->lossv = nullptr;
  const size_t h = static_cast<size_t>(B) * m->H, o = static_cast<size_t>(B) * m->d_out;
  KKT_CUDA_TRY(cudaMalloc(&m->a1, h * 4));
  KKT_CUDA_TRY(cudaMalloc(&m->a2, h * 4));
  KKT_CUDA_TRY(cudaMalloc(&m->y, o * 4));
  KKT_CUDA_TRY(cudaMalloc(&m->dy, o * 4));
  KKT_CUDA_TRY(cudaMalloc(&m->dh2, h * 4));
  KKT_CUDA_TRY(cudaMalloc(&m->dh1, h * 4));
  KKT_CUDA_TRY(cudaMalloc(&m->rscratch, o * sizeof(double)));
  KKT_CUDA_TRY(cudaMalloc(&m->lossv, static_cast<size_t>(B) * sizeof(double)));
  m->max_batch = B;
  return KKT_OK;
}

}  // namespace

// forward pass: X [B][d_in] -> m->y [B][d_out]; bf16 weights if use_bf16
int mlp_forward(kkt_mlp* m, const float* X, int B, int use_bf16, cudaStream_t st) {
  KKT_TRY(ensure_batch(m, B));
  const ParamView P = view(m->p, m);
  if (use_bf16) {
    const __nv_bfloat16* W1 = m->pb;
    const __nv_bfloat16* W2 = W1 + static_cast<long long>(m->H) * m->d_in + m->H;
    const __nv_bfloat16* W3 = W2 + static_cast<long long>(m->H) * m->H + m->H;
    KKT_TRY((gemm<0, 0, __nv_bfloat16>(B, m->H, m->d_in, X, m->d_in, W1, m->d_in, P.b1, 1, m->a1, m->H, st)));
    KKT_TRY((gemm<0, 0, __nv_bfloat16>(B, m->H, m->H, m->a1, m->H, W2, m->H, P.b2, 1, m->a2, m->H, st)));
    KKT_TRY((gemm<0, 0, __nv_bfloat16>(B, m->d_out, m->H, m->a2, m->H, W3, m->H, P.b3, 0, m->y, m->d_out, st)));
  } else {
    KKT_TRY((gemm<0, 0, float>(B, m->H, m->d_in, X, m->d_in, P.W1, m->d_in, P.b1, 1, m->a1, m->H, st)));
    KKT_TRY((gemm<0, 0, float>(B, m->H, m->H, m->a1, m->H, P.W2, m->H, P.b2, 1, m->a2, m->H, st)));
    KKT_TRY((gemm<0, 0, float>(B, m->d_out, m->H, m->a2, m->H, P.W3, m->H, P.b3, 0, m->y, m->d_out, st)));
  }
  return KKT_OK;
}

// Back-propagation from m->dy (= dloss/dY of the last forward pass on X) into m->g.
int mlp_backward(kkt_mlp* m, const float* X, int B, cudaStream_t st) {
  const ParamView P = view(m->p, m), G = view(m->g, m);
  const long long nh = static_cast<long long>(B) * m->H;
  // layer 3: dW3 = dY^T h2, db3 = colsum dY, dh2 = dY W3 masked
  KKT_TRY((gemm<1, 1, float>(m->d_out, m->H, B, m->dy, m->d_out, m->a2, m->H, nullptr, 0, G.W3, m->H, st)));
  colsum_kernel<<<(m->d_out + 127) / 128, 128, 0, st>>>(m->dy, B, m->d_out, G.b3);
  KKT_TRY((gemm<0, 1, float>(B, m->H, m->d_out, m->dy, m->d_out, P.W3, m->H, nullptr, 0, m->dh2, m->H, st)));
  relu_back_kernel<<<grid_for(nh), 256, 0, st>>>(m->dh2, m->a2, nh);
  // layer 2
  KKT_TRY((gemm<1, 1, float>(m->H, m->H, B, m->dh2, m->H, m->a1, m->H, nullptr, 0, G.W2, m->H, st)));
  colsum_kernel<<<(m->H + 127) / 128, 128, 0, st>>>(m->dh2, B, m->H, G.b2);
  KKT_TRY((gemm<0, 1, float>(B, m->H, m->H, m->dh2, m->H, P.W2, m->H, nullptr, 0, m->dh1, m->H, st)));
  relu_back_kernel<<<grid_for(nh), 256, 0, st>>>(m->dh1, m->a1, nh);
  // layer 1
  KKT_TRY((gemm<1, 1, float>(m->H, m->d_in, B, m->dh1, m->H, X, m->d_in, nullptr, 0, G.W1, m->d_in, st)));
  colsum_kernel<<<(m->H + 127) / 128, 128, 0, st>>>(m->dh1, B, m->H, G.b1);
  KKT_CUDA_TRY(cudaGetLastError());
  return KKT_OK;
}

// loss and gradients (FP32 weights) into m->g; returns the loss through *loss (synchronises)
int mlp_loss_grad(kkt_mlp* m, const float* X, const float* T, int B, double* loss, cudaStream_t st) {
  KKT_TRY(mlp_forward(m, X, B, 0, st));
  const long long no = static_cast<long long>(B) * m->d_out;
  const unsigned gb = grid_for(no);
  mse_grad_kernel<<<gb, 256, 0, st>>>(m->y, T, m->dy, no, 1.f / B, m->part);
  KKT_CUDA_TRY(cudaGetLastError());
  KKT_TRY(mlp_backward(m, X, B, st));
  if (loss) {
    std::vector<double> part(gb);
    KKT_CUDA_TRY(cudaMemcpyAsync(part.data(), m->part, gb * sizeof(double), cudaMemcpyDeviceToHost, st));
    KKT_CUDA_TRY(cudaStreamSynchronize(st));
    double s = 0;
    for (double v : part) s += v;
    *loss = 0.5 * s / B;
  }
  return KKT_OK;
}

MlpDecomp mlp_decomp(const kkt_mlp* m) {
  const int ns = m->cfg.n_sub;
  return MlpDecomp{ns, m->dof, m->dof + ns, m->dtab, m->dtab + m->cfg.Nt};
}

// Coarse-residual loss of the network output Y for inputs X (rows of d_in, the first 2 n_sub
// the normalised coarse right-hand side) and per-sample mu; with grad: dY into m->dy. *loss
// (the batch mean) is written after synchronising st when loss != nullptr; per-sample values
// stay in m->lossv.
int mlp_resid_eval(kkt_mlp* m, const float* Y, const float* X, const double* mu, int B, bool grad, double* loss,
                   cudaStream_t st) {
  KKT_TRY(ensure_batch(m, B));
  const int nc = m->d_out;
  resid_grad_kernel<<<static_cast<unsigned>((32LL * B + 127) / 128), 128, 0, st>>>(
      Y, X, m->d_in, mu, B, nc, mlp_decomp(m), m->rscratch, grad ? m->dy : nullptr, 1.f / B, m->lossv);
  KKT_CUDA_TRY(cudaGetLastError());
  if (loss) {
    std::vector<double> lv(B);
    KKT_CUDA_TRY(cudaMemcpyAsync(lv.data(), m->lossv, B * sizeof(double), cudaMemcpyDeviceToHost, st));
    KKT_CUDA_TRY(cudaStreamSynchronize(st));
    double s = 0;
    for (double v : lv) s += v;
    *loss = s / B;
  }
  return KKT_OK;
}

int mlp_resid_loss_grad(kkt_mlp* m, const float* X, const double* mu, int B, double* loss, cudaStream_t st) {
  KKT_TRY(mlp_forward(m, X, B, 0, st));
  KKT_TRY(mlp_resid_eval(m, m->y, X, mu, B, true, nullptr, st));
  KKT_TRY(mlp_backward(m, X, B, st));
  if (loss) {
    std::vector<double> lv(B);
    KKT_CUDA_TRY(cudaMemcpyAsync(lv.data(), m->lossv, B * sizeof(double), cudaMemcpyDeviceToHost, st));
    KKT_CUDA_TRY(cudaStreamSynchronize(st));
    double s = 0;
    for (double v : lv) s += v;
    *loss = s / B;
  }
  return KKT_OK;
}

int mlp_adam(kkt_mlp* m, float lr, cudaStream_t st) {
  m->t += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - std::pow(b1, static_cast<float>(m->t)), c2 = 1.f - std::pow(b2, static_cast<float>(m->t));
  ProfScope ps(KKT_K_AXPY, st, 10.0 * m->nparam, 20.0 * m->nparam);
  adam_kernel<<<grid_for(m->nparam), 256, 0, st>>>(m->p, m->g, m->m, m->v, m->nparam, lr, b1, b2, 1e-8f, c1, c2);
  KKT_CUDA_TRY(cudaGetLastError());
  return KKT_OK;
}

int mlp_refresh_bf16(kkt_mlp* m, cudaStream_t st) {
  to_bf16_kernel<<<grid_for(m->nparam), 256, 0, st>>>(m->p, m->pb, m->nparam);
  KKT_CUDA_TRY(cudaGetLastError());
  return KKT_OK;
}

int mlp_dims(const kkt_mlp* m, int* d_in, int* width, int* d_out) {
  *d_in = m->d_in;
  *width = m->H;
  *d_out = m->d_out;
  return KKT_OK;
}

const float* mlp_output(const kkt_mlp* m) { return m->y; }
const kkt_mlp_config& mlp_config(const kkt_mlp* m) { return m->cfg; }

int mlp_make_input(const double* c, const double* feat, long long S, int nc, float* X, cudaStream_t st) {
  const long long threads = S * 32;
  make_xy_kernel<<<static_cast<unsigned>((threads + 255) / 256), 256, 0, st>>>(c, nullptr, feat, S, nc, X, nullptr);
  KKT_CUDA_TRY(cudaGetLastError());
  return KKT_OK;
}

// The training geometry's time decomposition (balanced split, left partition of unity, the
// linear coarse function -1 + 2 (n - lo) / m_s on each subdomain's owned nodes, and the moment
// matrices of (1, phi) the coarse operator's blocks are built from), uploaded to m->dof / m->dtab.
int mlp_upload_decomp(kkt_mlp* m) {
  const kkt_mlp_config& c = m->cfg;
  std::vector<int> of(2 * c.n_sub);
  std::vector<double> tab(c.Nt + 9 * c.n_sub, 0.0);
  for (int s = 0; s < c.n_sub; ++s) {
    const int lo = static_cast<int>(static_cast<long long>(s) * c.Nt / c.n_sub);
    const int hi = static_cast<int>(static_cast<long long>(s + 1) * c.Nt / c.n_sub), m_s = hi - lo;
    of[s] = lo + 1;
    of[c.n_sub + s] = hi;
    double p0[3] = {0, 0, 0}, p1[3] = {0, 0, 0}, p2[3] = {0, 0, 0};
    for (int n = lo + 1; n <= hi; ++n) {
      const double ph = -1.0 + 2.0 * (n - lo) / m_s;
      tab[n - 1] = ph;
      p0[0] += 1;
      p0[1] += ph;
      p0[2] += ph * ph;
      if (n >= 2) {
        p1[0] += 1;
        p1[1] += ph;
        p1[2] += ph * ph;
      }
      if (n + 1 <= hi) {
        const double pn = -1.0 + 2.0 * (n + 1 - lo) / m_s;
        p2[0] += 2;
        p2[1] += ph + pn;
        p2[2] += 2 * ph * pn;
      }
    }
    for (int t = 0; t < 3; ++t) {
      tab[c.Nt + 9 * s + t] = p0[t];
      tab[c.Nt + 9 * s + 3 + t] = p1[t];
      tab[c.Nt + 9 * s + 6 + t] = p2[t];
    }
  }
  KKT_CUDA_TRY(cudaMalloc(&m->dof, of.size() * sizeof(int)));
  KKT_CUDA_TRY(cudaMalloc(&m->dtab, tab.size() * sizeof(double)));
  KKT_CUDA_TRY(cudaMemcpy(m->dof, of.data(), of.size() * sizeof(int), cudaMemcpyHostToDevice));
  KKT_CUDA_TRY(cudaMemcpy(m->dtab, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice));
  return KKT_OK;
}

}  // namespace kkt

using namespace kkt;

extern "C" {

int kkt_mlp_default_config(kkt_mlp_config* c) {
  if (!c) return set_error(KKT_ERR_INVALID_ARG, "null config");
  c->nx = 256;
  c->Nt = 2048;
  c->n_sub = 256;
  c->T = 1.0;
  c->modes = 32;
  c->width = 512;
  c->seed = 4;
  c->nu_lo = 0.1;
  c->nu_hi = 10.0;
  c->omega_lo = 1e-6;
  c->omega_hi = 1e-2;
  c->samples = 10240;
  c->epochs = 30;
  c->batch = 256;
  c->lr = 1e-3;
  c->resid_epochs = 30;
  return KKT_OK;
}

kkt_mlp* kkt_mlp_create(const kkt_mlp_config* cfg) {
  if (!cfg || cfg->n_sub < 1 || cfg->Nt / cfg->n_sub < 2 || cfg->width < 1 || cfg->modes < 1 || cfg->nx < 2 ||
      cfg->modes > cfg->nx - 1 || cfg->epochs < 0 || cfg->resid_epochs < 0) {
    set_error(KKT_ERR_INVALID_ARG, "invalid network configuration");
    return nullptr;
  }
  kkt_mlp* m = new kkt_mlp();
  m->cfg = *cfg;
  m->d_out = 2 * cfg->n_sub;
  m->d_in = m->d_out + 2;
  m->H = cfg->width;
  m->nparam = static_cast<long long>(m->H) * m->d_in + m->H + static_cast<long long>(m->H) * m->H + m->H +
              static_cast<long long>(m->d_out) * m->H + m->d_out;
  const size_t n = static_cast<size_t>(m->nparam);
  bool ok = cudaMalloc(&m->p, n * 4) == cudaSuccess && cudaMalloc(&m->g, n * 4) == cudaSuccess &&
            cudaMalloc(&m->m, n * 4) == cudaSuccess && cudaMalloc(&m->v, n * 4) == cudaSuccess &&
            cudaMalloc(&m->pb, n * 2) == cudaSuccess && cudaMalloc(&m->part, 4096 * sizeof(double)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    set_error(KKT_ERR_OOM, "network allocation failed");
    kkt_mlp_destroy(m);
    return nullptr;
  }
  // He-normal initialisation from the seed (std::mt19937_64), zero biases
  std::vector<float> h(n, 0.f);
  std::mt19937_64 rng(static_cast<unsigned long long>(cfg->seed));
  std::normal_distribution<double> nd(0.0, 1.0);
  ParamView P = view(h.data(), m);
  for (long long i = 0; i < static_cast<long long>(m->H) * m->d_in; ++i) P.W1[i] = static_cast<float>(nd(rng) * std::sqrt(2.0 / m->d_in));
  for (long long i = 0; i < static_cast<long long>(m->H) * m->H; ++i) P.W2[i] = static_cast<float>(nd(rng) * std::sqrt(2.0 / m->H));
  for (long long i = 0; i < static_cast<long long>(m->d_out) * m->H; ++i) P.W3[i] = static_cast<float>(nd(rng) * std::sqrt(2.0 / m->H));
  if (cudaMemcpy(m->p, h.data(), n * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(m->m, 0, n * 4) != cudaSuccess || cudaMemset(m->v, 0, n * 4) != cudaSuccess ||
      mlp_refresh_bf16(m, nullptr) < 0 || mlp_upload_decomp(m) < 0 || cudaDeviceSynchronize() != cudaSuccess) {
    set_error(KKT_ERR_CUDA, "network initialisation failed");
    kkt_mlp_destroy(m);
    return nullptr;
  }
  return m;
}

void kkt_mlp_destroy(kkt_mlp* m) {
  if (!m) return;
  cudaFree(m->p);
  cudaFree(m->pb);
  cudaFree(m->g);
  cudaFree(m->m);
  cudaFree(m->v);
  cudaFree(m->a1);
  cudaFree(m->a2);
  cudaFree(m->y);
  cudaFree(m->dy);
  cudaFree(m->dh2);
  cudaFree(m->dh1);
  cudaFree(m->part);
  cudaFree(m->dof);
  cudaFree(m->dtab);
  cudaFree(m->rscratch);
  cudaFree(m->lossv);
  delete m;
}

int kkt_mlp_param_count(const kkt_mlp* m, long long* count) {
  if (!m || !count) return set_error(KKT_ERR_INVALID_ARG, "null argument");
  *count = m->nparam;
  return KKT_OK;
}

int kkt_mlp_get_config(const kkt_mlp* m, kkt_mlp_config* cfg) {
  if (!m || !cfg) return set_error(KKT_ERR_INVALID_ARG, "null argument");
  *cfg = m->cfg;
  return KKT_OK;
}

int kkt_mlp_set_params(kkt_mlp* m, const float* host, long long count) {
  if (!m || !host || count != m->nparam) return set_error(KKT_ERR_INVALID_ARG, "parameter count mismatch");
  KKT_CUDA_TRY(cudaMemcpy(m->p, host, count * 4, cudaMemcpyHostToDevice));
  KKT_TRY(mlp_refresh_bf16(m, nullptr));
  KKT_CUDA_TRY(cudaDeviceSynchronize());
  return KKT_OK;
}

int kkt_mlp_get_params(const kkt_mlp* m, float* host, long long count) {
  if (!m || !host || count != m->nparam) return set_error(KKT_ERR_INVALID_ARG, "parameter count mismatch");
  KKT_CUDA_TRY(cudaMemcpy(host, m->p, count * 4, cudaMemcpyDeviceToHost));
  return KKT_OK;
}

int kkt_mlp_forward(kkt_mlp* m, const float* X, float* Y, int batch, int use_bf16, void* stream) {
  if (!m || !X || !Y || batch < 1) return set_error(KKT_ERR_INVALID_ARG, "invalid forward arguments");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  KKT_TRY(mlp_forward(m, X, batch, use_bf16, st));
  KKT_CUDA_TRY(cudaMemcpyAsync(Y, m->y, static_cast<size_t>(batch) * m->d_out * 4, cudaMemcpyDeviceToDevice, st));
  return KKT_OK;
}

int kkt_mlp_loss_grad(kkt_mlp* m, const float* X, const float* T, int batch, float* grad, double* loss, void* stream) {
  if (!m || !X || !T || batch < 1) return set_error(KKT_ERR_INVALID_ARG, "invalid gradient arguments");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  KKT_TRY(mlp_loss_grad(m, X, T, batch, loss, st));
  if (grad) KKT_CUDA_TRY(cudaMemcpyAsync(grad, m->g, m->nparam * 4, cudaMemcpyDeviceToDevice, st));
  return KKT_OK;
}

int kkt_mlp_adam_step(kkt_mlp* m, const float* X, const float* T, int batch, double lr, double* loss, void* stream) {
  if (!m || !X || !T || batch < 1) return set_error(KKT_ERR_INVALID_ARG, "invalid step arguments");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  KKT_TRY(mlp_loss_grad(m, X, T, batch, loss, st));
  KKT_TRY(mlp_adam(m, static_cast<float>(lr), st));
  return mlp_refresh_bf16(m, st);
}

int kkt_mlp_resid_loss_grad(kkt_mlp* m, const float* X, const double* mu, int batch, float* grad, double* loss,
                            void* stream) {
  if (!m || !X || !mu || batch < 1) return set_error(KKT_ERR_INVALID_ARG, "invalid gradient arguments");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  KKT_TRY(mlp_resid_loss_grad(m, X, mu, batch, loss, st));
  if (grad) KKT_CUDA_TRY(cudaMemcpyAsync(grad, m->g, m->nparam * 4, cudaMemcpyDeviceToDevice, st));
  return KKT_OK;
}

int kkt_mlp_coarse_data(kkt_mlp* m, const double* r, const double* mu, long long count, double* c, double* x,
                        void* stream) {
  if (!m || !r || !mu || !c || !x || count < 1) return set_error(KKT_ERR_INVALID_ARG, "invalid coarse-data arguments");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const kkt_mlp_config& cf = m->cfg;
  double* w = nullptr;
  KKT_CUDA_TRY(cudaMalloc(&w, static_cast<size_t>(count) * 5 * cf.n_sub * sizeof(double)));
  DecompView dv{cf.n_sub, cf.Nt, m->dof, m->dof + cf.n_sub, m->dtab, m->dtab + cf.Nt};
  coarse_data_kernel<<<static_cast<unsigned>((count + 127) / 128), 128, 0, st>>>(r, mu, count, dv, c, x, w);
  const cudaError_t e1 = cudaGetLastError();
  const cudaError_t e2 = cudaStreamSynchronize(st);
  cudaFree(w);
  KKT_CUDA_TRY(e1);
  KKT_CUDA_TRY(e2);
  return KKT_OK;
}

int kkt_mlp_train(kkt_mlp* m, kkt_mlp_train_stats* stats, void* stream) {
  if (!m) return set_error(KKT_ERR_INVALID_ARG, "null network");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const kkt_mlp_config& c = m->cfg;
  const int K = c.modes, nc = 2 * c.n_sub;
  const int per = K * K;                           // samples per (nu, omega) draw
  const int draws = std::max(1, (c.samples + per - 1) / per);
  const long long S = static_cast<long long>(draws) * per;
  // seeded samples: (nu, omega) log-uniform, modes k, l < K of the nx grid, residual time series
  std::mt19937_64 rng(static_cast<unsigned long long>(c.seed) * 7919ULL + 17ULL);
  std::uniform_real_distribution<double> uni(0.0, 1.0);
  std::normal_distribution<double> nd(0.0, 1.0);
  const double dt = c.T / c.Nt, dx = 1.0 / c.nx, pi = 3.14159265358979323846;
  std::vector<double> mu(S), feat(2 * S), r(static_cast<size_t>(c.Nt) * S);
  for (int dr = 0; dr < draws; ++dr) {
    const double nu = c.nu_lo * std::pow(c.nu_hi / c.nu_lo, uni(rng));
    const double om = c.omega_lo * std::pow(c.omega_hi / c.omega_lo, uni(rng));
    for (int l = 0; l < K; ++l)
      for (int k = 0; k < K; ++k) {
        const long long i = static_cast<long long>(dr) * per + l * K + k;
        const double sx = std::sin((k + 1) * pi / (2.0 * c.nx)), sy = std::sin((l + 1) * pi / (2.0 * c.nx));
        const double lam = 4.0 / (dx * dx) * (sx * sx + sy * sy);
        mu[i] = 1.0 + dt / std::sqrt(om) + dt * nu * lam;
        feat[2 * i] = std::log(dt * nu * lam);
        feat[2 * i + 1] = std::log(dt / std::sqrt(om));
        // smooth random time series plus noise
        double a[8], ph[8];
        for (int j = 0; j < 8; ++j) {
          a[j] = nd(rng) / (j + 1);
          ph[j] = 2 * pi * uni(rng);
        }
        const double noise = 0.2 * uni(rng);
        for (int n = 0; n < c.Nt; ++n) {
          double v = 0;
          for (int j = 0; j < 8; ++j) v += a[j] * std::sin(pi * (j + 1) * (n + 1.0) / c.Nt + ph[j]);
          r[static_cast<size_t>(n) * S + i] = v + noise * nd(rng);
        }
      }
  }
  // device buffers
  double *d_r = nullptr, *d_mu = nullptr, *d_feat = nullptr, *d_c = nullptr, *d_x = nullptr, *d_w = nullptr;
  float *X = nullptr, *Tt = nullptr;
  auto cleanup = [&]() {
    cudaFree(d_r);
    cudaFree(d_mu);
    cudaFree(d_feat);
    cudaFree(d_c);
    cudaFree(d_x);
    cudaFree(d_w);
    cudaFree(X);
    cudaFree(Tt);
  };
  auto fail = [&](const char* what) {
    cudaGetLastError();
    cleanup();
    return set_error(KKT_ERR_CUDA, std::string("network training: ") + what);
  };
  if (cudaMalloc(&d_r, r.size() * 8) || cudaMalloc(&d_mu, S * 8) || cudaMalloc(&d_feat, 2 * S * 8) ||
      cudaMalloc(&d_c, S * nc * 8) || cudaMalloc(&d_x, S * nc * 8) || cudaMalloc(&d_w, S * 5LL * c.n_sub * 8) ||
      cudaMalloc(&X, S * (nc + 2) * 4) || cudaMalloc(&Tt, S * nc * 4))
    return fail("allocation");
  if (cudaMemcpy(d_r, r.data(), r.size() * 8, cudaMemcpyHostToDevice) ||
      cudaMemcpy(d_mu, mu.data(), S * 8, cudaMemcpyHostToDevice) ||
      cudaMemcpy(d_feat, feat.data(), 2 * S * 8, cudaMemcpyHostToDevice))
    return fail("upload");
  DecompView dv{c.n_sub, c.Nt, m->dof, m->dof + c.n_sub, m->dtab, m->dtab + c.Nt};
  coarse_data_kernel<<<static_cast<unsigned>((S + 127) / 128), 128, 0, st>>>(d_r, d_mu, S, dv, d_c, d_x, d_w);
  make_xy_kernel<<<static_cast<unsigned>((S * 32 + 255) / 256), 256, 0, st>>>(d_c, d_x, d_feat, S, nc, X, Tt);
  if (cudaGetLastError() != cudaSuccess) return fail("sample generation");
  // held-out tenth for validation
  const long long ntrain = S - S / 10;
  const int B = std::max(1, c.batch);
  std::vector<long long> order(ntrain / B);
  for (size_t i = 0; i < order.size(); ++i) order[i] = static_cast<long long>(i) * B;
  double last = 0.0;
  int steps = 0;
  // phase 1: squared error to the unit target; phase 2: the coarse residual after the
  // minimal-residual step (the guard's quantity). Each phase steps at lr for its first two
  // thirds and at 0.3 lr after.
  const int total = c.epochs + c.resid_epochs;
  for (int ep = 0; ep < total; ++ep) {
    const bool resid = ep >= c.epochs;
    const int e_in = resid ? ep - c.epochs : ep, e_len = resid ? c.resid_epochs : c.epochs;
    std::shuffle(order.begin(), order.end(), rng);
    const float lr = static_cast<float>(c.lr * (e_in < e_len * 2 / 3 ? 1.0 : 0.3));
    for (size_t bi = 0; bi < order.size(); ++bi) {
      const long long o = order[bi];
      double* lp = (bi + 1 == order.size()) ? &last : nullptr;
      const int rc = resid ? mlp_resid_loss_grad(m, X + o * (nc + 2), d_mu + o, B, lp, st)
                           : mlp_loss_grad(m, X + o * (nc + 2), Tt + o * nc, B, lp, st);
      if (rc < 0 || mlp_adam(m, lr, st) < 0) {
        const std::string msg = kkt_last_error();
        cleanup();
        return set_error(KKT_ERR_CUDA, "network training step: " + msg);
      }
      ++steps;
    }
  }
  mlp_refresh_bf16(m, st);
  // validation on the held-out samples with the BF16 weights the preconditioner uses: mean
  // cosine to the unit target, and the coarse residual after the minimal-residual step (its mean
  // and the fraction within the guard's bound ||c - alpha G d||^2 <= ||c||^2 / 4)
  const long long nval = S - ntrain;
  double cos_sum = 0.0, val_loss = 0.0, res_sum = 0.0;
  long long within = 0;
  if (nval > 0) {
    std::vector<float> yv(static_cast<size_t>(nval) * nc), tv(static_cast<size_t>(nval) * nc);
    std::vector<double> lv(nval);
    if (mlp_forward(m, X + ntrain * (nc + 2), static_cast<int>(nval), 1, st) < 0 ||
        mlp_resid_eval(m, m->y, X + ntrain * (nc + 2), d_mu + ntrain, static_cast<int>(nval), false, nullptr, st) < 0)
      return fail("validation");
    cudaMemcpyAsync(yv.data(), m->y, yv.size() * 4, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(tv.data(), Tt + ntrain * nc, tv.size() * 4, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(lv.data(), m->lossv, lv.size() * 8, cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    for (long long i = 0; i < nval; ++i) {
      double dot = 0, yy = 0, e = 0;
      for (int j = 0; j < nc; ++j) {
        const double a = yv[i * nc + j], b = tv[i * nc + j];
        dot += a * b;
        yy += a * a;
        e += (a - b) * (a - b);
      }
      cos_sum += yy > 0 ? dot / std::sqrt(yy) : 0.0;
      val_loss += 0.5 * e;
      res_sum += lv[i];
      within += lv[i] <= 0.25 ? 1 : 0;
    }
  }
  cleanup();
  KKT_CUDA_TRY(cudaStreamSynchronize(st));
  if (stats) {
    stats->samples = static_cast<int>(S);
    stats->steps = steps;
    stats->final_train_loss = last;
    stats->val_loss = nval > 0 ? val_loss / nval : 0.0;
    stats->val_cosine = nval > 0 ? cos_sum / nval : 0.0;
    stats->val_resid = nval > 0 ? res_sum / nval : 0.0;
    stats->val_within_guard = nval > 0 ? static_cast<double>(within) / nval : 0.0;
  }
  return KKT_OK;
}

int kkt_mlp_save(const kkt_mlp* m, const char* path) {
  if (!m || !path) return set_error(KKT_ERR_INVALID_ARG, "null argument");
  std::vector<float> h(m->nparam);
  KKT_CUDA_TRY(cudaMemcpy(h.data(), m->p, h.size() * 4, cudaMemcpyDeviceToHost));
  FILE* f = std::fopen(path, "wb");
  if (!f) return set_error(KKT_ERR_INVALID_ARG, std::string("cannot open ") + path);
  const char magic[8] = {'K', 'K', 'T', 'M', 'L', 'P', '0', '2'};
  bool ok = std::fwrite(magic, 1, 8, f) == 8 && std::fwrite(&m->cfg, sizeof(kkt_mlp_config), 1, f) == 1 &&
            std::fwrite(&m->nparam, sizeof(long long), 1, f) == 1 && std::fwrite(h.data(), 4, h.size(), f) == h.size();
  std::fclose(f);
  return ok ? KKT_OK : set_error(KKT_ERR_INVALID_ARG, "write failed");
}

kkt_mlp* kkt_mlp_load(const char* path) {
  FILE* f = path ? std::fopen(path, "rb") : nullptr;
  if (!f) {
    set_error(KKT_ERR_INVALID_ARG, "cannot open network file");
    return nullptr;
  }
  char magic[8];
  kkt_mlp_config cfg;
  long long n = 0;
  bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "KKTMLP02", 8) == 0 &&
            std::fread(&cfg, sizeof(cfg), 1, f) == 1 && std::fread(&n, sizeof(n), 1, f) == 1;
  kkt_mlp* m = ok ? kkt_mlp_create(&cfg) : nullptr;
  if (m && n == m->nparam) {
    std::vector<float> h(n);
    ok = std::fread(h.data(), 4, n, f) == static_cast<size_t>(n) && kkt_mlp_set_params(m, h.data(), n) == KKT_OK;
  } else {
    ok = false;
  }
  std::fclose(f);
  if (!ok) {
    kkt_mlp_destroy(m);
    set_error(KKT_ERR_INVALID_ARG, "not a network file of this library");
    return nullptr;
  }
  return m;
}

}  // extern "C"
