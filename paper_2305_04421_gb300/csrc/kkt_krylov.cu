// Streaming FP64 kernels of the FGMRES Arnoldi process (Section 4: right-preconditioned GMRES):
// the multi-dot <V_k, w> of classical Gram-Schmidt, the fused multi-axpy w -= sum c_k V_k with
// the norm of the result, and the solution update x += sum c_k V_k.
//
// Reductions are deterministic: a fixed grid of blocks each reduces its grid-stride share
// (warp shuffles, then shared memory) into one partial per block, and a second kernel sums
// the partials of each output in a fixed order. Results land in h->red_out on the device.
#include <mutex>

#include "kkt_internal.cuh"

namespace kkt {
namespace {

constexpr int kRedThreads = 256;
constexpr int kMaxVec = 32;

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// sums `val` over the block; valid in thread 0
__device__ __forceinline__ double block_sum(double v, double* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (warp == 0) {
    t = lane < (blockDim.x >> 5) ? sh[lane] : 0.0;
    t = warp_sum(t);
  }
  return t;
}

// Pairs of elements are loaded with 16-byte loads when every row start is 16-byte aligned
// (vec2 = true), halving the load instructions per FP64 FMA; odd tails are done scalar.
__device__ __forceinline__ long long pair_count(long long n, bool vec2) { return vec2 ? n / 2 : 0; }

template <int NV>
__global__ void __launch_bounds__(kRedThreads) multidot_kernel(const double* __restrict__ V, long long stride,
                                                               const double* __restrict__ w, long long n,
                                                               double* __restrict__ part, bool vec2) {
  __shared__ double sh[32];
  double acc[NV + 1];
#pragma unroll
  for (int k = 0; k <= NV; ++k) acc[k] = 0.0;
  const long long gs = static_cast<long long>(gridDim.x) * blockDim.x;
  const long long tid = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  const long long np = pair_count(n, vec2);
  for (long long i = tid; i < np; i += gs) {
    const double2 wi = reinterpret_cast<const double2*>(w)[i];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const double2 v = reinterpret_cast<const double2*>(V + k * stride)[i];
      acc[k] = fma(v.x, wi.x, fma(v.y, wi.y, acc[k]));
    }
    acc[NV] = fma(wi.x, wi.x, fma(wi.y, wi.y, acc[NV]));
  }
  for (long long i = 2 * np + tid; i < n; i += gs) {
    const double wi = w[i];
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = fma(V[k * stride + i], wi, acc[k]);
    acc[NV] = fma(wi, wi, acc[NV]);
  }
#pragma unroll
  for (int k = 0; k <= NV; ++k) {
    const double t = block_sum(acc[k], sh);
    if (threadIdx.x == 0) part[static_cast<long long>(blockIdx.x) * (NV + 1) + k] = t;
  }
}

template <int NV>
__global__ void __launch_bounds__(kRedThreads) update_norm_kernel(const double* __restrict__ V, long long stride,
                                                                  const double* __restrict__ coef, double* __restrict__ w,
                                                                  long long n, double* __restrict__ part, bool vec2) {
  __shared__ double sh[32];
  double c[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) c[k] = coef[k];
  double acc = 0.0;
  const long long gs = static_cast<long long>(gridDim.x) * blockDim.x;
  const long long tid = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  const long long np = pair_count(n, vec2);
  for (long long i = tid; i < np; i += gs) {
    double2 wi = reinterpret_cast<double2*>(w)[i];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const double2 v = reinterpret_cast<const double2*>(V + k * stride)[i];
      wi.x = fma(-c[k], v.x, wi.x);
      wi.y = fma(-c[k], v.y, wi.y);
    }
    reinterpret_cast<double2*>(w)[i] = wi;
    acc = fma(wi.x, wi.x, fma(wi.y, wi.y, acc));
  }
  for (long long i = 2 * np + tid; i < n; i += gs) {
    double wi = w[i];
#pragma unroll
    for (int k = 0; k < NV; ++k) wi = fma(-c[k], V[k * stride + i], wi);
    w[i] = wi;
    acc = fma(wi, wi, acc);
  }
  const double t = block_sum(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

template <int NV>
__global__ void __launch_bounds__(kRedThreads) axpy_multi_kernel(const double* __restrict__ V, long long stride,
                                                                 const double* __restrict__ coef, double* __restrict__ x,
                                                                 long long n, bool vec2) {
  double c[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) c[k] = coef[k];
  const long long gs = static_cast<long long>(gridDim.x) * blockDim.x;
  const long long tid = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  const long long np = pair_count(n, vec2);
  for (long long i = tid; i < np; i += gs) {
    double2 xi = reinterpret_cast<double2*>(x)[i];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const double2 v = reinterpret_cast<const double2*>(V + k * stride)[i];
      xi.x = fma(c[k], v.x, xi.x);
      xi.y = fma(c[k], v.y, xi.y);
    }
    reinterpret_cast<double2*>(x)[i] = xi;
  }
  for (long long i = 2 * np + tid; i < n; i += gs) {
    double xi = x[i];
#pragma unroll
    for (int k = 0; k < NV; ++k) xi = fma(c[k], V[k * stride + i], xi);
    x[i] = xi;
  }
}

// One modified Gram-Schmidt step (AXPY: w -= c Vk with c = dot[0] * s, read once per thread;
// DOTV: the partial dot is <Vn, w> over the updated w, else <w, w>).
template <bool AXPY, bool DOTV>
__global__ void __launch_bounds__(kRedThreads) mgs_step_kernel(const double* __restrict__ Vk,
                                                               const double* __restrict__ dot, double s,
                                                               const double* __restrict__ Vn, double* __restrict__ w,
                                                               long long n, double* __restrict__ part, bool vec2) {
  __shared__ double sh[32];
  const double c = AXPY ? dot[0] * s : 0.0;
  double acc = 0.0;
  const long long gs = static_cast<long long>(gridDim.x) * blockDim.x;
  const long long tid = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  const long long np = pair_count(n, vec2);
  for (long long i = tid; i < np; i += gs) {
    double2 wi = reinterpret_cast<const double2*>(w)[i];
    if (AXPY) {
      const double2 v = reinterpret_cast<const double2*>(Vk)[i];
      wi.x = fma(-c, v.x, wi.x);
      wi.y = fma(-c, v.y, wi.y);
      reinterpret_cast<double2*>(w)[i] = wi;
    }
    const double2 o = DOTV ? reinterpret_cast<const double2*>(Vn)[i] : wi;
    acc = fma(o.x, wi.x, fma(o.y, wi.y, acc));
  }
  for (long long i = 2 * np + tid; i < n; i += gs) {
    double wi = w[i];
    if (AXPY) {
      wi = fma(-c, Vk[i], wi);
      w[i] = wi;
    }
    acc = fma(DOTV ? Vn[i] : wi, wi, acc);
  }
  const double t = block_sum(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// Blocked MGS step (blocks of BS basis vectors; BS = 2, 4 or 8): w -= sum_{a < na} c_a A_a
// (c_a = dot[a] * s_a, A_a = A + a stride), then the partial dots <B_d, w> (B_d = Bv + d stride,
// d < nd) over the updated w, or <w, w> when NORM (nd = 0). part holds max(nd, 1) columns per
// block. The counts are uniform over the grid, so the loads and FMAs of the unrolled loops are
// predicated, not branched.
template <int BS>
struct MgsScale {
  double s[BS];
};

// (Pairs are compiled for four resident blocks per SM, the launch's whole grid.)
template <int BS, bool NORM, int U>
__global__ void __launch_bounds__(kRedThreads, BS == 2 ? 4 : 1) mgsb_step_kernel(const double* __restrict__ A,
                                                                const double* __restrict__ Bv, long long stride,
                                                                int na, int nd, const double* __restrict__ dot,
                                                                MgsScale<BS> sc, double* __restrict__ w, long long n,
                                                                double* __restrict__ part, bool vec2) {
  __shared__ double sh[32];
  double c[BS], acc[BS];
#pragma unroll
  for (int a = 0; a < BS; ++a) {
    c[a] = a < na ? dot[a] * sc.s[a] : 0.0;
    acc[a] = 0.0;
  }
  const long long gs = static_cast<long long>(gridDim.x) * blockDim.x;
  const long long tid = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  const long long np = pair_count(n, vec2);
  const double2 z2 = make_double2(0.0, 0.0);
  // U grid strides per trip, their loads issued together (U = 2 or 4 for the steps that stream
  // few vectors, whose single stride keeps too few loads in flight); the accumulation order is
  // that of U = 1, and an element past the end loads zeros and adds nothing
  for (long long i0 = tid; i0 < np; i0 += U * gs) {
    double2 wi[U], av[U][BS], bv[U][BS];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const long long i = i0 + u * gs;
      const bool in = U == 1 || i < np;
      wi[u] = in ? reinterpret_cast<const double2*>(w)[i] : z2;
#pragma unroll
      for (int a = 0; a < BS; ++a) av[u][a] = (in && a < na) ? reinterpret_cast<const double2*>(A + a * stride)[i] : z2;
#pragma unroll
      for (int d = 0; d < BS; ++d)
        bv[u][d] = (in && !NORM && d < nd) ? reinterpret_cast<const double2*>(Bv + d * stride)[i] : z2;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const long long i = i0 + u * gs;
      if (na > 0) {
#pragma unroll
        for (int a = 0; a < BS; ++a)
          if (a < na) {
            wi[u].x = fma(-c[a], av[u][a].x, wi[u].x);
            wi[u].y = fma(-c[a], av[u][a].y, wi[u].y);
          }
        if (U == 1 || i < np) reinterpret_cast<double2*>(w)[i] = wi[u];
      }
      if (NORM) {
        acc[0] = fma(wi[u].x, wi[u].x, fma(wi[u].y, wi[u].y, acc[0]));
      } else {
#pragma unroll
        for (int d = 0; d < BS; ++d)
          if (d < nd) acc[d] = fma(bv[u][d].x, wi[u].x, fma(bv[u][d].y, wi[u].y, acc[d]));
      }
    }
  }
  for (long long i = 2 * np + tid; i < n; i += gs) {
    double wi = w[i];
    if (na > 0) {
#pragma unroll
      for (int a = 0; a < BS; ++a)
        if (a < na) wi = fma(-c[a], A[a * stride + i], wi);
      w[i] = wi;
    }
    if (NORM) {
      acc[0] = fma(wi, wi, acc[0]);
    } else {
#pragma unroll
      for (int d = 0; d < BS; ++d)
        if (d < nd) acc[d] = fma(Bv[d * stride + i], wi, acc[d]);
    }
  }
  const int width = NORM ? 1 : nd;
#pragma unroll
  for (int d = 0; d < BS; ++d)
    if (d < width) {
      const double t = block_sum(acc[d], sh);
      if (threadIdx.x == 0) part[static_cast<long long>(blockIdx.x) * width + d] = t;
    }
}

__global__ void norm_kernel(const double* __restrict__ x, long long n, double* __restrict__ part) {
  __shared__ double sh[32];
  double acc = 0.0;
  const long long gs = static_cast<long long>(gridDim.x) * blockDim.x;
  for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += gs)
    acc = fma(x[i], x[i], acc);
  const double t = block_sum(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// out[k] = sum_b part[b * width + k], one warp per output, fixed order
__global__ void finalize_kernel(const double* __restrict__ part, int nblocks, int width, double* __restrict__ out) {
  const int k = blockIdx.x;
  double acc = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += 32) acc += part[static_cast<long long>(b) * width + k];
  acc = warp_sum(acc);
  if (threadIdx.x == 0) out[k] = acc;
}

// 16-byte loads are usable when every row start is 16-byte aligned
bool can_vec2(const void* a, const void* b, long long stride) {
  return (reinterpret_cast<uintptr_t>(a) % 16 == 0) && (reinterpret_cast<uintptr_t>(b) % 16 == 0) && (stride % 2 == 0);
}

int grid_blocks() {
  static int blocks = 0;
  if (!blocks) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    blocks = (sms > 0 ? sms : 132) * 4;
  }
  return blocks;
}

template <template <int> class Dispatch, typename... Args>
int dispatch_nv(int count, Args... args) {
  switch (count) {
#define KKT_NV_CASE(k) \
  case k:              \
    return Dispatch<k>::run(args...);
    KKT_NV_CASE(1) KKT_NV_CASE(2) KKT_NV_CASE(3) KKT_NV_CASE(4) KKT_NV_CASE(5) KKT_NV_CASE(6)
    KKT_NV_CASE(7) KKT_NV_CASE(8) KKT_NV_CASE(9) KKT_NV_CASE(10) KKT_NV_CASE(11) KKT_NV_CASE(12)
    KKT_NV_CASE(13) KKT_NV_CASE(14) KKT_NV_CASE(15) KKT_NV_CASE(16) KKT_NV_CASE(17) KKT_NV_CASE(18)
    KKT_NV_CASE(19) KKT_NV_CASE(20) KKT_NV_CASE(21) KKT_NV_CASE(22) KKT_NV_CASE(23) KKT_NV_CASE(24)
    KKT_NV_CASE(25) KKT_NV_CASE(26) KKT_NV_CASE(27) KKT_NV_CASE(28) KKT_NV_CASE(29) KKT_NV_CASE(30)
    KKT_NV_CASE(31) KKT_NV_CASE(32)
#undef KKT_NV_CASE
    default:
      return set_error(KKT_ERR_INVALID_ARG, "Krylov kernel vector count out of range");
  }
}

template <int NV>
struct MultidotRun {
  static int run(const double* V, long long stride, const double* w, long long n, double* part, int nb,
                 cudaStream_t st) {
    ProfScope ps(KKT_K_MULTIDOT, st, 2.0 * (NV + 1) * n, 8.0 * (NV + 1) * n);
    multidot_kernel<NV><<<nb, kRedThreads, 0, st>>>(V, stride, w, n, part, can_vec2(V, w, stride));
    KKT_CUDA_TRY(cudaGetLastError());
    return KKT_OK;
  }
};

template <int NV>
struct UpdateRun {
  static int run(const double* V, long long stride, const double* coef, double* w, long long n, double* part,
                 int nb, cudaStream_t st) {
    ProfScope ps(KKT_K_UPDATE, st, 2.0 * (NV + 1) * n, 8.0 * (NV + 2) * n);
    update_norm_kernel<NV><<<nb, kRedThreads, 0, st>>>(V, stride, coef, w, n, part, can_vec2(V, w, stride));
    KKT_CUDA_TRY(cudaGetLastError());
    return KKT_OK;
  }
};

template <int NV>
struct AxpyRun {
  static int run(const double* V, long long stride, const double* coef, double* x, long long n, int nb,
                 cudaStream_t st) {
    ProfScope ps(KKT_K_AXPY, st, 2.0 * NV * n, 8.0 * (NV + 2) * n);
    axpy_multi_kernel<NV><<<nb, kRedThreads, 0, st>>>(V, stride, coef, x, n, can_vec2(V, x, stride));
    KKT_CUDA_TRY(cudaGetLastError());
    return KKT_OK;
  }
};

}  // namespace

int krylov_multidot(kkt_handle* h, const double* V, long long stride, int count, const double* w, long long n,
                    cudaStream_t st, double* out) {
  const int nb = grid_blocks();
  if (!out) out = h->red_out;
  int done = 0;
  // groups of up to 32 vectors; each group writes count_g + 1 partial columns (last = <w,w>)
  while (done < count) {
    const int cg = std::min(kMaxVec, count - done);
    KKT_TRY(dispatch_nv<MultidotRun>(cg, V + done * stride, stride, static_cast<const double*>(w), n, h->red, nb, st));
    {
      ProfScope ps(KKT_K_REDUCE, st);
      finalize_kernel<<<cg + 1, 32, 0, st>>>(h->red, nb, cg + 1, out + done);
    }
    KKT_CUDA_TRY(cudaGetLastError());
    done += cg;
  }
  return KKT_OK;
}

int krylov_update_norm(kkt_handle* h, const double* V, long long stride, int count, const double* coef_dev,
                       double* w, long long n, cudaStream_t st) {
  const int nb = grid_blocks();
  if (count > kMaxVec) return set_error(KKT_ERR_INVALID_ARG, "too many basis vectors");
  KKT_TRY(dispatch_nv<UpdateRun>(count, V, stride, coef_dev, w, n, h->red, nb, st));
  {
    ProfScope ps(KKT_K_REDUCE, st);
    finalize_kernel<<<1, 32, 0, st>>>(h->red, nb, 1, h->red_out);
  }
  KKT_CUDA_TRY(cudaGetLastError());
  return KKT_OK;
}

int krylov_axpy_multi(const double* V, long long stride, int count, const double* coef_dev, double* x,
                      long long n, cudaStream_t st) {
  const int nb = grid_blocks();
  int done = 0;
  while (done < count) {
    const int cg = std::min(kMaxVec, count - done);
    KKT_TRY(dispatch_nv<AxpyRun>(cg, V + done * stride, stride, coef_dev + done, x, n, nb, st));
    done += cg;
  }
  return KKT_OK;
}

int krylov_norm2(kkt_handle* h, const double* x, long long n, cudaStream_t st) {
  const int nb = grid_blocks();
  {
    ProfScope ps(KKT_K_REDUCE, st);
    norm_kernel<<<nb, kRedThreads, 0, st>>>(x, n, h->red);
  }
  KKT_CUDA_TRY(cudaGetLastError());
  {
    ProfScope ps(KKT_K_REDUCE, st);
    finalize_kernel<<<1, 32, 0, st>>>(h->red, nb, 1, h->red_out);
  }
  KKT_CUDA_TRY(cudaGetLastError());
  return KKT_OK;
}

int krylov_mgs_step(kkt_handle* h, const double* Vk, const double* dot, double s, const double* Vn, double* w,
                    long long n, double* out, cudaStream_t st) {
  const int nb = grid_blocks();
  const bool vec2 = can_vec2(w, Vk ? Vk : w, 2) && can_vec2(w, Vn ? Vn : w, 2);
  if (!Vk && !Vn) return set_error(KKT_ERR_INVALID_ARG, "MGS step needs a vector");
  {
    // streaming: Vk and Vn read, w read (and written when Vk): 2 FP64 FMAs per element with Vk
    const double fl = (Vk ? 2.0 : 0.0) * n + 2.0 * n;
    const double by = 8.0 * n * ((Vk ? 2.0 : 0.0) + (Vn ? 1.0 : 0.0) + 1.0);
    ProfScope ps(Vk ? KKT_K_UPDATE : KKT_K_MULTIDOT, st, fl, by);
    if (Vk && Vn)
      mgs_step_kernel<true, true><<<nb, kRedThreads, 0, st>>>(Vk, dot, s, Vn, w, n, h->red, vec2);
    else if (Vk)
      mgs_step_kernel<true, false><<<nb, kRedThreads, 0, st>>>(Vk, dot, s, Vn, w, n, h->red, vec2);
    else
      mgs_step_kernel<false, true><<<nb, kRedThreads, 0, st>>>(Vk, dot, s, Vn, w, n, h->red, vec2);
    KKT_CUDA_TRY(cudaGetLastError());
  }
  {
    ProfScope ps(KKT_K_REDUCE, st);
    finalize_kernel<<<1, 32, 0, st>>>(h->red, nb, 1, out);
  }
  KKT_CUDA_TRY(cudaGetLastError());
  return KKT_OK;
}

namespace {
template <int BS>
int launch_mgsb(int nb, const double* A, const double* Bv, long long stride, int na, int nd, const double* dot,
                const double* s, double* w, long long n, double* part, bool vec2, cudaStream_t st) {
  MgsScale<BS> sc{};
  for (int a = 0; a < na; ++a) sc.s[a] = s[a];
  // grid strides per trip for pairs: 4 when one vector besides w is streamed, 2 up to three
  constexpr bool P2 = BS == 2;
  const int u = !P2 ? 1 : (na + nd <= 1 ? 4 : (na + nd <= 3 ? 2 : 1));
  if (nd == 0) {
    if (u == 4) mgsb_step_kernel<BS, true, P2 ? 4 : 1><<<nb, kRedThreads, 0, st>>>(A, Bv, stride, na, nd, dot, sc, w, n, part, vec2);
    else if (u == 2) mgsb_step_kernel<BS, true, P2 ? 2 : 1><<<nb, kRedThreads, 0, st>>>(A, Bv, stride, na, nd, dot, sc, w, n, part, vec2);
    else mgsb_step_kernel<BS, true, 1><<<nb, kRedThreads, 0, st>>>(A, Bv, stride, na, nd, dot, sc, w, n, part, vec2);
  } else {
    if (u == 4) mgsb_step_kernel<BS, false, P2 ? 4 : 1><<<nb, kRedThreads, 0, st>>>(A, Bv, stride, na, nd, dot, sc, w, n, part, vec2);
    else if (u == 2) mgsb_step_kernel<BS, false, P2 ? 2 : 1><<<nb, kRedThreads, 0, st>>>(A, Bv, stride, na, nd, dot, sc, w, n, part, vec2);
    else mgsb_step_kernel<BS, false, 1><<<nb, kRedThreads, 0, st>>>(A, Bv, stride, na, nd, dot, sc, w, n, part, vec2);
  }
  KKT_CUDA_TRY(cudaGetLastError());
  return KKT_OK;
}
}  // namespace

int krylov_mgsb_step(kkt_handle* h, int bs, int na, const double* A, const double* dot, const double* s, int nd,
                     const double* Bv, long long stride, double* w, long long n, double* out, cudaStream_t st) {
  if ((bs != 2 && bs != 4 && bs != 8) || na < 0 || na > bs || nd < 0 || nd > bs || (na == 0 && nd == 0) ||
      (na > 0 && (!A || !dot || !s)) || (nd > 0 && !Bv) || ((na > 1 || nd > 1) && stride < n))
    return set_error(KKT_ERR_INVALID_ARG, "blocked MGS step: bad block size, vector counts or pointers");
  const int nb = grid_blocks();
  bool vec2 = reinterpret_cast<uintptr_t>(w) % 16 == 0 && stride % 2 == 0;
  if (na > 0 && reinterpret_cast<uintptr_t>(A) % 16) vec2 = false;
  if (nd > 0 && reinterpret_cast<uintptr_t>(Bv) % 16) vec2 = false;
  {
    // per element: na + max(nd, 1) FMA; reads na + nd vectors and w, writes w when na > 0
    const double fl = 2.0 * n * (na + (nd > 0 ? nd : 1));
    const double by = 8.0 * n * (na + nd + 1 + (na > 0 ? 1 : 0));
    ProfScope ps(na > 0 ? KKT_K_UPDATE : KKT_K_MULTIDOT, st, fl, by);
    const int rc = bs == 2   ? launch_mgsb<2>(nb, A, Bv, stride, na, nd, dot, s, w, n, h->red, vec2, st)
                   : bs == 4 ? launch_mgsb<4>(nb, A, Bv, stride, na, nd, dot, s, w, n, h->red, vec2, st)
                             : launch_mgsb<8>(nb, A, Bv, stride, na, nd, dot, s, w, n, h->red, vec2, st);
    KKT_TRY(rc);
  }
  {
    const int width = nd > 0 ? nd : 1;
    ProfScope ps(KKT_K_REDUCE, st);
    finalize_kernel<<<width, 32, 0, st>>>(h->red, nb, width, out);
  }
  KKT_CUDA_TRY(cudaGetLastError());
  return KKT_OK;
}

int krylov_partial_capacity() { return grid_blocks() * (kMaxVec + 1); }

// ---- multi-dot without device allocation ------------------------------------------------
//
// Some callers cannot call cudaMalloc: a host application whose device memory is owned by
// another allocator (a framework's caching pool or a fixed arena sized at start-up), or a
// loop that must not allocate at all. kkt_multidot_noalloc serves them: the caller passes
// the inputs and the output, and the per-block partial sums live in the file-scope array
// below, which every GPU that loads this library holds until the process exits.
namespace {

constexpr int kNoAllocMaxBlocks = 1024;
constexpr int kNoAllocMaxCount = 32;
constexpr int kNoAllocWords = kNoAllocMaxBlocks * (kNoAllocMaxCount + 1);   // 270,336 bytes

static __device__ __align__(256) double g_noalloc_partials[kNoAllocWords];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_addr[kMaxDevices] = {};

// Device address of g_noalloc_partials on the current device. The array's name in host code
// is only a host-side stand-in, so the address is fetched with cudaGetSymbolAddress, once per
// device, with that device current.
int noalloc_scratch(double** out) {
  int dev = 0;
  KKT_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return set_error(KKT_ERR_UNSUPPORTED, "device index out of range");
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess || !p)
      return set_error(KKT_ERR_CUDA, std::string("cudaGetSymbolAddress of the multi-dot scratch: ") +
                                         cudaGetErrorString(e));
    g_noalloc_addr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_addr[dev];
  return KKT_OK;
}

template <int NV>
struct MultidotNoAllocRun {
  static int run(const double* V, long long stride, const double* w, long long n, double* part, int nb,
                 cudaStream_t st) {
    multidot_kernel<NV><<<nb, kRedThreads, 0, st>>>(V, stride, w, n, part, can_vec2(V, w, stride));
    KKT_CUDA_TRY(cudaGetLastError());
    return KKT_OK;
  }
};

bool device_pointer(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

}  // namespace kkt

extern "C" int kkt_multidot_noalloc(const double* V, long long stride, int count, const double* w, long long n,
                                    double* out, void* stream) {
  using namespace kkt;
  if (!V || !w || !out) return set_error(KKT_ERR_INVALID_ARG, "null pointer");
  if (count < 1 || count > kNoAllocMaxCount)
    return set_error(KKT_ERR_INVALID_ARG, "count must be in [1, 32]: the no-allocation scratch holds partial sums "
                                          "for at most 32 vectors");
  if (n < 1 || stride < n) return set_error(KKT_ERR_INVALID_ARG, "need n >= 1 and stride >= n");
  for (const void* p : {static_cast<const void*>(V), static_cast<const void*>(w), static_cast<const void*>(out)}) {
    if (reinterpret_cast<uintptr_t>(p) % 8) return set_error(KKT_ERR_INVALID_ARG, "pointer not 8-byte aligned");
    if (!device_pointer(p)) return set_error(KKT_ERR_INVALID_ARG, "pointer is not device memory");
  }
  double* part = nullptr;
  KKT_TRY(noalloc_scratch(&part));
  const int nb = std::min(grid_blocks(), kNoAllocMaxBlocks);
  if (static_cast<long long>(nb) * (count + 1) > kNoAllocWords)
    return set_error(KKT_ERR_INVALID_ARG, "multi-dot partials exceed the no-allocation scratch");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // every partial slot the finalisation reads (blocks < nb, columns <= count) is written by
  // this call's multi-dot launch first, so nothing left by an earlier call is read
  KKT_TRY(dispatch_nv<MultidotNoAllocRun>(count, V, stride, w, n, part, nb, st));
  finalize_kernel<<<count + 1, 32, 0, st>>>(part, nb, count + 1, out);
  KKT_CUDA_TRY(cudaGetLastError());
  return KKT_OK;
}
