// Batched form (not in the paper): many independent KKT instances of uneven sizes solved
// together. Instances are packed into memory waves (the FGMRES(30) basis of all 64 instances of
// the batched workload does not fit in HBM); inside a wave every instance runs the same FGMRES
// in lockstep, and each phase of an Arnoldi step is ONE launch over all instances: persistent
// kernels that walk a table of (instance, tile) work items. The preconditioner + matvec phase of
// step j reads every per-step pointer from tables prepared once per wave, and the only value
// that changes between restart cycles (1 / eta of the basis vector) from a device array, so it
// is captured once per (wave, j) as a CUDA graph and replayed. A small autotuner times the
// candidate tile heights of the batched sine transform and block sizes of the batched sweeps
// on the wave's own data and keeps the fastest.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "kkt_internal.cuh"

namespace kkt {
namespace {

constexpr int kThreads = 256;
constexpr long long kChunk = kThreads * 64;   // elements per work item of the vector kernels
// Resident blocks per SM the persistent vector kernels are compiled for (their grid is this many
// blocks per SM, so the whole grid is resident at once: no tail of late-starting blocks).
constexpr int kBlocksPerSm = 4;
// The multi-vector kernels with many vectors need more than 64 registers a thread: compiled (and
// launched) for 2 blocks per SM above 8 vectors and 1 above 20, so they do not spill.
constexpr int blocks_per_sm(int nv) { return nv > 20 ? 1 : nv > 8 ? 2 : kBlocksPerSm; }

struct Seg {
  const double* V;   // first vector (basis V_0 or a single vector)
  long long stride;  // distance between basis vectors
  double* w;         // target vector
  long long n;       // elements
};

// Each block copies the segment table and its item prefix to shared memory once (at most
// KKT_BATCH_MAX instances), so finding an item's segment costs no global-memory round trips.
#define KKT_SEG_TABLE                                                       \
  __shared__ Seg ss[KKT_BATCH_MAX];                                         \
  __shared__ long long sp[KKT_BATCH_MAX + 1];                               \
  for (int i_ = threadIdx.x; i_ < nj; i_ += blockDim.x) ss[i_] = segs[i_]; \
  batch_prefix_load(sp, prefix, nj);

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

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

// Two sums over the block at once (one pair of barriers); valid in thread 0.
__device__ __forceinline__ double2 block_sum2(double a, double b, double2* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  a = warp_sum(a);
  b = warp_sum(b);
  __syncthreads();
  if (lane == 0) sh[warp] = make_double2(a, b);
  __syncthreads();
  double2 t = make_double2(0.0, 0.0);
  if (warp == 0) {
    const double2 v = lane < (blockDim.x >> 5) ? sh[lane] : make_double2(0.0, 0.0);
    t = make_double2(warp_sum(v.x), warp_sum(v.y));
  }
  return t;
}

// part[t][k] = sum over item t's elements of V_k w (k < NV), part[t][NV] = sum w^2
template <int NV>
__global__ void __launch_bounds__(kThreads, blocks_per_sm(NV)) multidot_b(const Seg* __restrict__ segs, const long long* __restrict__ prefix,
                                                       int nj, long long total, double* __restrict__ part) {
  __shared__ double sh[32];
  KKT_SEG_TABLE
  for (long long t = blockIdx.x; t < total; t += gridDim.x) {
    const int k = batch_find(sp, nj, t);
    const Seg S = ss[k];
    const long long e0 = (t - sp[k]) * kChunk, e1 = min(e0 + kChunk, S.n);
    double acc[NV + 1];
#pragma unroll
    for (int v = 0; v <= NV; ++v) acc[v] = 0.0;
    for (long long i = e0 + threadIdx.x; i < e1; i += kThreads) {
      const double wi = S.w[i];
#pragma unroll
      for (int v = 0; v < NV; ++v) acc[v] = fma(S.V[v * S.stride + i], wi, acc[v]);
      acc[NV] = fma(wi, wi, acc[NV]);
    }
#pragma unroll
    for (int v = 0; v <= NV; ++v) {
      const double s = block_sum(acc[v], sh);
      if (threadIdx.x == 0) part[t * (NV + 1) + v] = s;
    }
  }
}

// w -= sum_k coef[inst][k] V_k over the item; part[t] = sum w^2 (NV = 0: norm only)
template <int NV>
__global__ void __launch_bounds__(kThreads, blocks_per_sm(NV)) update_b(const Seg* __restrict__ segs, const long long* __restrict__ prefix,
                                                     int nj, long long total, const double* __restrict__ coef, int ldc,
                                                     double* __restrict__ part, int want_norm) {
  __shared__ double sh[32];
  KKT_SEG_TABLE
  for (long long t = blockIdx.x; t < total; t += gridDim.x) {
    const int k = batch_find(sp, nj, t);
    const Seg S = ss[k];
    double c[NV > 0 ? NV : 1];
#pragma unroll
    for (int v = 0; v < NV; ++v) c[v] = coef[k * ldc + v];
    const long long e0 = (t - sp[k]) * kChunk, e1 = min(e0 + kChunk, S.n);
    double acc = 0.0;
    for (long long i = e0 + threadIdx.x; i < e1; i += kThreads) {
      double wi = S.w[i];
#pragma unroll
      for (int v = 0; v < NV; ++v)   // uniform per item: zero coefficients skip their vector
        if (c[v] != 0.0) wi = fma(-c[v], S.V[v * S.stride + i], wi);
      if (NV > 0) S.w[i] = wi;
      acc = fma(wi, wi, acc);
    }
    if (want_norm) {
      const double s = block_sum(acc, sh);
      if (threadIdx.x == 0) part[t] = s;
    }
  }
}

// out = alpha[inst] * x + beta[inst] * y, x = V, y = w of the segment (out = w)
__global__ void __launch_bounds__(kThreads, kBlocksPerSm) axpby_b(const Seg* __restrict__ segs, const long long* __restrict__ prefix,
                                                    int nj, long long total, const double* __restrict__ ab) {
  KKT_SEG_TABLE
  for (long long t = blockIdx.x; t < total; t += gridDim.x) {
    const int k = batch_find(sp, nj, t);
    const Seg S = ss[k];
    const double a = ab[2 * k], b = ab[2 * k + 1];
    const long long e0 = (t - sp[k]) * kChunk, e1 = min(e0 + kChunk, S.n);
    for (long long i = e0 + threadIdx.x; i < e1; i += kThreads) S.w[i] = fma(a, S.V[i], b * S.w[i]);
  }
}

// One modified Gram-Schmidt step k for every instance: with AXPY, w -= c V_k where
// c = dots[inst][k] * sc[inst][k] (zero: the instance is left as it is); then the partial of
// <V_k+1, w> (DOTV) or <w, w> over the updated w. V_k = V + k stride of the segment.
template <bool AXPY, bool DOTV>
__global__ void __launch_bounds__(kThreads, kBlocksPerSm) mgs_b(const Seg* __restrict__ segs, const long long* __restrict__ prefix,
                                                  int nj, long long total, int k, const double* __restrict__ dots,
                                                  const double* __restrict__ sc, int ld, double* __restrict__ part) {
  __shared__ double sh[32];
  KKT_SEG_TABLE
  for (long long t = blockIdx.x; t < total; t += gridDim.x) {
    const int q = batch_find(sp, nj, t);
    const Seg S = ss[q];
    const double c = AXPY ? dots[q * ld + k] * sc[q * ld + k] : 0.0;
    const double* Vk = S.V + (AXPY ? k : 0) * S.stride;
    const double* Vn = S.V + (k + 1) * S.stride;
    const long long e0 = (t - sp[q]) * kChunk, e1 = min(e0 + kChunk, S.n);
    const bool ax = AXPY && c != 0.0;
    double acc = 0.0;
    // 4 elements per thread per round, all loads issued before the arithmetic (memory-level
    // parallelism: each thread keeps up to 12 loads in flight)
    for (long long base = e0 + threadIdx.x; base < e1; base += 4 * kThreads) {
      double wv[4], kv[4], nv[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const long long i = base + r * kThreads;
        const bool in = i < e1;
        wv[r] = in ? S.w[i] : 0.0;
        kv[r] = (in && ax) ? Vk[i] : 0.0;
        nv[r] = (in && DOTV) ? Vn[i] : 0.0;
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const long long i = base + r * kThreads;
        if (ax) {
          wv[r] = fma(-c, kv[r], wv[r]);
          if (i < e1) S.w[i] = wv[r];
        }
        acc = fma(DOTV ? nv[r] : wv[r], wv[r], acc);
      }
    }
    const double r = block_sum(acc, sh);
    if (threadIdx.x == 0) part[t] = r;
  }
}

// Paired MGS step over all instances: w -= c0 V_k + c1 V_k+1 (NA of them, c_i = dots[inst][k+i]
// * sc[inst][k+i]), then partial dots <V_k+NA, w>, <V_k+NA+1, w> (ND of them) or <w, w> when
// ND = 0, max(ND, 1) columns per item.
template <int NA, int ND>
__global__ void __launch_bounds__(kThreads, kBlocksPerSm) mgs2_b(const Seg* __restrict__ segs, const long long* __restrict__ prefix,
                                                   int nj, long long total, int k, const double* __restrict__ dots,
                                                   const double* __restrict__ sc, int ld, double* __restrict__ part) {
  __shared__ double sh[32];
  __shared__ double2 sh2[32];
  KKT_SEG_TABLE
  constexpr int W = ND > 1 ? 2 : 1;
  // the partial dots run on across this block's consecutive items of one instance and are
  // reduced over the block once, at its last item of that instance (the other items' slots get
  // zero): no barrier, and no drain of the loads in flight, between items of one instance
  double acc0 = 0.0, acc1 = 0.0;
  for (long long t = blockIdx.x; t < total; t += gridDim.x) {
    const int q = batch_find(sp, nj, t);
    const Seg S = ss[q];
    const double c0 = NA > 0 ? dots[q * ld + k] * sc[q * ld + k] : 0.0;
    const double c1 = NA > 1 ? dots[q * ld + k + 1] * sc[q * ld + k + 1] : 0.0;
    const double* A0 = S.V + k * S.stride;
    const double* A1 = A0 + S.stride;
    const double* B0 = S.V + (k + NA) * S.stride;
    const double* B1 = B0 + S.stride;
    const long long e0 = (t - sp[q]) * kChunk, e1 = min(e0 + kChunk, S.n);
    // 16-byte loads and stores when every vector of the step starts 16-byte aligned (item
    // starts are even: kChunk is); else 8-byte loads
    const uintptr_t al = reinterpret_cast<uintptr_t>(S.w) | reinterpret_cast<uintptr_t>(A0) |
                         reinterpret_cast<uintptr_t>(A1) | reinterpret_cast<uintptr_t>(B0) |
                         reinterpret_cast<uintptr_t>(B1);
    long long scalar_from = e0;
    if ((al & 15) == 0) {
      const long long p0 = e0 / 2, p1 = e1 / 2;   // whole pairs of the item
      double2* w2 = reinterpret_cast<double2*>(S.w);
      const double2* a02 = reinterpret_cast<const double2*>(A0);
      const double2* a12 = reinterpret_cast<const double2*>(A1);
      const double2* b02 = reinterpret_cast<const double2*>(B0);
      const double2* b12 = reinterpret_cast<const double2*>(B1);
      constexpr int RV = NA + ND >= 4 ? 1 : 2;   // 16-byte loads in flight: 5 (or up to 8) per thread
      for (long long base = p0 + threadIdx.x; base < p1; base += RV * kThreads) {
        double2 wv[RV], a0[RV], a1[RV], b0[RV], b1[RV];
#pragma unroll
        for (int r = 0; r < RV; ++r) {
          const long long i = base + r * kThreads;
          const bool in = i < p1;
          const double2 z = make_double2(0.0, 0.0);
          wv[r] = in ? w2[i] : z;
          a0[r] = (in && NA > 0) ? a02[i] : z;
          a1[r] = (in && NA > 1) ? a12[i] : z;
          b0[r] = (in && ND > 0) ? b02[i] : z;
          b1[r] = (in && ND > 1) ? b12[i] : z;
        }
#pragma unroll
        for (int r = 0; r < RV; ++r) {
          const long long i = base + r * kThreads;
          if (NA > 0) {
            wv[r].x = fma(-c0, a0[r].x, wv[r].x);
            wv[r].y = fma(-c0, a0[r].y, wv[r].y);
            if (NA > 1) {
              wv[r].x = fma(-c1, a1[r].x, wv[r].x);
              wv[r].y = fma(-c1, a1[r].y, wv[r].y);
            }
            if (i < p1) w2[i] = wv[r];
          }
          if (ND == 0) {
            acc0 = fma(wv[r].x, wv[r].x, fma(wv[r].y, wv[r].y, acc0));
          } else {
            acc0 = fma(b0[r].x, wv[r].x, fma(b0[r].y, wv[r].y, acc0));
            if (ND > 1) acc1 = fma(b1[r].x, wv[r].x, fma(b1[r].y, wv[r].y, acc1));
          }
        }
      }
      scalar_from = 2 * p1;   // an odd last element of the vector, if any
    }
    constexpr int R = NA + ND >= 4 ? 2 : 4;   // loads in flight per thread within 64 registers
    for (long long base = scalar_from + threadIdx.x; base < e1; base += R * kThreads) {
      double wv[R], a0[R], a1[R], b0[R], b1[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const long long i = base + r * kThreads;
        const bool in = i < e1;
        wv[r] = in ? S.w[i] : 0.0;
        a0[r] = (in && NA > 0) ? A0[i] : 0.0;
        a1[r] = (in && NA > 1) ? A1[i] : 0.0;
        b0[r] = (in && ND > 0) ? B0[i] : 0.0;
        b1[r] = (in && ND > 1) ? B1[i] : 0.0;
      }
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const long long i = base + r * kThreads;
        if (NA > 0) {
          wv[r] = fma(-c0, a0[r], wv[r]);
          if (NA > 1) wv[r] = fma(-c1, a1[r], wv[r]);
          if (i < e1) S.w[i] = wv[r];
        }
        if (ND == 0) {
          acc0 = fma(wv[r], wv[r], acc0);
        } else {
          acc0 = fma(b0[r], wv[r], acc0);
          if (ND > 1) acc1 = fma(b1[r], wv[r], acc1);
        }
      }
    }
    const long long tn = t + gridDim.x;
    if (tn < total && tn < sp[q + 1]) {   // this block's next item is of the same instance
      if (threadIdx.x == 0) {
        part[t * W] = 0.0;
        if (ND > 1) part[t * W + 1] = 0.0;
      }
      continue;
    }
    if (ND > 1) {
      const double2 r = block_sum2(acc0, acc1, sh2);
      if (threadIdx.x == 0) {
        part[t * W] = r.x;
        part[t * W + 1] = r.y;
      }
    } else {
      const double r0 = block_sum(acc0, sh);
      if (threadIdx.x == 0) part[t * W] = r0;
    }
    acc0 = 0.0;
    acc1 = 0.0;
  }
}

// out[inst * ld + col0 + c] = sum over the instance's items of part[t * width + c]
__global__ void finalize_cols_b(const double* __restrict__ part, const long long* __restrict__ prefix, int nj,
                                int width, double* __restrict__ out, int ld, int col0) {
  const int inst = blockIdx.x / width, c = blockIdx.x % width;
  if (inst >= nj) return;
  double acc = 0.0;
  for (long long t = prefix[inst] + threadIdx.x; t < prefix[inst + 1]; t += 32) acc += part[t * width + c];
  acc = warp_sum(acc);
  if (threadIdx.x == 0) out[inst * ld + col0 + c] = acc;
}

// out[inst * ld + col] = sum of part[t] over the instance's items
__global__ void finalize_col_b(const double* __restrict__ part, const long long* __restrict__ prefix, int nj,
                               double* __restrict__ out, int ld, int col) {
  const int inst = blockIdx.x;
  if (inst >= nj) return;
  double acc = 0.0;
  for (long long t = prefix[inst] + threadIdx.x; t < prefix[inst + 1]; t += 32) acc += part[t];
  acc = warp_sum(acc);
  if (threadIdx.x == 0) out[inst * ld + col] = acc;
}

// out[inst][v] = sum of part[t][v] over the instance's items, one warp per (inst, v)
__global__ void finalize_b(const double* __restrict__ part, const long long* __restrict__ prefix, int nj, int width,
                           double* __restrict__ out) {
  const int inst = blockIdx.x / width, v = blockIdx.x % width;
  if (inst >= nj) return;
  double acc = 0.0;
  for (long long t = prefix[inst] + threadIdx.x; t < prefix[inst + 1]; t += 32) acc += part[t * width + v];
  acc = warp_sum(acc);
  if (threadIdx.x == 0) out[inst * width + v] = acc;
}

template <template <int> class Run, typename... A>
int dispatch(int count, A... a) {
  switch (count) {
#define KKT_B_CASE(k) \
  case k:             \
    return Run<k>::go(a...);
    KKT_B_CASE(0) KKT_B_CASE(1) KKT_B_CASE(2) KKT_B_CASE(3) KKT_B_CASE(4) KKT_B_CASE(5) KKT_B_CASE(6)
    KKT_B_CASE(7) KKT_B_CASE(8) KKT_B_CASE(9) KKT_B_CASE(10) KKT_B_CASE(11) KKT_B_CASE(12) KKT_B_CASE(13)
    KKT_B_CASE(14) KKT_B_CASE(15) KKT_B_CASE(16) KKT_B_CASE(17) KKT_B_CASE(18) KKT_B_CASE(19) KKT_B_CASE(20)
    KKT_B_CASE(21) KKT_B_CASE(22) KKT_B_CASE(23) KKT_B_CASE(24) KKT_B_CASE(25) KKT_B_CASE(26) KKT_B_CASE(27)
    KKT_B_CASE(28) KKT_B_CASE(29) KKT_B_CASE(30) KKT_B_CASE(31) KKT_B_CASE(32)
#undef KKT_B_CASE
    default:
      return set_error(KKT_ERR_INVALID_ARG, "batched Krylov: vector count out of range");
  }
}

int persistent_grid(int per_sm = kBlocksPerSm) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return std::max(sms, 1) * per_sm;
}

template <int NV>
struct MultidotB {
  static int go(const Seg* s, const long long* p, int nj, long long tot, double* part, double flops, cudaStream_t st) {
    ProfScope ps(KKT_K_MULTIDOT, st, flops * (NV + 1), 8.0 * flops / 2 * (NV + 1));
    multidot_b<NV><<<static_cast<unsigned>(std::min<long long>(tot, persistent_grid(blocks_per_sm(NV)))), kThreads, 0,
                     st>>>(s, p, nj, tot, part);
    KKT_CUDA_TRY(cudaGetLastError());
    return KKT_OK;
  }
};

template <int NV>
struct UpdateB {
  static int go(const Seg* s, const long long* p, int nj, long long tot, const double* coef, int ldc, double* part,
                int want_norm, double flops, cudaStream_t st) {
    ProfScope ps(NV > 0 ? KKT_K_UPDATE : KKT_K_REDUCE, st, flops * (NV + 1), 8.0 * flops / 2 * (NV > 0 ? NV + 2 : 1));
    update_b<NV><<<static_cast<unsigned>(std::min<long long>(tot, persistent_grid(blocks_per_sm(NV)))), kThreads, 0, st>>>(
        s, p, nj, tot, coef, ldc, part, want_norm);
    KKT_CUDA_TRY(cudaGetLastError());
    return KKT_OK;
  }
};

// device + pinned host tables of one family of segments (e.g. "the new basis vector of every
// instance against its basis")
struct SegTable {
  int nj = 0;
  Seg* dev = nullptr;
  long long* prefix = nullptr;
  long long total = 0;
  double elems = 0;
  int set(const std::vector<Seg>& segs) {
    nj = static_cast<int>(segs.size());
    std::vector<long long> pre(nj + 1, 0);
    elems = 0;
    for (int k = 0; k < nj; ++k) {
      pre[k + 1] = pre[k] + (segs[k].n + kChunk - 1) / kChunk;
      elems += static_cast<double>(segs[k].n);
    }
    total = pre[nj];
    if (nj < 1 || nj > KKT_BATCH_MAX) return set_error(KKT_ERR_INVALID_ARG, "segment table size out of range");
    if (!dev) {   // capacity for the largest batch: the table is refilled with other counts
      KKT_CUDA_TRY(cudaMalloc(&dev, KKT_BATCH_MAX * sizeof(Seg)));
      KKT_CUDA_TRY(cudaMalloc(&prefix, (KKT_BATCH_MAX + 1) * sizeof(long long)));
    }
    KKT_CUDA_TRY(cudaMemcpy(dev, segs.data(), nj * sizeof(Seg), cudaMemcpyHostToDevice));
    KKT_CUDA_TRY(cudaMemcpy(prefix, pre.data(), (nj + 1) * sizeof(long long), cudaMemcpyHostToDevice));
    return KKT_OK;
  }
  void free() {
    cudaFree(dev);
    cudaFree(prefix);
    dev = nullptr;
    prefix = nullptr;
  }
};

}  // namespace
}  // namespace kkt

struct kkt_batch {
  std::vector<kkt_handle*> inst;
  kkt_options opt;
  int tuned_tile_lines = 0;   // 0 = not tuned yet
  int tuned_sweep_tb = 0;
  double tune_ms_dst[3] = {0, 0, 0};
  double tune_ms_sweep[3] = {0, 0, 0};
  long long mem_limit = 0;    // bytes of Krylov storage per wave; 0: 85% of the free device memory
  int use_graphs = 1;         // replay the preconditioner + matvec phase as CUDA graphs
  long long single_threshold = 1LL << 20;   // V at or above which an instance is solved alone
};

using namespace kkt;

namespace {

// One instance's FGMRES state inside a wave.
struct InstState {
  kkt_handle* h;
  const double* f;
  double* x;
  double du, dz, dw;
  double fnorm = 0, beta = 0;
  int its = 0, restarts = 0, status = 1, active = 1, jused = 0, cycle_done = 0;
  std::vector<double> H, cs, sn, g, eta, y, hist;
  double rel = 0;
};

}  // namespace

extern "C" {

kkt_batch* kkt_batch_create(int count, const kkt_instance* desc, const kkt_options* opt) {
  if (count < 1 || count > KKT_BATCH_MAX || !desc) {
    set_error(KKT_ERR_INVALID_ARG, "need 1 to KKT_BATCH_MAX instances");
    return nullptr;
  }
  kkt_options o;
  kkt_default_options(&o);
  if (opt) o = *opt;
  if (o.orth == KKT_ORTH_MGS4 || o.orth == KKT_ORTH_MGS8) {
    set_error(KKT_ERR_UNSUPPORTED, "the batched form orthogonalises with MGS, paired MGS or CGS2");
    return nullptr;
  }
  if (o.precision != KKT_PREC_FP64 || o.coarse == KKT_COARSE_LEARNED) {
    set_error(KKT_ERR_UNSUPPORTED, "the batched form runs the FP64 exact or one-level preconditioner");
    return nullptr;
  }
  kkt_batch* b = new kkt_batch();
  b->opt = o;
  for (int i = 0; i < count; ++i) {
    const kkt_instance& d = desc[i];
    kkt_handle* h = kkt_create(d.nx, d.ny, d.Nt, d.T, d.nu, d.omega, d.n_sub);
    if (!h || kkt_set_options(h, &o) < 0) {
      const std::string msg = std::string("instance ") + std::to_string(i) + ": " + kkt_last_error();
      if (h) kkt_destroy(h);
      kkt_batch_destroy(b);
      set_error(KKT_ERR_INVALID_ARG, msg);
      return nullptr;
    }
    b->inst.push_back(h);
  }
  return b;
}

void kkt_batch_destroy(kkt_batch* b) {
  if (!b) return;
  for (kkt_handle* h : b->inst) kkt_destroy(h);
  delete b;
}

int kkt_batch_set_graphs(kkt_batch* b, int on) {
  if (!b) return set_error(KKT_ERR_INVALID_ARG, "null batch");
  b->use_graphs = on != 0;
  return KKT_OK;
}

int kkt_batch_set_dst_method(kkt_batch* b, int method) {
  if (!b) return set_error(KKT_ERR_INVALID_ARG, "null batch");
  for (size_t i = 0; i < b->inst.size(); ++i) {
    const int rc = kkt_set_dst_method(b->inst[i], method);
    if (rc < 0) return set_error(rc, std::string("instance ") + std::to_string(i) + ": " + kkt_last_error());
  }
  return KKT_OK;
}

int kkt_batch_set_single_threshold(kkt_batch* b, long long points) {
  if (!b || points < 0) return set_error(KKT_ERR_INVALID_ARG, "bad single-solve threshold");
  b->single_threshold = points;
  return KKT_OK;
}

int kkt_batch_set_memory_limit(kkt_batch* b, long long bytes) {
  if (!b || bytes < 0) return set_error(KKT_ERR_INVALID_ARG, "bad memory limit");
  b->mem_limit = bytes;
  return KKT_OK;
}

int kkt_batch_get_info(const kkt_batch* b, int i, kkt_info* info) {
  if (!b || i < 0 || i >= static_cast<int>(b->inst.size())) return set_error(KKT_ERR_INVALID_ARG, "bad instance index");
  return kkt_get_info(b->inst[i], info);
}

int kkt_batch_solve(kkt_batch* b, const double* const* f, double* const* x, double tol, int maxit,
                    kkt_batch_stats* stats, void* stream) {
  if (!b || !f || !x) return set_error(KKT_ERR_INVALID_ARG, "null argument");
  if (!(tol > 0.0) || maxit < 1) return set_error(KKT_ERR_INVALID_ARG, "bad tol or maxit");
  const auto t_start = std::chrono::steady_clock::now();
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int n_inst = static_cast<int>(b->inst.size());
  const int m = b->opt.restart;
  const bool l2 = b->opt.residual_norm == KKT_NORM_L2;
  // memory waves: first-fit by decreasing size against the free device memory
  size_t free_b = 0, total_b = 0;
  KKT_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
  double budget = 0.85 * static_cast<double>(free_b);
  if (b->mem_limit > 0) budget = std::min(budget, static_cast<double>(b->mem_limit));
  const bool spectral = b->opt.basis == KKT_BASIS_SPECTRAL;
  // instances that fill the GPU alone: kkt_solve's path, one after another, before the waves
  std::vector<int> order, solo;
  for (int i = 0; i < n_inst; ++i)
    if (b->single_threshold > 0 && b->inst[i]->g.V >= b->single_threshold) solo.push_back(i);
    else order.push_back(i);
  std::vector<int> solo_its(n_inst, 0), solo_status(n_inst, KKT_OK);
  std::vector<double> solo_rel(n_inst, 0.0);
  if (!solo.empty()) {
    // one Krylov arena (and spectral copies) sized for the largest of them, lent to each
    // handle in turn: a single allocation instead of one per instance
    long long vmax = 0;
    for (int i : solo) vmax = std::max(vmax, b->inst[i]->g.V);
    double *sv = nullptr, *sz = nullptr, *sf = nullptr, *sx = nullptr;
    int rc = KKT_OK;
    if (cudaMalloc(&sv, sizeof(double) * (m + 1) * 3 * vmax) != cudaSuccess ||
        cudaMalloc(&sz, sizeof(double) * m * vmax) != cudaSuccess ||
        (spectral && (cudaMalloc(&sf, sizeof(double) * 3 * vmax) != cudaSuccess ||
                      cudaMalloc(&sx, sizeof(double) * 3 * vmax) != cudaSuccess)))
      rc = set_error(KKT_ERR_OOM, "single-solve Krylov arena");
    for (size_t q = 0; q < solo.size() && rc == KKT_OK; ++q) {
      const int i = solo[q];
      kkt_handle* h = b->inst[i];
      release_krylov(h);
      h->kV = sv;
      h->kZw = sz;
      h->ks_f = sf;
      h->ks_x = sx;
      h->kry_restart = m;
      kkt_stats ks;
      const int r = kkt_solve(h, f[i], x[i], tol, maxit, &ks, stream);
      h->kV = h->kZw = h->ks_f = h->ks_x = nullptr;   // borrowed: not freed with the handle
      h->kry_restart = 0;
      if (r < 0 && r != KKT_ERR_NONFINITE) rc = r;
      solo_its[i] = ks.iterations;
      solo_status[i] = r;
      solo_rel[i] = ks.rel_residual;
    }
    cudaFree(sv);
    cudaFree(sz);
    cudaFree(sf);
    cudaFree(sx);
    if (rc < 0) return rc;
  }
  // spectral basis: f and x run on sine-mode coefficients (x transformed in place, f into a copy)
  auto need = [&](int i) {
    return 8.0 * ((m + 1) * 3.0 + m + (spectral ? 3.0 : 0.0)) * static_cast<double>(b->inst[i]->g.V);
  };
  std::sort(order.begin(), order.end(), [&](int a, int c) { return need(a) > need(c); });
  std::vector<std::vector<int>> waves;
  std::vector<double> wave_mem;
  for (int i : order) {
    if (need(i) > budget) return set_error(KKT_ERR_OOM, "an instance's Krylov basis does not fit in device memory");
    bool placed = false;
    for (size_t w = 0; w < waves.size() && !placed; ++w)
      if (wave_mem[w] + need(i) <= budget) {
        waves[w].push_back(i);
        wave_mem[w] += need(i);
        placed = true;
      }
    if (!placed) {
      waves.push_back({i});
      wave_mem.push_back(need(i));
    }
  }
  double* h_tmp = nullptr;   // pinned: reductions and coefficients
  const int ldc = 64;
  KKT_CUDA_TRY(cudaMallocHost(&h_tmp, sizeof(double) * (3 * ldc * n_inst + 2 * 33 * n_inst + 4 * n_inst)));
  double* d_small = nullptr;
  KKT_CUDA_TRY(cudaMalloc(&d_small, sizeof(double) * (3 * ldc * n_inst + 33 * n_inst + 4 * n_inst)));
  double* d_coef = d_small;                       // [3][n][ldc]
  double* d_out = d_coef + 3 * ldc * n_inst;      // [n][33]
  double* d_scale = d_out + 33 * n_inst;          // [n] 1 / eta
  double* d_ab = d_scale + n_inst;                // [n][2]
  double* h_coef = h_tmp;
  double* h_out = h_coef + 3 * ldc * n_inst;
  double* h_scale = h_out + 2 * 33 * n_inst;
  int waves_done = 0, graphs_made = 0;
  long long graph_launches = 0;
  int rc_all = KKT_OK;
  std::vector<InstState> all(n_inst);
  // One Krylov arena for the whole call, sized for the largest wave and carved anew for each
  // wave (every buffer 256-byte aligned): no device allocation between waves.
  auto carve = [](long long doubles) { return (doubles + 31) / 32 * 32; };
  auto inst_doubles = [&](int i) {
    const long long V = b->inst[i]->g.V;
    return carve((m + 1) * 3 * V) + carve(m * V) + (spectral ? carve(3 * V) : 0);
  };
  long long arena_doubles = 0;
  for (const auto& wave : waves) {
    long long t = 0;
    for (int i : wave) t += inst_doubles(i);
    arena_doubles = std::max(arena_doubles, t);
  }
  double* arena = nullptr;
  if (arena_doubles > 0 && cudaMalloc(&arena, sizeof(double) * static_cast<size_t>(arena_doubles)) != cudaSuccess) {
    cudaGetLastError();
    cudaFreeHost(h_tmp);
    cudaFree(d_small);
    return set_error(KKT_ERR_OOM, "batched Krylov arena");
  }
  for (const auto& wave : waves) {
    const int nw = static_cast<int>(wave.size());
    // per-instance Krylov storage, carved from the arena
    std::vector<double*> Vb(nw, nullptr), Zw(nw, nullptr), Fs(nw, nullptr);
    std::vector<InstState*> S(nw);
    double* part = nullptr;
    long long max_items = 0;
    int rc = KKT_OK;
    long long cursor = 0;
    for (int k = 0; k < nw && rc == KKT_OK; ++k) {
      kkt_handle* h = b->inst[wave[k]];
      const long long V = h->g.V;
      Vb[k] = arena + cursor;
      cursor += carve((m + 1) * 3 * V);
      Zw[k] = arena + cursor;
      cursor += carve(m * V);
      if (spectral) {
        Fs[k] = arena + cursor;
        cursor += carve(3 * V);
      }
      max_items += (3 * V + kChunk - 1) / kChunk;
      InstState& I = all[wave[k]];
      I.h = h;
      I.f = f[wave[k]];
      I.x = x[wave[k]];
      I.du = l2 ? 1.0 / std::sqrt(h->g.h) : 1.0;
      I.dz = I.du;
      I.dw = l2 ? std::sqrt(h->g.h) : 1.0;
      I.H.assign((m + 1) * m, 0.0);
      I.cs.assign(m, 0.0);
      I.sn.assign(m, 0.0);
      I.g.assign(m + 1, 0.0);
      I.eta.assign(m + 1, 0.0);
      I.y.assign(m, 0.0);
      S[k] = &I;
    }
    // into the sine-mode basis: f -> Fs (copy), x in place (each block by the orthonormal 2D
    // DST-I, its own inverse); f then means Fs for the rest of the wave
    for (int k = 0; k < nw && rc == KKT_OK && spectral; ++k) {
      const long long V = S[k]->h->g.V;
      for (int bl = 0; bl < 3 && rc == KKT_OK; ++bl) {
        rc = dst2d(S[k]->h, S[k]->f + bl * V, Fs[k] + bl * V, st);
        if (rc == KKT_OK) rc = dst2d(S[k]->h, S[k]->x + bl * V, S[k]->x + bl * V, st);
      }
      S[k]->f = Fs[k];
    }
    if (rc == KKT_OK && cudaMalloc(&part, sizeof(double) * max_items * 33) != cudaSuccess)
      rc = set_error(KKT_ERR_OOM, "batched reduction scratch");
    std::vector<BatchSlot> slots(m);
    BatchSlot resid_slot, sub_slot;
    std::vector<cudaGraphExec_t> graphs(m, nullptr);
    std::vector<ProfCapture> graph_work(m);
    SegTable t_full, t_new, t_f[3], t_xu, t_xz, t_xw;
    auto Hs = [&](InstState& I, int i, int j) -> double& { return I.H[static_cast<size_t>(i) * m + j]; };
    auto fetch = [&](int cnt) -> int {
      KKT_CUDA_TRY(cudaMemcpyAsync(h_out, d_out, sizeof(double) * cnt, cudaMemcpyDeviceToHost, st));
      KKT_CUDA_TRY(cudaStreamSynchronize(st));
      return KKT_OK;
    };
    // per-instance sums of the per-item partials (width columns) into h_out[k * width + v]
    auto finalize = [&](const SegTable& t, int width) -> int {
      {
        ProfScope ps(KKT_K_REDUCE, st);
        finalize_b<<<t.nj * width, 32, 0, st>>>(part, t.prefix, t.nj, width, d_out);
        KKT_CUDA_TRY(cudaGetLastError());
      }
      return fetch(t.nj * width);
    };
    // per-instance squared norms of segment tables into h_out[k]
    auto norms = [&](SegTable& t) -> int {
      KKT_TRY(dispatch<UpdateB>(0, t.dev, t.prefix, t.nj, t.total, d_coef, ldc, part, 1, 2.0 * t.elems, st));
      return finalize(t, 1);
    };
    // preconditioner + matvec tables of step j (pointers fixed per j)
    // matvec job y = diag(du, dz, dw) K (su u, sz z, w), su, sz scaled by scale_dev[k] at run time
    auto fill_matvec = [&](MatvecJob& M, int k, const double* u, const double* z, const double* w, double* y,
                           double su, double sz) {
      InstState& I = *S[k];
      const Geometry& g = I.h->g;
      M.u = u;
      M.z = z;
      M.w = w;
      M.y = y;
      M.Mx = g.Mx;
      M.My = g.My;
      M.Nt = g.Nt;
      M.N = g.N;
      M.V = g.V;
      const double c0 = spectral ? 1.0 : 1.0 + 2.0 * g.cx + 2.0 * g.cy;
      const double cx = spectral ? 0.0 : g.cx, cy = spectral ? 0.0 : g.cy;
      M.uu = I.du * g.h * su;
      M.wc0 = I.du * c0;
      M.wcx = I.du * cx;
      M.wcy = I.du * cy;
      M.wn = I.du;
      M.zz = I.dz * g.omega * g.h * sz;
      M.zw = I.dz * g.dt;
      M.uc0 = I.dw * su * c0;
      M.ucx = I.dw * su * cx;
      M.ucy = I.dw * su * cy;
      M.up = I.dw * su;
      M.wz = I.dw * g.dt * sz;
      M.scale_index = k;
      M.spectral = spectral ? 1 : 0;
      M.lx = I.h->d_lx;
      M.ly = I.h->d_ly;
      M.dtnu = g.dtnu;
    };
    std::vector<int> everyone(nw);
    std::iota(everyone.begin(), everyone.end(), 0);
    // preconditioner + matvec tables of step j for the wave instances in `mem`
    auto prepare_slot = [&](BatchSlot& sl, int j, const std::vector<int>& mem) -> int {
      sl.sweep_tb = b->tuned_sweep_tb > 0 ? b->tuned_sweep_tb : 128;
      const int nm = static_cast<int>(mem.size());
      std::vector<DstJob> fwd, inv;
      sl.oz_jobs[0].clear();
      sl.oz_jobs[1].clear();
      std::vector<SpecJob> sj(nm);
      std::vector<MatvecJob> mj(nm);
      for (int q = 0; q < nm; ++q) {
        const int k = mem[q];
        InstState& I = *S[k];
        kkt_handle* h = I.h;
        const Geometry& g = h->g;
        const long long V = g.V;
        double* Vj = Vb[k] + static_cast<size_t>(j) * 3 * V;
        double* Zj = Zw[k] + static_cast<size_t>(j) * V;
        const bool alone = dst_tensor_fills_gpu(h);
        (alone ? sl.oz_jobs[0] : fwd).push_back(DstJob{h, Vj + 2 * V, h->spec});
        (alone ? sl.oz_jobs[1] : inv).push_back(DstJob{h, h->spec2, Zj});
        SpecJob& J = sj[q];
        J.p = make_spec_params(h);
        J.rhat = spectral ? Vj + 2 * V : h->spec;   // the spectral basis needs no transforms
        J.yhat = spectral ? Zj : h->spec2;
        J.cc = h->coarse_c;
        J.cy = h->coarse_w;
        J.scale_base = 1.0 / I.dw;
        J.max_len = h->td.max_len;
        J.scale_index = k;
        fill_matvec(mj[q], k, Vj, Vj + V, Zj, Vj + 3 * V, 1.0 / (g.h * I.du), 1.0 / (g.omega * g.h * I.dz));
      }
      const int tl = b->tuned_tile_lines;
      if (!spectral) {
        KKT_TRY(dst_batched_prepare(sl, 0, fwd.data(), static_cast<int>(fwd.size()), tl));
        KKT_TRY(dst_batched_prepare(sl, 2, inv.data(), static_cast<int>(inv.size()), tl));
      }
      KKT_TRY(spectral_batched_prepare(sl, sj.data(), nm));
      KKT_TRY(matvec_batched_prepare(sl, mj.data(), nm));
      return KKT_OK;
    };
    auto phase_launch = [&](const BatchSlot& sl, cudaStream_t s2) -> int {
      if (spectral) {
        KKT_TRY(spectral_batched_launch(sl, d_scale, s2));
        return matvec_batched_launch(sl, d_scale, s2);
      }
      KKT_TRY(dst_batched_launch(sl, 0, s2));
      KKT_TRY(dst_batched_launch(sl, 1, s2));
      for (const DstJob& d : sl.oz_jobs[0]) KKT_TRY(oz_dst2d(d.h->oz, d.in, d.out, s2));
      KKT_TRY(spectral_batched_launch(sl, d_scale, s2));
      KKT_TRY(dst_batched_launch(sl, 2, s2));
      KKT_TRY(dst_batched_launch(sl, 3, s2));
      for (const DstJob& d : sl.oz_jobs[1]) KKT_TRY(oz_dst2d(d.h->oz, d.in, d.out, s2));
      KKT_TRY(matvec_batched_launch(sl, d_scale, s2));
      return KKT_OK;
    };
    // autotune once per batch on the first wave: sine-transform tile height, sweep block size.
    // Candidates that a wave's sizes rule out (shared memory) are skipped.
    // the sweep block is re-tuned on every wave (its shared memory depends on the wave's
    // longest subdomain); the transform tile height once per batch
    const bool tune_tiles = b->tuned_tile_lines == 0;
    if (rc == KKT_OK) {
      const int cand_tl[3] = {8, 16, 32}, cand_tb[3] = {64, 128, 256};
      if (tune_tiles)
        for (int a = 0; a < 3; ++a) b->tune_ms_dst[a] = 0.0;
      cudaEvent_t e0 = nullptr, e1 = nullptr;
      KKT_CUDA_TRY(cudaEventCreate(&e0));
      KKT_CUDA_TRY(cudaEventCreate(&e1));
      for (int k = 0; k < nw; ++k) KKT_CUDA_TRY(cudaMemsetAsync(Vb[k], 0, sizeof(double) * 3 * S[k]->h->g.V, st));
      for (int k = 0; k < nw; ++k) h_scale[k] = 1.0;
      KKT_CUDA_TRY(cudaMemcpyAsync(d_scale, h_scale, sizeof(double) * nw, cudaMemcpyHostToDevice, st));
      KKT_CUDA_TRY(cudaStreamSynchronize(st));
      // mean ms of two runs of body (1e30 if a launch was refused, e.g. too much shared memory)
      auto time_it = [&](auto&& body) -> double {
        bool ok = true;
        cudaEventRecord(e0, st);
        for (int r = 0; r < 2 && ok; ++r) ok = body() == KKT_OK;
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (!ok) cudaGetLastError();
        return ok ? ms / 2.0 : 1e30;
      };
      int best_tl = 1, best_tb = 1;
      for (int a = 0; a < 3 && !spectral && tune_tiles; ++a) {   // (no transforms in the spectral basis)
        b->tuned_tile_lines = cand_tl[a];
        b->tuned_sweep_tb = 128;
        b->tune_ms_dst[a] = 1e30;
        if (prepare_slot(slots[0], 0, everyone) == KKT_OK)
          b->tune_ms_dst[a] = time_it([&] {
            const int r = dst_batched_launch(slots[0], 0, st);
            return r != KKT_OK ? r : dst_batched_launch(slots[0], 1, st);
          });
        batch_slot_free(slots[0]);
        if (b->tune_ms_dst[a] < b->tune_ms_dst[best_tl]) best_tl = a;
      }
      if (tune_tiles) b->tuned_tile_lines = cand_tl[best_tl];
      for (int a = 0; a < 3; ++a) {
        b->tuned_sweep_tb = cand_tb[a];
        b->tune_ms_sweep[a] = 1e30;
        // (the first candidate also runs the forward transform once, so the sweeps read data)
        auto forward = [&]() -> int {
          KKT_TRY(dst_batched_launch(slots[0], 0, st));
          KKT_TRY(dst_batched_launch(slots[0], 1, st));
          for (const DstJob& d : slots[0].oz_jobs[0]) KKT_TRY(oz_dst2d(d.h->oz, d.in, d.out, st));
          return KKT_OK;
        };
        if (prepare_slot(slots[0], 0, everyone) == KKT_OK && (a > 0 || forward() == KKT_OK))
          b->tune_ms_sweep[a] = time_it([&] { return spectral_batched_launch(slots[0], d_scale, st); });
        batch_slot_free(slots[0]);
        if (b->tune_ms_sweep[a] < b->tune_ms_sweep[best_tb]) best_tb = a;
      }
      b->tuned_sweep_tb = cand_tb[best_tb];
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      const cudaError_t e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) rc = set_error(KKT_ERR_CUDA, std::string("autotuning: ") + cudaGetErrorString(e));
      else if ((tune_tiles && b->tune_ms_dst[best_tl] >= 1e30) || b->tune_ms_sweep[best_tb] >= 1e30)
        rc = set_error(KKT_ERR_UNSUPPORTED, "batched form: no tile or sweep block fits this wave");
      else
        set_error(KKT_OK, "");
    }
    // static segment tables of the wave: full vectors f and x blocks
    std::vector<Seg> sf[3], sxu, sxz, sxw;
    for (int k = 0; k < nw && rc == KKT_OK; ++k) {
      const long long V = S[k]->h->g.V;
      for (int bl = 0; bl < 3; ++bl) sf[bl].push_back(Seg{S[k]->f + bl * V, 0, Vb[k] + bl * V, V});
      sxu.push_back(Seg{Vb[k], 3 * V, S[k]->x, V});
      sxz.push_back(Seg{Vb[k] + V, 3 * V, S[k]->x + V, V});
      sxw.push_back(Seg{Zw[k], V, S[k]->x + 2 * V, V});
    }
    if (rc == KKT_OK) {
      for (int bl = 0; bl < 3 && rc == KKT_OK; ++bl) rc = t_f[bl].set(sf[bl]);
      if (rc == KKT_OK) rc = t_xu.set(sxu);
      if (rc == KKT_OK) rc = t_xz.set(sxz);
      if (rc == KKT_OK) rc = t_xw.set(sxw);
    }
    // residual: V_0 = D (f - K x): matvec of x (scales 1) then V_0 = d f - V_0, blockwise
    auto residual = [&]() -> int {
      std::vector<MatvecJob> mj(nw);
      for (int k = 0; k < nw; ++k) {
        const long long V = S[k]->h->g.V;
        fill_matvec(mj[k], k, S[k]->x, S[k]->x + V, S[k]->x + 2 * V, Vb[k], 1.0, 1.0);
        h_scale[k] = 1.0;
      }
      KKT_CUDA_TRY(cudaMemcpyAsync(d_scale, h_scale, sizeof(double) * nw, cudaMemcpyHostToDevice, st));
      KKT_TRY(matvec_batched_prepare(resid_slot, mj.data(), nw));
      KKT_TRY(matvec_batched_launch(resid_slot, d_scale, st));
      for (int bl = 0; bl < 3; ++bl) {
        for (int k = 0; k < nw; ++k) {
          const double d = bl == 0 ? S[k]->du : (bl == 1 ? S[k]->dz : S[k]->dw);
          h_coef[2 * k] = d;
          h_coef[2 * k + 1] = -1.0;
        }
        KKT_CUDA_TRY(cudaMemcpyAsync(d_ab, h_coef, sizeof(double) * 2 * nw, cudaMemcpyHostToDevice, st));
        ProfScope ps(KKT_K_AXPY, st, 3.0 * t_f[bl].elems, 24.0 * t_f[bl].elems);
        axpby_b<<<static_cast<unsigned>(std::min<long long>(t_f[bl].total, persistent_grid())), kThreads, 0, st>>>(
            t_f[bl].dev, t_f[bl].prefix, nw, t_f[bl].total, d_ab);
        KKT_CUDA_TRY(cudaGetLastError());
        KKT_CUDA_TRY(cudaStreamSynchronize(st));
      }
      std::vector<Seg> s0(nw);
      for (int k = 0; k < nw; ++k) s0[k] = Seg{Vb[k], 0, Vb[k], 3 * S[k]->h->g.V};
      KKT_TRY(t_full.set(s0));
      KKT_TRY(norms(t_full));
      for (int k = 0; k < nw; ++k) S[k]->beta = std::sqrt(h_out[k]);
      return KKT_OK;
    };
    // right-hand side norms (weighted)
    if (rc == KKT_OK) {
      std::vector<double> acc(nw, 0.0);
      for (int bl = 0; bl < 3 && rc == KKT_OK; ++bl) {
        std::vector<Seg> sfb(nw);
        for (int k = 0; k < nw; ++k) sfb[k] = Seg{S[k]->f + bl * S[k]->h->g.V, 0, const_cast<double*>(S[k]->f) + bl * S[k]->h->g.V, S[k]->h->g.V};
        SegTable tt;
        rc = tt.set(sfb);
        if (rc == KKT_OK) rc = norms(tt);
        for (int k = 0; k < nw && rc == KKT_OK; ++k) {
          const double d = bl == 0 ? S[k]->du : (bl == 1 ? S[k]->dz : S[k]->dw);
          acc[k] += d * d * h_out[k];
        }
        tt.free();
      }
      for (int k = 0; k < nw; ++k) S[k]->fnorm = std::sqrt(acc[k]);
    }
    if (rc == KKT_OK) rc = residual();
    for (int k = 0; k < nw && rc == KKT_OK; ++k) {
      InstState& I = *S[k];
      if (!std::isfinite(I.fnorm) || !std::isfinite(I.beta)) {
        I.status = KKT_ERR_NONFINITE;
        I.active = 0;
      } else if (I.fnorm == 0.0 || I.beta / I.fnorm <= tol) {
        I.rel = I.fnorm == 0.0 ? 0.0 : I.beta / I.fnorm;
        I.status = KKT_OK;
        I.active = 0;
      }
    }
    // restart cycles in lockstep
    while (rc == KKT_OK) {
      int n_active = 0;
      for (int k = 0; k < nw; ++k) n_active += S[k]->active;
      if (n_active == 0) break;
      for (int k = 0; k < nw; ++k) {
        InstState& I = *S[k];
        std::fill(I.H.begin(), I.H.end(), 0.0);
        std::fill(I.g.begin(), I.g.end(), 0.0);
        I.g[0] = I.beta;
        I.eta[0] = I.beta > 0 ? I.beta : 1.0;
        I.jused = 0;
        I.cycle_done = !I.active;
      }
      for (int j = 0; j < m && rc == KKT_OK; ++j) {
        // instances still iterating in this cycle; the others are left out of every launch
        std::vector<int> mem;
        for (int k = 0; k < nw; ++k)
          if (!S[k]->cycle_done) mem.push_back(k);
        const int nr = static_cast<int>(mem.size());
        if (nr == 0) break;
        for (int k = 0; k < nw; ++k) h_scale[k] = 1.0 / S[k]->eta[j];
        KKT_CUDA_TRY(cudaMemcpyAsync(d_scale, h_scale, sizeof(double) * nw, cudaMemcpyHostToDevice, st));
        if (nr < nw || !b->use_graphs) {
          // a subset (or graphs off): tables for the running instances, direct launches
          rc = prepare_slot(sub_slot, j, mem);
          if (rc == KKT_OK) rc = phase_launch(sub_slot, st);
          if (rc != KKT_OK) break;
        } else {
          if (slots[j].njobs == 0) {
            rc = prepare_slot(slots[j], j, everyone);
            if (rc != KKT_OK) break;
          }
          if (!graphs[j]) {
            cudaStream_t cs_ = nullptr;
            KKT_CUDA_TRY(cudaStreamCreateWithFlags(&cs_, cudaStreamNonBlocking));
            cudaGraph_t gr = nullptr;
            KKT_CUDA_TRY(cudaStreamBeginCapture(cs_, cudaStreamCaptureModeRelaxed));
            graph_work[j] = ProfCapture();
            prof_capture(&graph_work[j]);
            const int prc = phase_launch(slots[j], cs_);
            prof_capture(nullptr);
            const cudaError_t ec = cudaStreamEndCapture(cs_, &gr);
            cudaStreamDestroy(cs_);
            if (prc < 0 || ec != cudaSuccess) {
              rc = set_error(KKT_ERR_CUDA, "graph capture of the batched phase failed");
              break;
            }
            KKT_CUDA_TRY(cudaGraphInstantiate(&graphs[j], gr, 0));
            cudaGraphDestroy(gr);
            ++graphs_made;
          }
          rc = prof_graph_launch(graphs[j], graph_work[j], st);
          if (rc != KKT_OK) break;
          ++graph_launches;
        }
        // Gram-Schmidt of the new vectors of the running instances (position q = mem index)
        std::vector<Seg> sn(nr);
        for (int q = 0; q < nr; ++q) {
          const int k = mem[q];
          const long long V = S[k]->h->g.V;
          sn[q] = Seg{Vb[k], 3 * V, Vb[k] + static_cast<size_t>(j + 1) * 3 * V, 3 * V};
        }
        rc = t_new.set(sn);
        if (rc != KKT_OK) break;
        std::vector<double> wn2(nw, 0.0), before(nr, 0.0);
        std::vector<char> need(nr, 1);
        if (b->opt.orth == KKT_ORTH_MGS2) {
          // paired MGS over all running instances: one pass subtracts a pair of basis vectors
          // and takes the next pair's dots (as kkt_solve does)
          for (int q = 0; q < nr; ++q)
            for (int i = 0; i <= j; ++i) h_coef[q * 33 + i] = 1.0 / (S[mem[q]]->eta[i] * S[mem[q]]->eta[i]);
          KKT_CUDA_TRY(cudaMemcpyAsync(d_coef, h_coef, sizeof(double) * 33 * nr, cudaMemcpyHostToDevice, st));
          const unsigned grid = static_cast<unsigned>(std::min<long long>(t_new.total, persistent_grid()));
          auto step = [&](int na, int nd, int k) -> int {
            const double el = t_new.elems;
            {
              ProfScope ps(na > 0 ? KKT_K_UPDATE : KKT_K_MULTIDOT, st, 2.0 * el * (na + (nd > 0 ? nd : 1)),
                           8.0 * el * (na + nd + 1 + (na > 0 ? 1 : 0)));
#define KKT_MGS2B(NA_, ND_)                                                                                     \
  if (na == NA_ && nd == ND_)                                                                                   \
    mgs2_b<NA_, ND_><<<grid, kThreads, 0, st>>>(t_new.dev, t_new.prefix, nr, t_new.total, k, d_out, d_coef, 33, part);
              KKT_MGS2B(0, 1) KKT_MGS2B(0, 2) KKT_MGS2B(1, 0) KKT_MGS2B(1, 1) KKT_MGS2B(1, 2) KKT_MGS2B(2, 0)
              KKT_MGS2B(2, 1) KKT_MGS2B(2, 2)
#undef KKT_MGS2B
              KKT_CUDA_TRY(cudaGetLastError());
            }
            const int width = nd > 1 ? 2 : 1;
            ProfScope ps(KKT_K_REDUCE, st);
            finalize_cols_b<<<nr * width, 32, 0, st>>>(part, t_new.prefix, nr, width, d_out, 33, nd > 0 ? k + na : j + 1);
            KKT_CUDA_TRY(cudaGetLastError());
            return KKT_OK;
          };
          rc = step(0, std::min(2, j + 1), 0);
          for (int k = 0; k <= j && rc == KKT_OK;) {
            const int na = std::min(2, j + 1 - k);
            const int nd = std::min(2, j + 1 - (k + na));
            rc = step(na, nd, k);
            k += na;
          }
          if (rc != KKT_OK) break;
          KKT_CUDA_TRY(cudaMemcpyAsync(h_out, d_out, sizeof(double) * 33 * nr, cudaMemcpyDeviceToHost, st));
          KKT_CUDA_TRY(cudaStreamSynchronize(st));
          for (int q = 0; q < nr; ++q) {
            InstState& I = *S[mem[q]];
            for (int i = 0; i <= j; ++i) Hs(I, i, j) = h_out[q * 33 + i] / I.eta[i];
            wn2[mem[q]] = h_out[q * 33 + j + 1];
          }
        }
        if (b->opt.orth == KKT_ORTH_MGS) {
          // modified Gram-Schmidt, step k over all running instances at once; the dots stay on
          // the device (d_out[q][k]) and feed the next step, the host reads the columns once
          for (int q = 0; q < nr; ++q)
            for (int i = 0; i <= j; ++i) h_coef[q * 33 + i] = 1.0 / (S[mem[q]]->eta[i] * S[mem[q]]->eta[i]);
          KKT_CUDA_TRY(cudaMemcpyAsync(d_coef, h_coef, sizeof(double) * 33 * nr, cudaMemcpyHostToDevice, st));
          const unsigned grid = static_cast<unsigned>(std::min<long long>(t_new.total, persistent_grid()));
          for (int k = -1; k <= j && rc == KKT_OK; ++k) {
            {
              const double el = t_new.elems;
              ProfScope ps(k < 0 ? KKT_K_MULTIDOT : KKT_K_UPDATE, st, (k < 0 ? 2.0 : 4.0) * el,
                           8.0 * el * (k < 0 ? 2.0 : (k < j ? 4.0 : 3.0)));
              if (k < 0)
                mgs_b<false, true><<<grid, kThreads, 0, st>>>(t_new.dev, t_new.prefix, nr, t_new.total, -1, d_out,
                                                              d_coef, 33, part);
              else if (k < j)
                mgs_b<true, true><<<grid, kThreads, 0, st>>>(t_new.dev, t_new.prefix, nr, t_new.total, k, d_out,
                                                             d_coef, 33, part);
              else
                mgs_b<true, false><<<grid, kThreads, 0, st>>>(t_new.dev, t_new.prefix, nr, t_new.total, k, d_out,
                                                              d_coef, 33, part);
              if (cudaGetLastError() != cudaSuccess) rc = set_error(KKT_ERR_CUDA, "batched MGS launch failed");
            }
            ProfScope ps(KKT_K_REDUCE, st);
            finalize_col_b<<<nr, 32, 0, st>>>(part, t_new.prefix, nr, d_out, 33, k + 1);
          }
          if (rc != KKT_OK) break;
          KKT_CUDA_TRY(cudaMemcpyAsync(h_out, d_out, sizeof(double) * 33 * nr, cudaMemcpyDeviceToHost, st));
          KKT_CUDA_TRY(cudaStreamSynchronize(st));
          for (int q = 0; q < nr; ++q) {
            InstState& I = *S[mem[q]];
            for (int i = 0; i <= j; ++i) Hs(I, i, j) = h_out[q * 33 + i] / I.eta[i];
            wn2[mem[q]] = h_out[q * 33 + j + 1];
          }
        }
        for (int pass = 0; pass < 2 && rc == KKT_OK && b->opt.orth == KKT_ORTH_CGS2; ++pass) {
          rc = dispatch<MultidotB>(j + 1, t_new.dev, t_new.prefix, nr, t_new.total, part, 2.0 * t_new.elems, st);
          if (rc != KKT_OK) break;
          rc = finalize(t_new, j + 2);
          if (rc != KKT_OK) break;
          for (int q = 0; q < nr; ++q) {
            InstState& I = *S[mem[q]];
            if (need[q]) before[q] = h_out[q * (j + 2) + j + 1];
            for (int i = 0; i <= j; ++i) {
              const double hk = need[q] ? h_out[q * (j + 2) + i] / I.eta[i] : 0.0;
              Hs(I, i, j) += hk;
              h_coef[q * ldc + i] = hk / I.eta[i];
            }
          }
          KKT_CUDA_TRY(cudaMemcpyAsync(d_coef, h_coef, sizeof(double) * ldc * nr, cudaMemcpyHostToDevice, st));
          rc = dispatch<UpdateB>(j + 1, t_new.dev, t_new.prefix, nr, t_new.total, d_coef, ldc, part, 1,
                                 2.0 * t_new.elems, st);
          if (rc != KKT_OK) break;
          rc = finalize(t_new, 1);
          if (rc != KKT_OK) break;
          bool again = false;
          for (int q = 0; q < nr; ++q) {
            if (!need[q]) continue;
            wn2[mem[q]] = h_out[q];
            need[q] = h_out[q] < 0.5 * before[q];
            again = again || need[q];
          }
          if (!again) break;
        }
        if (rc != KKT_OK) break;
        for (int k = 0; k < nw; ++k) {
          InstState& I = *S[k];
          const double hn = std::sqrt(wn2[k]);
          I.eta[j + 1] = (hn > 0 && std::isfinite(hn)) ? hn : 1.0;
          if (I.cycle_done) continue;
          if (!std::isfinite(hn)) {
            I.status = KKT_ERR_NONFINITE;
            I.active = 0;
            I.cycle_done = 1;
            continue;
          }
          Hs(I, j + 1, j) = hn;
          for (int i = 0; i < j; ++i) {
            const double t = I.cs[i] * Hs(I, i, j) + I.sn[i] * Hs(I, i + 1, j);
            Hs(I, i + 1, j) = -I.sn[i] * Hs(I, i, j) + I.cs[i] * Hs(I, i + 1, j);
            Hs(I, i, j) = t;
          }
          const double d = std::hypot(Hs(I, j, j), Hs(I, j + 1, j));
          I.cs[j] = d > 0 ? Hs(I, j, j) / d : 1.0;
          I.sn[j] = d > 0 ? Hs(I, j + 1, j) / d : 0.0;
          Hs(I, j, j) = d;
          Hs(I, j + 1, j) = 0.0;
          I.g[j + 1] = -I.sn[j] * I.g[j];
          I.g[j] = I.cs[j] * I.g[j];
          I.its++;
          I.jused = j + 1;
          const double est = std::fabs(I.g[j + 1]) / I.fnorm;
          I.hist.push_back(est);
          if (est <= tol || I.its >= maxit || hn == 0.0) I.cycle_done = 1;
        }
      }
      if (rc != KKT_OK) break;
      // x += Z y per instance (coefficients zero for instances without steps this cycle)
      int jmax = 0;
      for (int k = 0; k < nw; ++k) {
        InstState& I = *S[k];
        jmax = std::max(jmax, I.jused);
        for (int i = I.jused - 1; i >= 0; --i) {
          double s = I.g[i];
          for (int c = i + 1; c < I.jused; ++c) s -= Hs(I, i, c) * I.y[c];
          I.y[i] = Hs(I, i, i) != 0.0 ? s / Hs(I, i, i) : 0.0;
        }
        for (int i = 0; i < ldc; ++i) {
          const bool on = I.active && i < I.jused;
          h_coef[k * ldc + i] = on ? -I.y[i] / (I.h->g.h * I.du * I.eta[i]) : 0.0;
          h_coef[(nw + k) * ldc + i] = on ? -I.y[i] / (I.h->g.omega * I.h->g.h * I.dz * I.eta[i]) : 0.0;
          h_coef[(2 * nw + k) * ldc + i] = on ? -I.y[i] : 0.0;
        }
      }
      if (jmax > 0) {
        KKT_CUDA_TRY(cudaMemcpyAsync(d_coef, h_coef, sizeof(double) * 3 * ldc * nw, cudaMemcpyHostToDevice, st));
        // update_b subtracts: x -= (-y) V
        rc = dispatch<UpdateB>(jmax, t_xu.dev, t_xu.prefix, nw, t_xu.total, d_coef, ldc, part, 0, 2.0 * t_xu.elems, st);
        if (rc == KKT_OK)
          rc = dispatch<UpdateB>(jmax, t_xz.dev, t_xz.prefix, nw, t_xz.total, d_coef + nw * ldc, ldc, part, 0,
                                 2.0 * t_xz.elems, st);
        if (rc == KKT_OK)
          rc = dispatch<UpdateB>(jmax, t_xw.dev, t_xw.prefix, nw, t_xw.total, d_coef + 2 * nw * ldc, ldc, part, 0,
                                 2.0 * t_xw.elems, st);
      }
      if (rc != KKT_OK) break;
      for (int k = 0; k < nw; ++k)
        if (S[k]->active && S[k]->jused > 0) S[k]->restarts++;
      rc = residual();
      if (rc != KKT_OK) break;
      for (int k = 0; k < nw; ++k) {
        InstState& I = *S[k];
        if (!I.active) continue;
        I.rel = I.beta / I.fnorm;
        if (!std::isfinite(I.rel)) {
          I.status = KKT_ERR_NONFINITE;
          I.active = 0;
        } else if (I.rel <= tol) {
          I.status = KKT_OK;
          I.active = 0;
        } else if (I.its >= maxit) {
          I.status = KKT_NOT_CONVERGED;
          I.active = 0;
        }
      }
    }
    for (int j = 0; j < m; ++j) {
      if (graphs[j]) cudaGraphExecDestroy(graphs[j]);
      batch_slot_free(slots[j]);
    }
    batch_slot_free(resid_slot);
    batch_slot_free(sub_slot);
    t_full.free();
    t_new.free();
    for (int bl = 0; bl < 3; ++bl) t_f[bl].free();
    t_xu.free();
    t_xz.free();
    t_xw.free();
    cudaFree(part);
    // back to grid values: x in place
    for (int k = 0; k < nw && spectral; ++k) {
      const long long V = S[k]->h->g.V;
      for (int bl = 0; bl < 3; ++bl)
        if (dst2d(S[k]->h, S[k]->x + bl * V, S[k]->x + bl * V, st) < 0 && rc == KKT_OK) rc = KKT_ERR_CUDA;
    }
    if (rc != KKT_OK) {
      rc_all = rc;
      break;
    }
    ++waves_done;
  }
  cudaFreeHost(h_tmp);
  cudaFree(d_small);
  cudaFree(arena);
  if (rc_all < 0) return rc_all;
  // a tensor-core transform that gave up waiting on its pipeline fails its instance
  std::vector<char> is_solo(n_inst, 0);
  for (int i : solo) is_solo[i] = 1;
  for (int i = 0; i < n_inst; ++i)
    if (!is_solo[i] && b->inst[i]->dst_tensor && oz_check(b->inst[i]->oz, st) < 0) all[i].status = KKT_ERR_TIMEOUT;
  for (int i : solo) {
    all[i].its = solo_its[i];
    all[i].status = solo_status[i];
    all[i].rel = solo_rel[i];
  }
  int worst = KKT_OK;
  for (int i = 0; i < n_inst; ++i) {
    if (all[i].status < 0) worst = std::min(worst, all[i].status);
    else if (all[i].status == KKT_NOT_CONVERGED && worst == KKT_OK) worst = KKT_NOT_CONVERGED;
  }
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    stats->solo = static_cast<int>(solo.size());
    stats->waves = waves_done;
    stats->graphs = graphs_made;
    stats->graph_launches = graph_launches;
    stats->tile_lines = b->tuned_tile_lines;
    stats->sweep_block = b->tuned_sweep_tb;
    for (int a = 0; a < 3; ++a) {
      stats->tune_ms_dst[a] = b->tune_ms_dst[a];
      stats->tune_ms_sweep[a] = b->tune_ms_sweep[a];
    }
    stats->time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    for (int i = 0; i < n_inst && i < KKT_BATCH_MAX; ++i) {
      stats->iterations[i] = all[i].its;
      stats->status[i] = all[i].status;
      stats->rel_residual[i] = all[i].rel;
    }
  }
  return worst;
}

}  // extern "C"
