// Orthonormal DST-I of every grid line of a space-time block: the spatial transform that
// diagonalises the 5-point Laplacian of Eq 2, so that each implicit step of the sweeps in
// Eq 13 becomes a division per sine mode (the paper solves the implicit operator in space
// "with a direct solve", Section 4).
//
// For n = 2^p intervals a line of n-1 points is transformed with a real FFT of length n,
// itself a complex FFT of length n/2 (radix-2, decimation in time, in shared memory):
//   y_0 = 0, y_j = sin(j pi/n)(x_j + x_{n-j}) + (x_j - x_{n-j})/2,   j = 1..n-1
//   Y_k = sum_j y_j exp(-2 pi i j k / n) = R_k - i I_k
//   S_2k = I_k,  S_2k+1 = S_2k-1 + R_k  (S_1 = R_0 / 2),   S_k = sum_j x_j sin(pi j k / n)
// (the odd-symmetric DST-I folded onto a half-length real transform; the odd outputs are a
// prefix sum, computed with a warp scan). Other n use the direct O(n^2) sum.
//
// Work layout: a CTA stages a tile of `tile_lines` lines in shared memory with coalesced
// loads (rows: one contiguous run; columns: 32 consecutive columns per grid row), each of
// its 8 warps transforms whole lines, and the tile is stored back the same way.
// Every output element is written by exactly one thread; in == out is allowed.
#include <algorithm>
#include <cmath>
#include <vector>

#include "kkt_internal.cuh"

namespace kkt {
namespace {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;



__device__ __forceinline__ int bit_reverse(int v, int bits) {
  return bits > 0 ? static_cast<int>(__brev(static_cast<unsigned>(v)) >> (32 - bits)) : 0;
}

// Padded position of complex element i in a warp's FFT buffer: one spare 16-byte slot after
// every 8 elements, so the butterflies' power-of-two strides spread over the banks.
__device__ __forceinline__ int pidx(int i) { return i + (i >> 3); }
// doubles per warp: n/2 + n/16 double2 and slack, kept even so every warp's buffer is 16-byte aligned
constexpr int fft_buf_words(int n) { return (n + n / 8 + 2 + 1) & ~1; }

// Complex product v w (4 FP64 instructions).
__device__ __forceinline__ double2 cmul(double2 v, double2 w) {
  return make_double2(fma(v.x, w.x, -v.y * w.y), fma(v.x, w.y, v.y * w.x));
}

// One line x[0..n-2] (x[j-1] holds the j-th point), in place, on G lanes of a warp (lane `sub`
// of the group); the warp's 32 / G groups transform 32 / G lines side by side, each with its own
// buf (n/2 double2, padded). G is about P / 4, so every lane has a radix-4 butterfly in each pass
// of a short line (one line per warp from 256 intervals up).
// FP64 is the bound on this part (2 DFMA-pipe instructions per clock per SM), so the line is
// arranged to spend as few FP64 instructions as possible: the orthonormal scale is folded into
// the pre-processing weights (y_j = w+_j x_j + w-_j x_n-j), stages 1 and 2 of the FFT (twiddles
// 1 and -i) are one radix-4 pass of additions only, later stages go two at a time as radix-4
// passes (3 complex products per 4 points instead of 4), and R_0 / 2 is taken out of the
// prefix sum once per lane instead of per output.
template <int G>
__device__ void dst_line_fft(double* x, double2* buf, const DstLaunch& L, int sub) {
  const int n = L.n, P = n >> 1, logp = L.logn - 1;
  const double2* pw = reinterpret_cast<const double2*>(L.pre);   // c (sin + 1/2), c (sin - 1/2)
  for (int j = sub; j < n; j += G) {
    double yj = 0.0;
    if (j > 0) {
      const double a = x[j - 1], b = x[n - j - 1];
      const double2 q = pw[j <= P ? j : n - j];
      yj = fma(q.x, a, q.y * b);
    }
    reinterpret_cast<double*>(buf + pidx(bit_reverse(j >> 1, logp)))[j & 1] = yj;
  }
  __syncwarp();
  int s = 1;
  if (logp >= 2) {
    // stages 1 and 2: pairs (0,1), (2,3) with twiddle 1, then (0,2) with 1 and (1,3) with -i
    for (int b = sub; b < (P >> 2); b += G) {
      const int i0 = 4 * b;
      const double2 a0 = buf[pidx(i0)], a1 = buf[pidx(i0 + 1)], a2 = buf[pidx(i0 + 2)], a3 = buf[pidx(i0 + 3)];
      const double2 b0 = make_double2(a0.x + a1.x, a0.y + a1.y), b1 = make_double2(a0.x - a1.x, a0.y - a1.y);
      const double2 b2 = make_double2(a2.x + a3.x, a2.y + a3.y), b3 = make_double2(a2.x - a3.x, a2.y - a3.y);
      buf[pidx(i0)] = make_double2(b0.x + b2.x, b0.y + b2.y);
      buf[pidx(i0 + 2)] = make_double2(b0.x - b2.x, b0.y - b2.y);
      buf[pidx(i0 + 1)] = make_double2(b1.x + b3.y, b1.y - b3.x);   // b1 + (-i) b3
      buf[pidx(i0 + 3)] = make_double2(b1.x - b3.y, b1.y + b3.x);
    }
    __syncwarp();
    s = 3;
  }
  // stages s, s+1 merged: with W = exp(-2 pi i / 2^(s+1)) and k the position in the group,
  // p0 = a0, p1 = W^k a2, p2 = W^2k a1, p3 = W^3k a3 (a_r at distance r 2^(s-1)), outputs
  // (p0 + p2) +- (p1 + p3) and (p0 - p2) -+ i (p1 - p3); tw[m] = exp(-2 pi i m / P)
  for (; s + 1 <= logp; s += 2) {
    const int half = 1 << (s - 1), tsh = logp - s - 1;
    for (int b = sub; b < (P >> 2); b += G) {
      const int k = b & (half - 1);
      const int i0 = ((b >> (s - 1)) << (s + 1)) + k;
      const double2 p0 = buf[pidx(i0)];
      const double2 p2 = cmul(buf[pidx(i0 + half)], L.tw[(2 * k) << tsh]);
      const double2 p1 = cmul(buf[pidx(i0 + 2 * half)], L.tw[k << tsh]);
      const double2 p3 = cmul(buf[pidx(i0 + 3 * half)], L.tw[(3 * k) << tsh]);
      const double2 S = make_double2(p0.x + p2.x, p0.y + p2.y), T = make_double2(p1.x + p3.x, p1.y + p3.y);
      const double2 U = make_double2(p0.x - p2.x, p0.y - p2.y), D = make_double2(p1.x - p3.x, p1.y - p3.y);
      buf[pidx(i0)] = make_double2(S.x + T.x, S.y + T.y);
      buf[pidx(i0 + 2 * half)] = make_double2(S.x - T.x, S.y - T.y);
      buf[pidx(i0 + half)] = make_double2(U.x + D.y, U.y - D.x);       // U - i D
      buf[pidx(i0 + 3 * half)] = make_double2(U.x - D.y, U.y + D.x);   // U + i D
    }
    __syncwarp();
  }
  if (s == logp) {   // one radix-2 stage left
    const int half = 1 << (s - 1);
    for (int b = sub; b < (P >> 1); b += G) {
      const int k = b & (half - 1);
      const int i0 = ((b >> (s - 1)) << s) + k;
      const int i1 = i0 + half;
      const double2 u = buf[pidx(i0)];
      const double2 t = cmul(buf[pidx(i1)], L.tw[k << (logp - s)]);
      buf[pidx(i0)] = make_double2(u.x + t.x, u.y + t.y);
      buf[pidx(i1)] = make_double2(u.x - t.x, u.y - t.y);
    }
    __syncwarp();
  }
  // Unpack Y_k (times 2) from the half-length FFT; even outputs directly, odd ones by a scan.
  const int chunk = P >= G ? P / G : 1;
  const int k0 = sub * chunk;
  const bool active = k0 < P;
  double total = 0.0;
  if (active) {
    for (int t = 0; t < chunk; ++t) {
      const int k = k0 + t;
      const double2 zk = buf[pidx(k)];
      const double2 zc = buf[pidx((P - k) & (P - 1))];
      const double er = zk.x + zc.x, nei = zc.y - zk.y;    // Z_k + conj(Z_{P-k}) (imaginary part negated)
      const double orr = zk.y + zc.y, oi = zc.x - zk.x;    // (Z_k - conj(Z_{P-k})) / i
      const double2 w = L.post[k];                         // exp(-2 pi i k / n)
      const double yr = fma(w.x, orr, fma(-w.y, oi, er));
      const double nyi = fma(-w.x, oi, fma(-w.y, orr, nei));
      if (k > 0) x[2 * k - 1] = nyi;                       // S_2k = I_k = -Im Y_k
      total += yr;                                         // R_0 + R_1 + ... + R_k
      x[2 * k] = total;
    }
  }
  double incl = total;   // inclusive scan over the G lanes of this line
#pragma unroll
  for (int o = 1; o < G; o <<= 1) {
    const double v = __shfl_up_sync(0xffffffffu, incl, o, G);
    if (sub >= o) incl += v;
  }
  const double prev = __shfl_up_sync(0xffffffffu, incl, 1, G);
  // S_2k+1 = R_0 / 2 + R_1 + ... + R_k: the exclusive prefix of the lanes before, less R_0 / 2
  // (R_0 = 2 (Z_0.x + Z_0.y) in the times-2 convention)
  const double corr = (sub == 0 ? 0.0 : prev) - (buf[0].x + buf[0].y);   // (pidx(0) = 0)
  if (active)
    for (int t = 0; t < chunk; ++t) x[2 * (k0 + t)] += corr;
  __syncwarp();
}

// Direct transform for n that is not a power of two: S_k = sum_j x_j sin(pi j k / n).
__device__ void dst_line_direct(double* x, double* tmp, const DstLaunch& L, int lane) {
  const int n = L.n, M = L.M, n2 = 2 * n;
  for (int k = lane + 1; k <= M; k += 32) {
    double acc = 0.0;
    int idx = 0;                       // (j k) mod 2n, advanced incrementally
    for (int j = 1; j <= M; ++j) {
      idx += k;
      if (idx >= n2) idx -= n2;
      acc = fma(x[j - 1], L.sintab[idx], acc);
    }
    tmp[k - 1] = acc;
  }
  __syncwarp();
  for (int k = lane; k < M; k += 32) x[k] = tmp[k];
  __syncwarp();
}

// Lanes per line of the FFT path: about P / 4 (one radix-4 butterfly per lane and pass), at
// most 32, and at least 32 / tile_lines so that a warp's lines stay inside the tile (tile_lines
// is then a multiple of the lines per warp).
__host__ __device__ inline int fft_group_for(int n, int tile_lines) {
  int g = (n >> 1) / 4;
  if (g < 1) g = 1;
  if (g > 32) g = 32;
  const int gmin = 32 / tile_lines;
  return g < gmin ? gmin : g;
}

// A warp's 32 / G lines side by side. Groups whose line index passes nl work on the tile's
// unused rows (below tile_lines) and their results are never stored.
template <int G>
__device__ void fft_lines(const DstLaunch& L, double* tile, double* fbase, int nl, int warp, int lane) {
  constexpr int LW = 32 / G;
  const int grp = lane / G, sub = lane % G;
  double2* fbuf = reinterpret_cast<double2*>(fbase + (warp * LW + grp) * fft_buf_words(L.n));
  for (int l0 = warp * LW; l0 < nl; l0 += kWarps * LW) dst_line_fft<G>(tile + (l0 + grp) * L.ldt, fbuf, L, sub);
}

// One tile of lines: load, transform, store. `bid` is the tile index within the launch.
__device__ void dst_tile_body(const DstLaunch& L, long long bid, double* smem) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double* tile = smem;
  const int tile_words = (L.tile_lines * L.ldt + 1) & ~1;
  double* fbase = smem + tile_words;   // FFT buffers: kWarps x (32 / G) lines

  long long base = 0;
  int nl = 0;
  if (L.mode == 0) {
    const long long first = bid * L.tile_lines;
    { const long long rem = L.total_lines - first; nl = static_cast<int>(rem < L.tile_lines ? rem : L.tile_lines); }
    base = first * L.M;
    for (int l = warp; l < nl; l += kWarps)
      for (int e = lane; e < L.M; e += 32) tile[l * L.ldt + e] = L.in[base + static_cast<long long>(l) * L.M + e];
  } else {
    const long long sl = bid / L.tiles_per_slice;
    const int col0 = static_cast<int>(bid % L.tiles_per_slice) * L.tile_lines;
    nl = min(L.tile_lines, L.cols - col0);
    base = sl * L.slice + col0;
    for (int e = warp; e < L.M; e += kWarps)
      for (int l = lane; l < nl; l += 32) tile[l * L.ldt + e] = L.in[base + static_cast<long long>(e) * L.cols + l];
  }
  __syncthreads();
  if (L.logn >= 2) {
    switch (L.fft_group) {
      case 32: fft_lines<32>(L, tile, fbase, nl, warp, lane); break;
      case 16: fft_lines<16>(L, tile, fbase, nl, warp, lane); break;
      case 8: fft_lines<8>(L, tile, fbase, nl, warp, lane); break;
      case 4: fft_lines<4>(L, tile, fbase, nl, warp, lane); break;
      case 2: fft_lines<2>(L, tile, fbase, nl, warp, lane); break;
      default: fft_lines<1>(L, tile, fbase, nl, warp, lane); break;
    }
  } else {
    double* tmp = fbase + warp * fft_buf_words(L.n);
    for (int l = warp; l < nl; l += kWarps) dst_line_direct(tile + l * L.ldt, tmp, L, lane);
  }
  __syncthreads();
  if (L.mode == 0) {
    for (int l = warp; l < nl; l += kWarps)
      for (int e = lane; e < L.M; e += 32) L.out[base + static_cast<long long>(l) * L.M + e] = tile[l * L.ldt + e];
  } else {
    for (int e = warp; e < L.M; e += kWarps)
      for (int l = lane; l < nl; l += 32) L.out[base + static_cast<long long>(e) * L.cols + l] = tile[l * L.ldt + e];
  }
}

// Short lines (at most kLaneMaxM points, n <= 32): one thread transforms one whole line by
// the direct sum S_k = sum_j x_j sin(pi j k / n) (M FMAs per output, the same order as
// dst_line_direct), its inputs held in registers. A warp's 32 lines keep every lane busy, where
// the warp-per-line FFT of an 8- or 16-point half-length transform leaves most lanes idle. The
// sine table index is the same on every lane (a broadcast load). Lines are read and written in
// place of the tile staging: rows mode line t starts at t M (stride 1), columns mode line
// (slice, c) at slice * slice_size + c (stride cols). A thread writes only its own line, after
// reading all of it, so in == out is allowed.
constexpr int kLaneMaxM = 31;

__device__ void dst_lane_body(const DstLaunch& L, long long t) {
  if (t >= L.lines) return;
  long long base;
  long long stride;
  if (L.mode == 0) {
    base = t * L.M;
    stride = 1;
  } else {
    const long long sl = t / L.cols;
    base = sl * L.slice + (t - sl * L.cols);
    stride = L.cols;
  }
  const int M = L.M, n2 = 2 * L.n;
  double x[kLaneMaxM];
#pragma unroll
  for (int j = 0; j < kLaneMaxM; ++j) x[j] = j < M ? L.in[base + j * stride] : 0.0;
  // four outputs at a time: four independent FMA chains (outputs past M are computed with
  // k <= M + 3 < 2n and not stored)
  for (int k = 1; k <= M; k += 4) {
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    int idx[4] = {0, 0, 0, 0};   // (j (k + u)) mod 2n for j = 1, 2, ...
#pragma unroll
    for (int j = 0; j < kLaneMaxM; ++j) {
      if (j < M) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          idx[u] += k + u;
          if (idx[u] >= n2) idx[u] -= n2;
          acc[u] = fma(x[j], __ldg(L.sintab + idx[u]), acc[u]);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (k + u <= M) L.out[base + (k + u - 1) * stride] = acc[u];
  }
}

// 64-thread CTAs: the few hundred CTAs of a small grid then spread evenly over the SMs (with
// 256 threads, 188 CTAs on 152 SMs left 36 SMs with twice the work)
constexpr int kLaneThreads = 64;

__global__ void __launch_bounds__(kLaneThreads) dst_lane_kernel(DstLaunch L) {
  dst_lane_body(L, static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x);
}

__global__ void __launch_bounds__(kThreads) dst_tile_kernel(DstLaunch L) {
  extern __shared__ double smem[];
  dst_tile_body(L, blockIdx.x, smem);
}

// Several launches (instances, passes) in one grid: item t belongs to launch k with
// prefix[k] <= t < prefix[k+1]; blocks loop over the items.
__global__ void __launch_bounds__(kThreads) dst_tile_batched(const DstLaunch* __restrict__ Ls,
                                                             const long long* __restrict__ prefix, int nl,
                                                             long long total) {
  extern __shared__ double smem[];
  __shared__ long long sp[KKT_BATCH_MAX + 1];
  batch_prefix_load(sp, prefix, nl);
  for (long long t = blockIdx.x; t < total; t += gridDim.x) {
    const int k = batch_find(sp, nl, t);
    if (Ls[k].lane) {   // an item is kThreads lines, one per thread
      dst_lane_body(Ls[k], (t - sp[k]) * kThreads + threadIdx.x);
    } else {
      dst_tile_body(Ls[k], t - sp[k], smem);
      __syncthreads();
    }
  }
}

int tile_lines_for(int n) { return n > 512 ? 16 : 32; }

size_t smem_bytes(int n, int tl) {
  const int M = n - 1;
  const int ldt = M | 1;
  const size_t tile_words = (static_cast<size_t>(tl) * ldt + 1) & ~static_cast<size_t>(1);
  const int lines_per_warp = 32 / fft_group_for(n, tl);   // (the direct path uses one buffer per warp)
  return (tile_words + static_cast<size_t>(kWarps) * lines_per_warp * fft_buf_words(n)) * sizeof(double);
}

DstLaunch make_launch(const DstPlan& p, const double* in, double* out, int mode, long long total_lines, int cols,
                      long long slice, int tile_lines, long long nslices) {
  DstLaunch L;
  L.in = in;
  L.out = out;
  L.n = p.n;
  L.logn = p.logn;
  L.M = p.n - 1;
  L.ldt = L.M | 1;
  L.tile_lines = tile_lines > 0 ? tile_lines : tile_lines_for(p.n);
  L.mode = mode;
  L.total_lines = total_lines;
  L.cols = cols;
  L.slice = slice;
  L.tiles_per_slice = (cols + L.tile_lines - 1) / L.tile_lines;
  L.pre = p.d_pre;
  L.tw = p.d_tw;
  L.post = p.d_post;
  L.sintab = p.d_sin;
  L.lane = p.lane_direct && L.M <= kLaneMaxM;
  L.lines = mode == 0 ? total_lines : nslices * cols;
  L.fft_group = fft_group_for(p.n, L.tile_lines);
  return L;
}

long long launch_tiles(const DstLaunch& L, long long nslices) {
  if (L.lane) return (L.lines + kThreads - 1) / kThreads;
  return L.mode == 0 ? (L.total_lines + L.tile_lines - 1) / L.tile_lines : nslices * L.tiles_per_slice;
}

int launch_lines(const DstPlan& p, const double* in, double* out, int mode, long long total_lines,
                 int cols, long long slice, long long nslices, cudaStream_t st) {
  const DstLaunch L = make_launch(p, in, out, mode, total_lines, cols, slice, p.tile_lines, nslices);
  if (L.lane) {
    const long long lines = L.lines;
    if (lines <= 0) return KKT_OK;
    const long long grid = (lines + kLaneThreads - 1) / kLaneThreads;
    if (grid > 2147483647LL) return set_error(KKT_ERR_UNSUPPORTED, "DST grid too large");
    // the same algorithmic count as the FFT path (the work the transform needs), not the
    // direct sum's M FMAs per output
    ProfScope ps(KKT_K_DST, st, lines * 2.5 * L.M * std::log2(2.0 * p.n), lines * L.M * 16.0);
    dst_lane_kernel<<<static_cast<unsigned>(grid), kLaneThreads, 0, st>>>(L);
    KKT_CUDA_TRY(cudaGetLastError());
    return KKT_OK;
  }
  const size_t sm = smem_bytes(p.n, L.tile_lines);
  KKT_CUDA_TRY(cudaFuncSetAttribute(dst_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    static_cast<int>(sm)));
  long long grid = launch_tiles(L, nslices);
  if (grid <= 0) return KKT_OK;
  if (grid > 2147483647LL) return set_error(KKT_ERR_UNSUPPORTED, "DST grid too large");
  // one real DST-I of M points by FFT: 2.5 M log2(2n) flops; each point read and written once
  const double lines = mode == 0 ? static_cast<double>(total_lines) : static_cast<double>(nslices) * cols;
  ProfScope ps(KKT_K_DST, st, lines * 2.5 * L.M * std::log2(2.0 * p.n), lines * L.M * 16.0);
  dst_tile_kernel<<<static_cast<unsigned>(grid), kThreads, sm, st>>>(L);
  KKT_CUDA_TRY(cudaGetLastError());
  return KKT_OK;
}

}  // namespace

int dst_plan_create(DstPlan& p, int n) {
  if (n < 2 || n > 1024) return set_error(KKT_ERR_UNSUPPORTED, "grid intervals per direction must be in [2, 1024]");
  p.n = n;
  int lg = 0;
  while ((1 << lg) < n) ++lg;
  p.logn = ((1 << lg) == n && n >= 4) ? lg : -1;
  const double pi = 3.14159265358979323846;
  std::vector<double> pre(2 * (n / 2 + 1)), sintab(2 * n);
  std::vector<double2> tw(std::max(n / 2, 1)), post(n / 2 + 1);
  const double c = 1.0 / std::sqrt(2.0 * n);   // orthonormal scale of the FFT path's outputs
  for (int j = 0; j <= n / 2; ++j) {
    pre[2 * j] = c * (std::sin(j * pi / n) + 0.5);
    pre[2 * j + 1] = c * (std::sin(j * pi / n) - 0.5);
  }
  for (int k = 0; k < static_cast<int>(tw.size()); ++k)
    tw[k] = make_double2(std::cos(2 * pi * k / (n / 2)), -std::sin(2 * pi * k / (n / 2)));
  for (int k = 0; k <= n / 2; ++k) post[k] = make_double2(std::cos(2 * pi * k / n), -std::sin(2 * pi * k / n));
  const double sc = std::sqrt(2.0 / n);
  for (int m = 0; m < 2 * n; ++m) sintab[m] = sc * std::sin(m * pi / n);
  KKT_CUDA_TRY(cudaMalloc(&p.d_pre, pre.size() * sizeof(double)));
  KKT_CUDA_TRY(cudaMalloc(&p.d_tw, tw.size() * sizeof(double2)));
  KKT_CUDA_TRY(cudaMalloc(&p.d_post, post.size() * sizeof(double2)));
  KKT_CUDA_TRY(cudaMalloc(&p.d_sin, sintab.size() * sizeof(double)));
  KKT_CUDA_TRY(cudaMemcpy(p.d_pre, pre.data(), pre.size() * sizeof(double), cudaMemcpyHostToDevice));
  KKT_CUDA_TRY(cudaMemcpy(p.d_tw, tw.data(), tw.size() * sizeof(double2), cudaMemcpyHostToDevice));
  KKT_CUDA_TRY(cudaMemcpy(p.d_post, post.data(), post.size() * sizeof(double2), cudaMemcpyHostToDevice));
  KKT_CUDA_TRY(cudaMemcpy(p.d_sin, sintab.data(), sintab.size() * sizeof(double), cudaMemcpyHostToDevice));
  return KKT_OK;
}

void dst_plan_destroy(DstPlan& p) {
  cudaFree(p.d_pre);
  cudaFree(p.d_tw);
  cudaFree(p.d_post);
  cudaFree(p.d_sin);
  p = DstPlan();
}

// Batched 2D DST over several instances: one launch for all row passes, one for all column
// passes; tables filled once per slot (outside any graph capture), launches read them.
int dst_batched_prepare(BatchSlot& slot, int first_pass, const DstJob* jobs, int njobs, int tile_lines) {
  if (njobs < 0 || njobs > KKT_BATCH_MAX) return set_error(KKT_ERR_INVALID_ARG, "batched jobs out of range");
  slot.dst_njobs = njobs;
  if (njobs == 0) {   // every instance of the slot transforms on its own
    for (int pass = first_pass; pass < first_pass + 2; ++pass) {
      slot.dst_total[pass] = 0;
      slot.dst_smem[pass] = 0;
      slot.dst_flops[pass] = slot.dst_bytes[pass] = 0.0;
    }
    return KKT_OK;
  }
  if (!slot.dst) {
    // capacity for the largest batch, so a slot can be refilled with any job count
    KKT_CUDA_TRY(cudaMalloc(&slot.dst, 4 * static_cast<size_t>(KKT_BATCH_MAX) * sizeof(DstLaunch)));
    KKT_CUDA_TRY(cudaMalloc(&slot.dst_prefix, 4 * static_cast<size_t>(KKT_BATCH_MAX + 1) * sizeof(long long)));
  }
  for (int pass = first_pass; pass < first_pass + 2; ++pass) {
    const bool rows = (pass % 2) == 0;
    std::vector<DstLaunch> L(njobs);
    std::vector<long long> prefix(njobs + 1, 0);
    size_t sm = 0;
    double flops = 0, bytes = 0;
    for (int k = 0; k < njobs; ++k) {
      const kkt_handle* h = jobs[k].h;
      const Geometry& g = h->g;
      L[k] = rows ? make_launch(h->dst_x, jobs[k].in, jobs[k].out, 0, static_cast<long long>(g.Nt) * g.My, g.Mx, 0,
                                tile_lines, 0)
                  : make_launch(h->dst_y, jobs[k].out, jobs[k].out, 1, 0, g.Mx, g.N, tile_lines, g.Nt);
      prefix[k + 1] = prefix[k] + launch_tiles(L[k], g.Nt);
      sm = std::max(sm, smem_bytes(L[k].n, L[k].tile_lines));
      const double lines = rows ? static_cast<double>(g.Nt) * g.My : static_cast<double>(g.Nt) * g.Mx;
      flops += lines * 2.5 * L[k].M * std::log2(2.0 * L[k].n);
      bytes += lines * L[k].M * 16.0;
    }
    KKT_CUDA_TRY(cudaMemcpy(slot.dst + static_cast<size_t>(pass) * KKT_BATCH_MAX, L.data(), njobs * sizeof(DstLaunch),
                            cudaMemcpyHostToDevice));
    KKT_CUDA_TRY(cudaMemcpy(slot.dst_prefix + static_cast<size_t>(pass) * (KKT_BATCH_MAX + 1), prefix.data(),
                            (njobs + 1) * sizeof(long long), cudaMemcpyHostToDevice));
    slot.dst_total[pass] = prefix[njobs];
    slot.dst_smem[pass] = sm;
    slot.dst_flops[pass] = flops;
    slot.dst_bytes[pass] = bytes;
  }
  return KKT_OK;
}

int dst_batched_launch(const BatchSlot& slot, int pass, cudaStream_t st) {
  const long long total = slot.dst_total[pass];
  if (total <= 0) return KKT_OK;
  const size_t sm = slot.dst_smem[pass];
  KKT_CUDA_TRY(cudaFuncSetAttribute(dst_tile_batched, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm)));
  int dev = 0, sms = 0, per_sm = 0;
  KKT_CUDA_TRY(cudaGetDevice(&dev));
  KKT_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  KKT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dst_tile_batched, kThreads, sm));
  const long long grid = std::min<long long>(total, static_cast<long long>(std::max(sms, 1)) * std::max(per_sm, 1));
  ProfScope ps(KKT_K_DST, st, slot.dst_flops[pass], slot.dst_bytes[pass]);
  dst_tile_batched<<<static_cast<unsigned>(grid), kThreads, sm, st>>>(
      slot.dst + static_cast<size_t>(pass) * KKT_BATCH_MAX, slot.dst_prefix + static_cast<size_t>(pass) * (KKT_BATCH_MAX + 1),
      slot.dst_njobs, total);
  KKT_CUDA_TRY(cudaGetLastError());
  return KKT_OK;
}

void batch_slot_free(BatchSlot& slot) {
  cudaFree(slot.dst);
  cudaFree(slot.dst_prefix);
  cudaFree(slot.spec);
  cudaFree(slot.coarse_prefix);
  cudaFree(slot.sweep_prefix);
  cudaFree(slot.spec_cr);
  cudaFree(slot.cr_prefix);
  cudaFree(slot.mv);
  cudaFree(slot.mv_prefix);
  slot = BatchSlot();
}

// Smallest grid the create-time timing offers the tensor-core transform to (below it the lines
// are short enough that the FFT and direct-sum tiles are cheap and accurate to rounding).
constexpr int kTensorMinN = 64;

int dst_autotune(kkt_handle* h) {
  const Geometry& g = h->g;
  KKT_CUDA_TRY(cudaMemset(h->spec, 0, static_cast<size_t>(g.V) * sizeof(double)));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  KKT_CUDA_TRY(cudaEventCreate(&e0));
  KKT_CUDA_TRY(cudaEventCreate(&e1));
  auto time_pass = [&](DstPlan& p, int tl, bool rows) -> double {
    p.tile_lines = tl;
    auto run = [&]() {
      return rows ? launch_lines(h->dst_x, h->spec, h->spec2, 0, static_cast<long long>(g.Nt) * g.My, g.Mx, 0, 0, nullptr)
                  : launch_lines(h->dst_y, h->spec2, h->spec2, 1, 0, g.Mx, g.N, g.Nt, nullptr);
    };
    if (run() != KKT_OK) {   // refused (shared memory): not a candidate
      cudaGetLastError();
      return 1e30;
    }
    cudaEventRecord(e0, nullptr);
    for (int r = 0; r < 2; ++r) run();
    cudaEventRecord(e1, nullptr);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    return ms;
  };
  for (int pass = 0; pass < 2; ++pass) {
    DstPlan& p = pass == 0 ? h->dst_x : h->dst_y;
    int best = 0;
    double best_ms = 1e30;
    p.lane_direct = false;
    for (int tl : {8, 16, 32}) {
      const double ms = time_pass(p, tl, pass == 0);
      if (ms < best_ms) {
        best_ms = ms;
        best = tl;
      }
    }
    p.tile_lines = best;   // 0 (the default) if no candidate ran
    if (p.n - 1 <= kLaneMaxM) {   // short lines: the thread-per-line transform is a candidate too
      p.lane_direct = true;
      const double ms = time_pass(p, best, pass == 0);
      p.lane_direct = ms < best_ms;
    }
  }
  // square grids with lines of 63..255 points: the tensor-core FP64 transform against the two
  // tuned passes, both timed as whole 2D transforms
  h->dst_tensor = false;
  if (g.nx == g.ny && g.nx >= kTensorMinN && g.nx - 1 <= 255) {
    auto time_2d = [&]() -> double {
      dst2d(h, h->spec, h->spec2, nullptr);   // warm-up
      cudaEventRecord(e0, nullptr);
      for (int r = 0; r < 2; ++r) dst2d(h, h->spec, h->spec2, nullptr);
      cudaEventRecord(e1, nullptr);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      return ms;
    };
    const double ms_tiles = time_2d();
    if (!h->oz.qs && oz_plan_create(h->oz, g.nx, g.Nt) == KKT_OK) h->bytes += h->oz.bytes;
    if (h->oz.qs) {
      h->dst_tensor = true;
      const double ms_tensor = time_2d();
      if (cudaGetLastError() != cudaSuccess || !(ms_tensor < ms_tiles)) {
        h->dst_tensor = false;
        h->bytes -= h->oz.bytes;
        oz_plan_destroy(h->oz);
      }
    } else {
      cudaGetLastError();   // no room for the digit planes: the tiles stay
      oz_plan_destroy(h->oz);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return set_error(KKT_ERR_CUDA, std::string("transform autotuning: ") + cudaGetErrorString(e));
  set_error(KKT_OK, "");
  return KKT_OK;
}

int dst_set_method(kkt_handle* h, int method) {
  for (DstPlan* p : {&h->dst_x, &h->dst_y}) {
    if (method == KKT_DST_LANE && p->n - 1 > kLaneMaxM)
      return set_error(KKT_ERR_UNSUPPORTED, "the thread-per-line transform needs lines of at most 31 points");
  }
  if (method == KKT_DST_TENSOR) {
    const Geometry& g = h->g;
    if (g.nx != g.ny || g.nx - 1 > 255)
      return set_error(KKT_ERR_UNSUPPORTED, "the tensor-core FP64 transform needs a square grid of at most 256 intervals");
    if (!h->oz.qs) {
      const int rc = oz_plan_create(h->oz, g.nx, g.Nt);
      if (rc < 0) {
        const std::string msg = kkt_last_error();
        oz_plan_destroy(h->oz);
        return set_error(rc, msg);
      }
      h->bytes += h->oz.bytes;
    }
    h->dst_tensor = true;
    return KKT_OK;
  }
  h->dst_tensor = false;
  if (h->oz.qs) {
    h->bytes -= h->oz.bytes;
    oz_plan_destroy(h->oz);
  }
  if (method == KKT_DST_AUTO) return dst_autotune(h);
  for (DstPlan* p : {&h->dst_x, &h->dst_y}) p->lane_direct = method == KKT_DST_LANE;
  return KKT_OK;
}

bool dst_tensor_fills_gpu(const kkt_handle* h) {
  if (!h->dst_tensor || !h->oz.qs) return false;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return false;
  return oz_tiles(h->oz) >= sms;
}

int dst2d(const kkt_handle* h, const double* in, double* out, cudaStream_t st) {
  if (h->dst_tensor) return oz_dst2d(h->oz, in, out, st);
  const Geometry& g = h->g;
  // rows: Nt * My lines of Mx contiguous points (transform along x)
  KKT_TRY(launch_lines(h->dst_x, in, out, 0, static_cast<long long>(g.Nt) * g.My, g.Mx, 0, 0, st));
  // columns: per slice, Mx lines of My points with stride Mx (transform along y)
  KKT_TRY(launch_lines(h->dst_y, out, out, 1, 0, g.Mx, g.N, g.Nt, st));
  return KKT_OK;
}

}  // namespace kkt
