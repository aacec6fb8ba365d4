// Stencil kernels on the space-time grid: the KKT matvec of Eq 5, the right-hand side,
// the time-coupled Jhat / Jhat^T products (Eq 7) and a scaling pass.
//
// K (u, z, w) per time node n (Eqs 2-5), with B0 = I + dt nu A and the 5-point A of Eq 2:
//   y_u^n = h u^n + B0 w^n - w^{n+1}          (w^{Nt+1} = 0)
//   y_z^n = omega h z^n - dt w^n
//   y_w^n = B0 u^n - u^{n-1} - dt z^n         (u^0 = 0; the initial state lives in f)
// One thread per grid point computes all three outputs; every input value is read from
// global memory, neighbours hit L1/L2. The Krylov driver applies the matvec to scaled
// inputs (su u, sz z, sw w) and scales the three output blocks (ou, oz, ow); every scale is
// folded into the stencil coefficients so one point costs 16 FP64 instructions.
#include <algorithm>
#include <vector>

#include "kkt_internal.cuh"

namespace kkt {
namespace {

struct Stencil {
  int Mx, My, Nt;
  long long N, V;
  double c0, cx, cy;   // B v = c0 v - cx (v_w + v_e) - cy (v_s + v_n)
};

__device__ __forceinline__ double apply_b(const double* __restrict__ v, long long idx, int i, int j,
                                          const Stencil& s) {
  const double c = v[idx];
  const double we = (i > 0 ? v[idx - 1] : 0.0) + (i + 1 < s.Mx ? v[idx + 1] : 0.0);
  const double sn = (j > 0 ? v[idx - s.Mx] : 0.0) + (j + 1 < s.My ? v[idx + s.Mx] : 0.0);
  return fma(s.c0, c, -fma(s.cx, we, s.cy * sn));
}

// Coefficients of the scaled matvec:
//   y_u = uu u + wc0 w - wcx (w_w + w_e) - wcy (w_s + w_n) - wn w^{n+1}
//   y_z = zz z - zw w
//   y_w = uc0 u - ucx (u_w + u_e) - ucy (u_s + u_n) - up u^{n-1} - wz z
constexpr long long kMvItem = 2048;   // points per work item of the batched matvec

struct MatvecCoef {
  double uu, wc0, wcx, wcy, wn;
  double zz, zw;
  double uc0, ucx, ucy, up, wz;
};

__global__ void matvec_kernel(const double* __restrict__ u, const double* __restrict__ z,
                              const double* __restrict__ w, double* __restrict__ y, Stencil s, MatvecCoef c) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int n = blockIdx.z;
  if (i >= s.Mx || j >= s.My) return;
  const long long idx = static_cast<long long>(n) * s.N + static_cast<long long>(j) * s.Mx + i;
  const bool hw = i > 0, he = i + 1 < s.Mx, hs = j > 0, hn = j + 1 < s.My;
  const double wc = w[idx];
  const double wwe = (hw ? w[idx - 1] : 0.0) + (he ? w[idx + 1] : 0.0);
  const double wsn = (hs ? w[idx - s.Mx] : 0.0) + (hn ? w[idx + s.Mx] : 0.0);
  const double wnx = n + 1 < s.Nt ? w[idx + s.N] : 0.0;
  const double uc = u[idx];
  const double uwe = (hw ? u[idx - 1] : 0.0) + (he ? u[idx + 1] : 0.0);
  const double usn = (hs ? u[idx - s.Mx] : 0.0) + (hn ? u[idx + s.Mx] : 0.0);
  const double upr = n > 0 ? u[idx - s.N] : 0.0;
  const double zc = z[idx];
  double t = fma(c.wcy, wsn, fma(c.wcx, wwe, c.wn * wnx));
  y[idx] = fma(c.uu, uc, fma(c.wc0, wc, -t));
  y[s.V + idx] = fma(c.zz, zc, -c.zw * wc);
  t = fma(c.ucy, usn, fma(c.ucx, uwe, fma(c.up, upr, c.wz * zc)));
  y[2 * s.V + idx] = fma(c.uc0, uc, -t);
}

// The same matvec on sine-mode coefficients (every block transformed by the orthonormal 2D
// DST-I, layout [n][l][k]): B0 acts on mode (k, l) as the scalar mu0 = 1 + dt nu (lx_k + ly_l),
// so the stencil becomes a product. wc0 and uc0 hold the coefficients without the stencil's
// centre weight.
__global__ void matvec_spectral_kernel(const double* __restrict__ u, const double* __restrict__ z,
                                       const double* __restrict__ w, double* __restrict__ y, Stencil s,
                                       MatvecCoef c, const double* __restrict__ lx, const double* __restrict__ ly,
                                       double dtnu) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int n = blockIdx.z;
  if (i >= s.Mx || j >= s.My) return;
  const long long idx = static_cast<long long>(n) * s.N + static_cast<long long>(j) * s.Mx + i;
  const double mu0 = fma(dtnu, __ldg(lx + i) + __ldg(ly + j), 1.0);
  const double wc = w[idx];
  const double wnx = n + 1 < s.Nt ? w[idx + s.N] : 0.0;
  const double uc = u[idx];
  const double upr = n > 0 ? u[idx - s.N] : 0.0;
  const double zc = z[idx];
  y[idx] = fma(c.uu, uc, fma(c.wc0 * mu0, wc, -c.wn * wnx));
  y[s.V + idx] = fma(c.zz, zc, -c.zw * wc);
  y[2 * s.V + idx] = fma(c.uc0 * mu0, uc, -fma(c.up, upr, c.wz * zc));
}

// out_n = scale * (B in_n - in_{n+dir}), dir = +1: Jhat^T, dir = -1: Jhat (zero outside 1..Nt)
__global__ void jhat_time_kernel(const double* __restrict__ in, double* __restrict__ out, Stencil s,
                                 int dir, double scale) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int n = blockIdx.z;
  if (i >= s.Mx || j >= s.My) return;
  const long long idx = static_cast<long long>(n) * s.N + static_cast<long long>(j) * s.Mx + i;
  const int nn = n + dir;
  const double nb = (nn >= 0 && nn < s.Nt) ? in[idx + dir * s.N] : 0.0;
  out[idx] = scale * (apply_b(in, idx, i, j, s) - nb);
}

__global__ void rhs_kernel(const double* __restrict__ ut, const double* __restrict__ u0, double* __restrict__ f,
                           long long V, long long N, double h) {
  const long long t = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= V) return;
  f[t] = h * ut[t];
  f[V + t] = 0.0;
  f[2 * V + t] = (t < N && u0) ? u0[t] : 0.0;
}

__global__ void scale_kernel(const double* __restrict__ x, double s, double* __restrict__ y, long long n) {
  const long long t = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  const long long st = static_cast<long long>(gridDim.x) * blockDim.x;
  for (long long k = t; k < n; k += st) y[k] = s * x[k];
}

// y_u = su r_u and y_z = sz r_z (the u and z blocks of P^-1 of Eq 7) in one pass: two
// elements per thread and block with 16-byte loads and stores where all four pointers allow it.
__global__ void scale2_kernel(const double* __restrict__ xu, double su, double* __restrict__ yu,
                              const double* __restrict__ xz, double sz, double* __restrict__ yz, long long n,
                              int vec) {
  const long long t = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  const long long st = static_cast<long long>(gridDim.x) * blockDim.x;
  if (vec) {
    const long long n2 = n / 2;
    const double2* xu2 = reinterpret_cast<const double2*>(xu);
    const double2* xz2 = reinterpret_cast<const double2*>(xz);
    double2* yu2 = reinterpret_cast<double2*>(yu);
    double2* yz2 = reinterpret_cast<double2*>(yz);
    for (long long k = t; k < n2; k += st) {
      const double2 a = __ldcs(xu2 + k), b = __ldcs(xz2 + k);
      __stcs(yu2 + k, make_double2(su * a.x, su * a.y));
      __stcs(yz2 + k, make_double2(sz * b.x, sz * b.y));
    }
    if (t == 0 && (n & 1)) {
      yu[n - 1] = su * xu[n - 1];
      yz[n - 1] = sz * xz[n - 1];
    }
  } else {
    for (long long k = t; k < n; k += st) {
      yu[k] = su * xu[k];
      yz[k] = sz * xz[k];
    }
  }
}

__global__ void axpby_kernel(double alpha, const double* __restrict__ x, double beta, const double* __restrict__ y,
                             double* __restrict__ out, long long n) {
  const long long t = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  const long long st = static_cast<long long>(gridDim.x) * blockDim.x;
  for (long long k = t; k < n; k += st) out[k] = fma(alpha, x[k], beta * y[k]);
}

// Batched matvec: item = a block of 256 points of one instance; coefficients of the su / sz
// terms scaled by the instance's scale_dev entry (1 / eta of the Krylov vector being applied).
// (i, j, n) of a flat block index; 32-bit divisions while the block has fewer than 2^32
// points (64-bit integer division is built from FP64 arithmetic, the scarce pipe here)
__device__ __forceinline__ void split_index(long long idx, const MatvecJob& J, int& i, int& j, int& n) {
  if (J.V < (1LL << 32)) {
    const unsigned int u = static_cast<unsigned int>(idx), mx = J.Mx, my = J.My;
    const unsigned int r = u / mx;
    i = static_cast<int>(u - r * mx);
    const unsigned int nn = r / my;
    j = static_cast<int>(r - nn * my);
    n = static_cast<int>(nn);
  } else {
    const long long r = idx / J.Mx;
    i = static_cast<int>(idx - r * J.Mx);
    j = static_cast<int>(r % J.My);
    n = static_cast<int>(r / J.My);
  }
}

__global__ void matvec_batched(const MatvecJob* __restrict__ jobs, const long long* __restrict__ prefix, int nj,
                               long long total, const double* __restrict__ scale_dev) {
  __shared__ long long sp[KKT_BATCH_MAX + 1];
  batch_prefix_load(sp, prefix, nj);
  for (long long t = blockIdx.x; t < total; t += gridDim.x) {
    const int k = batch_find(sp, nj, t);
    const MatvecJob J = jobs[k];   // (a register copy: the stores below cannot alias it)
    const double e = scale_dev[J.scale_index];
    const long long idx0 = (t - sp[k]) * kMvItem;
    const long long idx1 = idx0 + kMvItem < J.V ? idx0 + kMvItem : J.V;
    if (J.spectral) {
      for (long long idx = idx0 + threadIdx.x; idx < idx1; idx += blockDim.x) {
        int i, j, n;
        split_index(idx, J, i, j, n);
        const double mu0 = fma(J.dtnu, __ldg(J.lx + i) + __ldg(J.ly + j), 1.0);
        const double wc = J.w[idx];
        const double wnx = n + 1 < J.Nt ? J.w[idx + J.N] : 0.0;
        const double uc = J.u[idx];
        const double upr = n > 0 ? J.u[idx - J.N] : 0.0;
        const double zc = J.z[idx];
        J.y[idx] = fma(J.uu * e, uc, fma(J.wc0 * mu0, wc, -J.wn * wnx));
        J.y[J.V + idx] = fma(J.zz * e, zc, -J.zw * wc);
        J.y[2 * J.V + idx] = fma(J.uc0 * e * mu0, uc, -fma(J.up * e, upr, (J.wz * e) * zc));
      }
      continue;
    }
    for (long long idx = idx0 + threadIdx.x; idx < idx1; idx += blockDim.x) {
      int i, j, n;
      split_index(idx, J, i, j, n);
      const bool hw = i > 0, he = i + 1 < J.Mx, hs = j > 0, hn = j + 1 < J.My;
      const double wc = J.w[idx];
      const double wwe = (hw ? J.w[idx - 1] : 0.0) + (he ? J.w[idx + 1] : 0.0);
      const double wsn = (hs ? J.w[idx - J.Mx] : 0.0) + (hn ? J.w[idx + J.Mx] : 0.0);
      const double wnx = n + 1 < J.Nt ? J.w[idx + J.N] : 0.0;
      const double uc = J.u[idx];
      const double uwe = (hw ? J.u[idx - 1] : 0.0) + (he ? J.u[idx + 1] : 0.0);
      const double usn = (hs ? J.u[idx - J.Mx] : 0.0) + (hn ? J.u[idx + J.Mx] : 0.0);
      const double upr = n > 0 ? J.u[idx - J.N] : 0.0;
      const double zc = J.z[idx];
      double tt = fma(J.wcy, wsn, fma(J.wcx, wwe, J.wn * wnx));
      J.y[idx] = fma(J.uu * e, uc, fma(J.wc0, wc, -tt));
      J.y[J.V + idx] = fma(J.zz * e, zc, -J.zw * wc);
      tt = fma(J.ucy * e, usn, fma(J.ucx * e, uwe, fma(J.up * e, upr, (J.wz * e) * zc)));
      J.y[2 * J.V + idx] = fma(J.uc0 * e, uc, -tt);
    }
  }
}

Stencil make_stencil(const Geometry& g, double shift) {
  Stencil s;
  s.Mx = g.Mx;
  s.My = g.My;
  s.Nt = g.Nt;
  s.N = g.N;
  s.V = g.V;
  s.cx = g.cx;
  s.cy = g.cy;
  s.c0 = shift + 2.0 * g.cx + 2.0 * g.cy;
  return s;
}

}  // namespace

int launch_matvec(const kkt_handle* h, const double* u, double su, const double* z, double sz,
                  const double* w, double sw, double* y, cudaStream_t st, double ou, double oz, double ow) {
  const Geometry& g = h->g;
  const Stencil s = make_stencil(g, 1.0);   // B0 = I + dt nu A
  MatvecCoef c;
  c.uu = ou * g.h * su;
  c.wc0 = ou * sw * s.c0;
  c.wcx = ou * sw * s.cx;
  c.wcy = ou * sw * s.cy;
  c.wn = ou * sw;
  c.zz = oz * g.omega * g.h * sz;
  c.zw = oz * g.dt * sw;
  c.uc0 = ow * su * s.c0;
  c.ucx = ow * su * s.cx;
  c.ucy = ow * su * s.cy;
  c.up = ow * su;
  c.wz = ow * g.dt * sz;
  dim3 tb(32, 8);
  dim3 grid((g.Mx + 31) / 32, (g.My + 7) / 8, g.Nt);
  // 16 FP64 instructions (12 FMA) per point: 28 flops; 3 blocks in, 3 out
  ProfScope ps(KKT_K_MATVEC, st, 28.0 * g.V, 48.0 * g.V);
  matvec_kernel<<<grid, tb, 0, st>>>(u, z, w, y, s, c);
  KKT_CUDA_TRY(cudaGetLastError());
  return KKT_OK;
}

int launch_matvec_spectral(const kkt_handle* h, const double* u, double su, const double* z, double sz,
                           const double* w, double sw, double* y, cudaStream_t st, double ou, double oz, double ow) {
  const Geometry& g = h->g;
  const Stencil s = make_stencil(g, 1.0);
  MatvecCoef c;
  c.uu = ou * g.h * su;
  c.wc0 = ou * sw;
  c.wcx = c.wcy = 0.0;
  c.wn = ou * sw;
  c.zz = oz * g.omega * g.h * sz;
  c.zw = oz * g.dt * sw;
  c.uc0 = ow * su;
  c.ucx = c.ucy = 0.0;
  c.up = ow * su;
  c.wz = ow * g.dt * sz;
  dim3 tb(32, 8);
  dim3 grid((g.Mx + 31) / 32, (g.My + 7) / 8, g.Nt);
  // 12 FP64 instructions per point; 3 blocks in, 3 out
  ProfScope ps(KKT_K_MATVEC, st, 20.0 * g.V, 48.0 * g.V);
  matvec_spectral_kernel<<<grid, tb, 0, st>>>(u, z, w, y, s, c, h->d_lx, h->d_ly, g.dtnu);
  KKT_CUDA_TRY(cudaGetLastError());
  return KKT_OK;
}

int matvec_batched_prepare(BatchSlot& slot, const MatvecJob* jobs, int nj) {
  if (nj < 1 || nj > KKT_BATCH_MAX) return set_error(KKT_ERR_INVALID_ARG, "batched jobs out of range");
  std::vector<long long> pre(nj + 1, 0);
  double V = 0;
  for (int k = 0; k < nj; ++k) {
    pre[k + 1] = pre[k] + (jobs[k].V + kMvItem - 1) / kMvItem;
    V += static_cast<double>(jobs[k].V);
  }
  if (!slot.mv) {
    KKT_CUDA_TRY(cudaMalloc(&slot.mv, KKT_BATCH_MAX * sizeof(MatvecJob)));
    KKT_CUDA_TRY(cudaMalloc(&slot.mv_prefix, (KKT_BATCH_MAX + 1) * sizeof(long long)));
  }
  KKT_CUDA_TRY(cudaMemcpy(slot.mv, jobs, nj * sizeof(MatvecJob), cudaMemcpyHostToDevice));
  KKT_CUDA_TRY(cudaMemcpy(slot.mv_prefix, pre.data(), (nj + 1) * sizeof(long long), cudaMemcpyHostToDevice));
  slot.mv_total = pre[nj];
  slot.mv_V = V;
  slot.njobs = nj;
  return KKT_OK;
}

int matvec_batched_launch(const BatchSlot& slot, const double* scale_dev, cudaStream_t st) {
  if (slot.mv_total <= 0) return KKT_OK;
  int dev = 0, sms = 0;
  KKT_CUDA_TRY(cudaGetDevice(&dev));
  KKT_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const long long grid = std::min<long long>(slot.mv_total, static_cast<long long>(sms) * 8);
  ProfScope ps(KKT_K_MATVEC, st, 28.0 * slot.mv_V, 48.0 * slot.mv_V);
  matvec_batched<<<static_cast<unsigned>(grid), 256, 0, st>>>(slot.mv, slot.mv_prefix, slot.njobs, slot.mv_total,
                                                              scale_dev);
  KKT_CUDA_TRY(cudaGetLastError());
  return KKT_OK;
}

int launch_jhat_time(const kkt_handle* h, const double* in, double* out, int dir, double scale,
                     cudaStream_t st) {
  const Geometry& g = h->g;
  const Stencil s = make_stencil(g, g.a);   // Bhat = a I + dt nu A
  dim3 tb(32, 8);
  dim3 grid((g.Mx + 31) / 32, (g.My + 7) / 8, g.Nt);
  ProfScope ps(KKT_K_MATVEC, st);
  jhat_time_kernel<<<grid, tb, 0, st>>>(in, out, s, dir, scale);
  KKT_CUDA_TRY(cudaGetLastError());
  return KKT_OK;
}

int launch_build_rhs(const kkt_handle* h, const double* ut, const double* u0, double* f, cudaStream_t st) {
  const Geometry& g = h->g;
  const int tb = 256;
  const long long nb = (g.V + tb - 1) / tb;
  ProfScope ps(KKT_K_AXPY, st);
  rhs_kernel<<<static_cast<unsigned>(nb), tb, 0, st>>>(ut, u0, f, g.V, g.N, g.h);
  KKT_CUDA_TRY(cudaGetLastError());
  return KKT_OK;
}

int launch_scale(const double* x, double s, double* y, long long n, cudaStream_t st) {
  if (n <= 0) return KKT_OK;
  const int tb = 256;
  long long nb = (n + tb - 1) / tb;
  if (nb > 65535LL * 8) nb = 65535LL * 8;
  ProfScope ps(KKT_K_AXPY, st);
  scale_kernel<<<static_cast<unsigned>(nb), tb, 0, st>>>(x, s, y, n);
  KKT_CUDA_TRY(cudaGetLastError());
  return KKT_OK;
}

int launch_scale2(const double* xu, double su, double* yu, const double* xz, double sz, double* yz, long long n,
                  cudaStream_t st) {
  if (n <= 0) return KKT_OK;
  const int tb = 256;
  int dev = 0, sms = 0;
  KKT_CUDA_TRY(cudaGetDevice(&dev));
  KKT_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int vec = ((reinterpret_cast<uintptr_t>(xu) | reinterpret_cast<uintptr_t>(yu) | reinterpret_cast<uintptr_t>(xz) |
                    reinterpret_cast<uintptr_t>(yz)) & 15) == 0;
  const long long work = vec ? n / 2 : n;
  const long long nb = std::min<long long>((work + tb - 1) / tb, static_cast<long long>(sms) * 8);
  ProfScope ps(KKT_K_AXPY, st, static_cast<double>(n) * 2.0, 32.0 * static_cast<double>(n));
  scale2_kernel<<<static_cast<unsigned>(std::max<long long>(nb, 1)), tb, 0, st>>>(xu, su, yu, xz, sz, yz, n, vec);
  KKT_CUDA_TRY(cudaGetLastError());
  return KKT_OK;
}

int launch_axpby(double alpha, const double* x, double beta, const double* y, double* out, long long n,
                 cudaStream_t st) {
  if (n <= 0) return KKT_OK;
  const int tb = 256;
  long long nb = (n + tb - 1) / tb;
  if (nb > 65535LL * 8) nb = 65535LL * 8;
  ProfScope ps(KKT_K_AXPY, st);
  axpby_kernel<<<static_cast<unsigned>(nb), tb, 0, st>>>(alpha, x, beta, y, out, n);
  KKT_CUDA_TRY(cudaGetLastError());
  return KKT_OK;
}

}  // namespace kkt
