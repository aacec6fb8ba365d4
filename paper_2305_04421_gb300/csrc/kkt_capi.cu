// Exported C ABI (include/kkt.h): handle set-up, the block preconditioner of Eq 7 built
// from the device kernels, and the flexible GMRES driver of Section 4.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <functional>
#include <string>
#include <vector>

#include "kkt_internal.cuh"

namespace kkt {

namespace {
thread_local std::string g_last_error;
}

int set_error(int status, const std::string& msg) {
  g_last_error = msg;
  return status;
}

namespace {

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

// Subdomains of Section 3 (balanced split b_s = floor(s Nt / N_D)), D_s ownership, the linear
// coarse function phi of Eq 14 per owned node, and the coarse moment matrices.
void build_decomp(int Nt, int n_sub, int pou, TimeDecomp& td) {
  td = TimeDecomp();
  td.n_sub = n_sub;
  std::vector<long long> b(n_sub + 1);
  for (int s = 0; s <= n_sub; ++s) b[s] = static_cast<long long>(s) * Nt / n_sub;
  td.owner.assign(Nt, 0);
  td.phi.assign(Nt, 0.0);
  for (int s = 0; s < n_sub; ++s) {
    const int lo = static_cast<int>(b[s]), hi = static_cast<int>(b[s + 1]);
    const int first = std::max(lo, 1), last = hi;
    int of, ol;
    if (pou == KKT_POU_LEFT) {
      of = lo + 1;
      ol = hi;
    } else {
      of = first;
      ol = (s == n_sub - 1) ? hi : hi - 1;
    }
    const int m = hi - lo;
    td.first.push_back(first);
    td.last.push_back(last);
    td.ofirst.push_back(of);
    td.olast.push_back(ol);
    td.max_len = std::max(td.max_len, last - first + 1);
    double p0[3] = {0, 0, 0}, p1[3] = {0, 0, 0}, p2[3] = {0, 0, 0};
    for (int n = of; n <= ol; ++n) {
      const double ph = -1.0 + 2.0 * (n - lo) / m;
      td.owner[n - 1] = s;
      td.phi[n - 1] = ph;
      p0[0] += 1.0;
      p0[1] += ph;
      p0[2] += ph * ph;
      if (n >= 2) {
        p1[0] += 1.0;
        p1[1] += ph;
        p1[2] += ph * ph;
      }
      if (n + 1 <= ol) {
        const double pn = -1.0 + 2.0 * (n + 1 - lo) / m;
        p2[0] += 2.0;
        p2[1] += ph + pn;
        p2[2] += 2.0 * ph * pn;
      }
    }
    for (int t = 0; t < 3; ++t) {
      td.P0.push_back(p0[t]);
      td.P1.push_back(p1[t]);
      td.P2.push_back(p2[t]);
    }
  }
}

int upload_decomp(kkt_handle* h) {
  const TimeDecomp& td = h->td;
  DeviceDecomp& dd = h->dd;
  if (dd.base) cudaFree(dd.base);
  dd = DeviceDecomp();
  const int S = td.n_sub, Nt = h->g.Nt;
  const size_t ints = 4 * S + Nt;
  const size_t ints_bytes = ((ints * sizeof(int) + 255) / 256) * 256;
  const size_t dbl = Nt + 9 * S;
  const size_t total = ints_bytes + dbl * sizeof(double) + Nt * sizeof(float);
  void* base = nullptr;
  KKT_CUDA_TRY(cudaMalloc(&base, total));
  std::vector<char> host(total, 0);
  int* ip = reinterpret_cast<int*>(host.data());
  std::copy(td.first.begin(), td.first.end(), ip);
  std::copy(td.last.begin(), td.last.end(), ip + S);
  std::copy(td.ofirst.begin(), td.ofirst.end(), ip + 2 * S);
  std::copy(td.olast.begin(), td.olast.end(), ip + 3 * S);
  std::copy(td.owner.begin(), td.owner.end(), ip + 4 * S);
  double* dp = reinterpret_cast<double*>(host.data() + ints_bytes);
  std::copy(td.phi.begin(), td.phi.end(), dp);
  for (int s = 0; s < S; ++s)
    for (int t = 0; t < 3; ++t) {
      dp[Nt + 9 * s + t] = td.P0[3 * s + t];
      dp[Nt + 9 * s + 3 + t] = td.P1[3 * s + t];
      dp[Nt + 9 * s + 6 + t] = td.P2[3 * s + t];
    }
  float* fp = reinterpret_cast<float*>(dp + dbl);
  for (int n = 0; n < Nt; ++n) fp[n] = static_cast<float>(td.phi[n]);
  KKT_CUDA_TRY(cudaMemcpy(base, host.data(), total, cudaMemcpyHostToDevice));
  int* dip = static_cast<int*>(base);
  dd.base = base;
  dd.n_sub = S;
  dd.max_len = td.max_len;
  dd.Nt = Nt;
  dd.first = dip;
  dd.last = dip + S;
  dd.ofirst = dip + 2 * S;
  dd.olast = dip + 3 * S;
  dd.owner = dip + 4 * S;
  dd.phi = reinterpret_cast<double*>(static_cast<char*>(base) + ints_bytes);
  dd.moments = dd.phi + Nt;
  dd.phi_f = reinterpret_cast<float*>(dd.phi + dbl);
  return KKT_OK;
}

template <typename T>
int dev_alloc(kkt_handle* h, T** p, size_t count) {
  if (*p) {
    cudaFree(*p);
    *p = nullptr;
  }
  if (count == 0) return KKT_OK;
  const cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return set_error(e == cudaErrorMemoryAllocation ? KKT_ERR_OOM : KKT_ERR_CUDA,
                     std::string("cudaMalloc of ") + std::to_string(count * sizeof(T)) + " bytes: " +
                         cudaGetErrorString(e));
  }
  h->bytes += count * sizeof(T);
  return KKT_OK;
}

// Everything that depends on the options: geometry, eigenvalue tables, decomposition, sweep launch shape.
int configure(kkt_handle* h) {
  Geometry& g = h->g;
  const kkt_options& o = h->opt;
  g.Lx = o.Lx;
  g.Ly = o.Ly;
  g.dx = g.Lx / g.nx;
  g.dy = g.Ly / g.ny;
  g.dt = g.T / g.Nt;
  g.h = g.dt * g.dx * g.dy;
  g.a = 1.0 - o.jhat_sign * g.dt / std::sqrt(g.omega);
  g.dtnu = g.dt * g.nu;
  g.cx = g.dtnu / (g.dx * g.dx);
  g.cy = g.dtnu / (g.dy * g.dy);
  const double pi = 3.14159265358979323846;
  std::vector<double> lx(g.Mx), ly(g.My);
  for (int k = 1; k <= g.Mx; ++k) {
    const double s = std::sin(k * pi / (2.0 * g.nx));
    lx[k - 1] = 4.0 / (g.dx * g.dx) * s * s;
  }
  for (int l = 1; l <= g.My; ++l) {
    const double s = std::sin(l * pi / (2.0 * g.ny));
    ly[l - 1] = 4.0 / (g.dy * g.dy) * s * s;
  }
  if (!h->d_lx) KKT_TRY(dev_alloc(h, &h->d_lx, g.Mx));
  if (!h->d_ly) KKT_TRY(dev_alloc(h, &h->d_ly, g.My));
  KKT_CUDA_TRY(cudaMemcpy(h->d_lx, lx.data(), g.Mx * sizeof(double), cudaMemcpyHostToDevice));
  KKT_CUDA_TRY(cudaMemcpy(h->d_ly, ly.data(), g.My * sizeof(double), cudaMemcpyHostToDevice));
  build_decomp(g.Nt, g.n_sub, o.pou, h->td);
  KKT_TRY(upload_decomp(h));
  // reduced-precision forms: tensor-core transform plan over the padded mode grid
  const bool mixed = o.precision != KKT_PREC_FP64;
  const int bf16 = o.precision == KKT_PREC_BF16;
  if (h->tc.q && (!mixed || h->tc.bf16 != bf16)) {
    h->bytes -= h->tc.bytes;
    tc_plan_destroy(h->tc);
  }
  long long modes = g.N;
  if (mixed) {
    if (!h->tc.q) {
      KKT_TRY(tc_plan_create(h->tc, g.nx, g.Nt, bf16));
      h->bytes += h->tc.bytes;
    }
    const int P = h->tc.P;
    std::vector<double> lxp(P, 0.0), lyp(P, 0.0);
    std::copy(lx.begin(), lx.end(), lxp.begin());
    std::copy(ly.begin(), ly.end(), lyp.begin());
    if (!h->d_lx_pad) KKT_TRY(dev_alloc(h, &h->d_lx_pad, P));
    if (!h->d_ly_pad) KKT_TRY(dev_alloc(h, &h->d_ly_pad, P));
    KKT_CUDA_TRY(cudaMemcpy(h->d_lx_pad, lxp.data(), P * sizeof(double), cudaMemcpyHostToDevice));
    KKT_CUDA_TRY(cudaMemcpy(h->d_ly_pad, lyp.data(), P * sizeof(double), cudaMemcpyHostToDevice));
    modes = std::max(modes, static_cast<long long>(P) * P);
  }
  if (modes > h->coarse_modes) {
    KKT_TRY(dev_alloc(h, &h->coarse_c, 2 * static_cast<size_t>(g.n_sub) * modes));
    KKT_TRY(dev_alloc(h, &h->coarse_w, 2 * static_cast<size_t>(g.n_sub) * modes));
    h->coarse_modes = modes;
  }
  // block-Thomas factors of the coarse operator, per mode (FP64), recomputed for these options
  if (!h->coarse_f) KKT_TRY(dev_alloc(h, &h->coarse_f, 3 * static_cast<size_t>(g.n_sub) * g.N));
  KKT_TRY(spectral_coarse_factor(h, false, h->coarse_f, nullptr));
  if (mixed) {
    KKT_TRY(dev_alloc(h, &h->coarse_f_pad, 3 * static_cast<size_t>(g.n_sub) * h->tc.P * h->tc.P));
    KKT_TRY(spectral_coarse_factor(h, true, h->coarse_f_pad, nullptr));
  } else if (h->coarse_f_pad) {
    cudaFree(h->coarse_f_pad);
    h->coarse_f_pad = nullptr;
  }
  // the cyclic reduction's factors (only when that is the FP64 path's coarse solve). The factor
  // kernel runs on the legacy default stream; this device-wide sync must stay, so that no solve
  // on a caller's (non-blocking) stream reads h->cr_factors before they are written.
  KKT_TRY(spectral_cr_factor(h));
  KKT_CUDA_TRY(cudaDeviceSynchronize());
  // sweep storage: shared memory when a subdomain's nodes fit (32 threads x max_len doubles
  // within 200 KB), else a global scratch sized for every mode
  const size_t words = h->opt.local == KKT_LOCAL_RAS ? 2 : 1;
  if (words * h->td.max_len * 32 * sizeof(double) > 200 * 1024) {
    if (h->vscratch) cudaFree(h->vscratch);
    h->vscratch = nullptr;
    KKT_TRY(dev_alloc(h, &h->vscratch, words * g.n_sub * h->td.max_len * modes));
  } else if (h->vscratch) {
    cudaFree(h->vscratch);
    h->vscratch = nullptr;
  }
  return KKT_OK;
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  const cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

// Device-side address of a pinned (mapped) host buffer; nullptr for any other memory.
const void* mapped_host(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// dst[0..n) = src[0..n) with the SMs, one side being mapped host memory: 16-byte accesses when
// both are 16-byte aligned, four independent loads per thread in flight to cover the link's
// latency; every element is copied by exactly one thread.
__global__ void link_copy_kernel(const double* __restrict__ src, double* __restrict__ dst, long long n) {
  const long long t = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
  const bool vec = ((reinterpret_cast<unsigned long long>(src) | reinterpret_cast<unsigned long long>(dst)) & 15) == 0;
  if (vec) {
    const double2* s2 = reinterpret_cast<const double2*>(src);
    double2* d2 = reinterpret_cast<double2*>(dst);
    const long long n2 = n / 2;
    long long i = t;
    for (; i + 3 * stride < n2; i += 4 * stride) {
      const double2 a = s2[i], b = s2[i + stride], c = s2[i + 2 * stride], d = s2[i + 3 * stride];
      d2[i] = a;
      d2[i + stride] = b;
      d2[i + 2 * stride] = c;
      d2[i + 3 * stride] = d;
    }
    for (; i < n2; i += stride) d2[i] = s2[i];
    if (t == 0 && (n & 1)) dst[n - 1] = src[n - 1];
  } else {
    for (long long i = t; i < n; i += stride) dst[i] = src[i];
  }
}

// Host <-> device copy of n doubles for kkt_solve's staging (one side is device memory).
int stage_copy(const kkt_handle* h, double* dst, const double* src, long long n, cudaMemcpyKind kind,
               cudaStream_t st) {
  const void* mapped = nullptr;
  if (h->staging == KKT_STAGING_AUTO)
    mapped = mapped_host(kind == cudaMemcpyHostToDevice ? static_cast<const void*>(src) : static_cast<const void*>(dst));
  if (!mapped) {
    KKT_CUDA_TRY(cudaMemcpyAsync(dst, src, n * sizeof(double), kind, st));
    return KKT_OK;
  }
  const double* s = kind == cudaMemcpyHostToDevice ? static_cast<const double*>(mapped) : src;
  double* d = kind == cudaMemcpyHostToDevice ? dst : static_cast<double*>(const_cast<void*>(mapped));
  int sms = 0;
  KKT_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
  link_copy_kernel<<<static_cast<unsigned>(sms * 8), 256, 0, st>>>(s, d, n);
  KKT_CUDA_TRY(cudaGetLastError());
  return KKT_OK;
}

int check_handle(const kkt_handle* h) {
  if (!h) return set_error(KKT_ERR_INVALID_ARG, "null handle");
  return KKT_OK;
}

int check_ptrs(std::initializer_list<const void*> ps) {
  for (const void* p : ps) {
    if (!p) return set_error(KKT_ERR_INVALID_ARG, "null vector pointer");
    if (reinterpret_cast<uintptr_t>(p) % 8) return set_error(KKT_ERR_INVALID_ARG, "vector pointer not 8-byte aligned");
    if (!is_device_ptr(p)) return set_error(KKT_ERR_INVALID_ARG, "vector pointer is not device memory");
  }
  return KKT_OK;
}

int ensure_precision(const kkt_handle* h) {
  if (h->opt.precision != KKT_PREC_FP64)
    return set_error(KKT_ERR_UNSUPPORTED, "this entry point runs in FP64 only");
  return KKT_OK;
}

// y_w = S-hat_2level^{-1} (scale * r_w): DST, spectral two-level solve, inverse DST.
// FP64: the FFT-based transforms. BF16 / TF32: pack into padded slices, two tensor-core
// transforms into FP32 coefficients, FP32 sweeps (FP64 coarse solve), two transforms back.
int schur_precond_w(kkt_handle* h, const double* rw, double scale, double* yw, cudaStream_t st) {
  if (h->opt.precision == KKT_PREC_FP64) {
    KKT_TRY(dst2d(h, rw, h->spec, st));
    KKT_TRY(spectral_schur_precond(h, h->spec, h->spec2, scale, st));
    KKT_TRY(dst2d(h, h->spec2, yw, st));
    return KKT_OK;
  }
  const TcPlan& t = h->tc;
  const bool sp = h->opt.tc_split != 0;
  const int mid = sp ? 3 : (t.bf16 ? 0 : 1);
  const int valid = h->g.nx - 1;
  KKT_TRY(tc_pack(t, rw, valid, st));                              // hi (+ lo) parts, unscaled
  KKT_TRY(tc_gemm(t, 0, mid, t.x1, valid, st, sp, t.x1_lo));        // along x: [n][j][i] -> [n][k][j]
  KKT_TRY(tc_gemm(t, 1, 1, t.rhat, valid, st, sp));                 // along y: -> [n][l][k], FP32
  KKT_TRY(spectral_schur_precond_mixed(h, t.rhat, scale, t.yin, sp ? t.yin_lo : nullptr, t.bf16, st));
  KKT_TRY(tc_gemm(t, 2, mid, t.x0, valid, st, sp, t.x0_lo));        // back along x: [n][l][k] -> [n][i][l]
  KKT_TRY(tc_gemm(t, 0, 2, yw, valid, st, sp));                     // back along y: -> [n][j][i], FP64
  return KKT_OK;
}

}  // namespace

void release_krylov(kkt_handle* h) {
  for (double** b : {&h->kV, &h->kZw, &h->kx, &h->kf, &h->ks_f, &h->ks_x}) {
    cudaFree(*b);
    *b = nullptr;
  }
  h->kry_restart = 0;
}

namespace {

int ensure_krylov(kkt_handle* h) {
  const int m = h->opt.restart;
  // the small reduction and coefficient buffers, also when the basis storage is lent
  if (!h->red) KKT_TRY(dev_alloc(h, &h->red, static_cast<size_t>(krylov_partial_capacity())));
  if (!h->red_out) KKT_TRY(dev_alloc(h, &h->red_out, 128));
  if (!h->dcoef) KKT_TRY(dev_alloc(h, &h->dcoef, 4 * 128));
  if (!h->h_red) KKT_CUDA_TRY(cudaMallocHost(&h->h_red, 6 * 128 * sizeof(double)));
  if (h->kry_restart == m && h->kV) return KKT_OK;
  const size_t n3 = 3 * static_cast<size_t>(h->g.V);
  KKT_TRY(dev_alloc(h, &h->kV, (m + 1) * n3));
  KKT_TRY(dev_alloc(h, &h->kZw, static_cast<size_t>(m) * h->g.V));
  h->kry_restart = m;
  return KKT_OK;
}

}  // namespace
}  // namespace kkt

using namespace kkt;

extern "C" {

const char* kkt_last_error(void) { return kkt::g_last_error.c_str(); }

const char* kkt_status_string(int status) {
  switch (status) {
    case KKT_OK: return "ok";
    case KKT_NOT_CONVERGED: return "not converged within maxit";
    case KKT_ERR_INVALID_ARG: return "invalid argument";
    case KKT_ERR_OOM: return "out of device memory";
    case KKT_ERR_CUDA: return "CUDA error";
    case KKT_ERR_NONFINITE: return "non-finite value";
    case KKT_ERR_TIMEOUT: return "device wait timed out";
    case KKT_ERR_BREAKDOWN: return "Krylov breakdown";
    case KKT_ERR_UNSUPPORTED: return "unsupported configuration";
    default: return "unknown status";
  }
}

int kkt_default_options(kkt_options* opt) {
  if (!opt) return set_error(KKT_ERR_INVALID_ARG, "null options");
  opt->precision = KKT_PREC_FP64;
  opt->coarse = KKT_COARSE_EXACT;
  opt->variant = KKT_MULTIPLICATIVE;
  opt->pou = KKT_POU_LEFT;
  opt->restart = 30;
  opt->jhat_sign = -1;
  opt->residual_norm = KKT_NORM_L2;
  opt->tc_split = 1;
  opt->orth = KKT_ORTH_MGS2;
  opt->basis = KKT_BASIS_PHYSICAL;
  opt->local = KKT_LOCAL_RASQ;
  opt->Lx = 1.0;
  opt->Ly = 1.0;
  opt->coarse_solve = KKT_COARSE_SOLVE_AUTO;
  return KKT_OK;
}

kkt_handle* kkt_create(int nx, int ny, int Nt, double T, double nu, double omega, int n_sub) {
  if (nx < 2 || ny < 2 || nx > 1024 || ny > 1024) {
    set_error(KKT_ERR_INVALID_ARG, "nx, ny must be in [2, 1024]");
    return nullptr;
  }
  if (Nt < 2 || Nt > 65535) {
    set_error(KKT_ERR_INVALID_ARG, "Nt must be in [2, 65535]");
    return nullptr;
  }
  if (n_sub < 1 || Nt / n_sub < 2 || n_sub > 65535) {
    set_error(KKT_ERR_INVALID_ARG, "n_sub must satisfy 1 <= n_sub and Nt / n_sub >= 2");
    return nullptr;
  }
  if (!finite_pos(T) || !finite_pos(nu) || !finite_pos(omega)) {
    set_error(KKT_ERR_INVALID_ARG, "T, nu and omega must be positive and finite");
    return nullptr;
  }
  kkt_handle* h = new kkt_handle();
  cudaGetDevice(&h->device);
  Geometry& g = h->g;
  g.nx = nx;
  g.ny = ny;
  g.Nt = Nt;
  g.n_sub = n_sub;
  g.Mx = nx - 1;
  g.My = ny - 1;
  g.N = static_cast<long long>(g.Mx) * g.My;
  g.V = g.N * Nt;
  g.T = T;
  g.nu = nu;
  g.omega = omega;
  kkt_default_options(&h->opt);
  int st = configure(h);
  if (st >= 0) st = dst_plan_create(h->dst_x, nx);
  if (st >= 0) st = dst_plan_create(h->dst_y, ny);
  if (st >= 0) st = dev_alloc(h, &h->spec, g.V);
  if (st >= 0) st = dev_alloc(h, &h->spec2, g.V);
  if (st >= 0) st = dst_autotune(h);
  if (st >= 0) st = dev_alloc(h, &h->red, static_cast<size_t>(krylov_partial_capacity()));
  if (st >= 0) st = dev_alloc(h, &h->red_out, 128);
  if (st < 0) {
    const std::string msg = kkt::g_last_error;
    kkt_destroy(h);
    set_error(st, msg);
    return nullptr;
  }
  return h;
}

void kkt_destroy(kkt_handle* h) {
  if (!h) return;
  dst_plan_destroy(h->dst_x);
  dst_plan_destroy(h->dst_y);
  if (h->tc.q) tc_plan_destroy(h->tc);
  oz_plan_destroy(h->oz);
  cudaFree(h->d_lx_pad);
  cudaFree(h->d_ly_pad);
  cudaFree(h->learn_c);
  cudaFree(h->learn_feat);
  cudaFree(h->learn_x);
  cudaFree(h->learn_count);
  if (h->dd.base) cudaFree(h->dd.base);
  cudaFree(h->ks_f);
  cudaFree(h->ks_x);
  cudaFree(h->d_lx);
  cudaFree(h->d_ly);
  cudaFree(h->spec);
  cudaFree(h->spec2);
  cudaFree(h->coarse_c);
  cudaFree(h->coarse_w);
  cudaFree(h->coarse_f);
  cudaFree(h->coarse_f_pad);
  cudaFree(h->cr_factors);
  cudaFree(h->vscratch);
  cudaFree(h->kV);
  cudaFree(h->kZw);
  cudaFree(h->kx);
  cudaFree(h->kf);
  cudaFree(h->red);
  cudaFree(h->red_out);
  cudaFree(h->dcoef);
  if (h->h_red) cudaFreeHost(h->h_red);
  delete h;
}

int kkt_set_options(kkt_handle* h, const kkt_options* opt) {
  KKT_TRY(check_handle(h));
  if (!opt) return set_error(KKT_ERR_INVALID_ARG, "null options");
  if (opt->precision < KKT_PREC_FP64 || opt->precision > KKT_PREC_TF32)
    return set_error(KKT_ERR_INVALID_ARG, "precision out of range");
  if (opt->coarse < KKT_COARSE_EXACT || opt->coarse > KKT_COARSE_LEARNED)
    return set_error(KKT_ERR_INVALID_ARG, "coarse out of range");
  if (opt->variant != KKT_MULTIPLICATIVE && opt->variant != KKT_ADDITIVE)
    return set_error(KKT_ERR_INVALID_ARG, "variant out of range");
  if (opt->pou != KKT_POU_LEFT && opt->pou != KKT_POU_RIGHT) return set_error(KKT_ERR_INVALID_ARG, "pou out of range");
  if (opt->restart < 1 || opt->restart > 32) return set_error(KKT_ERR_INVALID_ARG, "restart must be in [1, 32]");
  if (opt->jhat_sign != -1 && opt->jhat_sign != 1) return set_error(KKT_ERR_INVALID_ARG, "jhat_sign must be -1 or +1");
  if (opt->residual_norm != KKT_NORM_L2 && opt->residual_norm != KKT_NORM_EUCLIDEAN)
    return set_error(KKT_ERR_INVALID_ARG, "residual_norm out of range");
  if (opt->tc_split != 0 && opt->tc_split != 1) return set_error(KKT_ERR_INVALID_ARG, "tc_split must be 0 or 1");
  if (opt->orth < KKT_ORTH_MGS || opt->orth > KKT_ORTH_MGS8) return set_error(KKT_ERR_INVALID_ARG, "orth out of range");
  if (opt->local != KKT_LOCAL_RASQ && opt->local != KKT_LOCAL_RAS) return set_error(KKT_ERR_INVALID_ARG, "local out of range");
  if (opt->basis != KKT_BASIS_PHYSICAL && opt->basis != KKT_BASIS_SPECTRAL)
    return set_error(KKT_ERR_INVALID_ARG, "basis out of range");
  if (opt->basis == KKT_BASIS_SPECTRAL && opt->precision != KKT_PREC_FP64)
    return set_error(KKT_ERR_UNSUPPORTED, "the spectral basis runs the FP64 preconditioner (it has no transforms)");
  if (!finite_pos(opt->Lx) || !finite_pos(opt->Ly)) return set_error(KKT_ERR_INVALID_ARG, "Lx, Ly must be positive");
  if (opt->coarse_solve < KKT_COARSE_SOLVE_AUTO || opt->coarse_solve > KKT_COARSE_SOLVE_CYCLIC)
    return set_error(KKT_ERR_INVALID_ARG, "coarse_solve out of range");
  // with the shared node given to the later subdomain, the first subdomain owns nodes
  // 1 .. b_1 - 1; its linear coarse function needs two of them
  if (opt->pou == KKT_POU_RIGHT && h->g.Nt / h->g.n_sub < 3)
    return set_error(KKT_ERR_INVALID_ARG, "pou=right needs Nt / n_sub >= 3");
  if (opt->precision != KKT_PREC_FP64 && h->g.nx != h->g.ny)
    return set_error(KKT_ERR_UNSUPPORTED, "the tensor-core transforms need a square grid (nx == ny)");
  if (opt->coarse == KKT_COARSE_LEARNED && !h->mlp)
    return set_error(KKT_ERR_INVALID_ARG, "coarse = learned needs a network attached with kkt_attach_mlp");
  h->opt = *opt;
  return configure(h);
}

int kkt_get_options(const kkt_handle* h, kkt_options* opt) {
  KKT_TRY(check_handle(h));
  if (!opt) return set_error(KKT_ERR_INVALID_ARG, "null options");
  *opt = h->opt;
  return KKT_OK;
}

int kkt_get_info(const kkt_handle* h, kkt_info* info) {
  KKT_TRY(check_handle(h));
  if (!info) return set_error(KKT_ERR_INVALID_ARG, "null info");
  info->nx = h->g.nx;
  info->ny = h->g.ny;
  info->Nt = h->g.Nt;
  info->n_sub = h->g.n_sub;
  info->N = h->g.N;
  info->V = h->g.V;
  info->dx = h->g.dx;
  info->dy = h->g.dy;
  info->dt = h->g.dt;
  info->h = h->g.h;
  info->workspace_bytes = static_cast<long long>(h->bytes);
  return KKT_OK;
}

int kkt_build_rhs(kkt_handle* h, const double* u_target, const double* u0, double* f, void* stream) {
  KKT_TRY(check_handle(h));
  if (!u_target || !f) return set_error(KKT_ERR_INVALID_ARG, "null pointer");
  cudaStream_t st = as_stream(stream);
  const Geometry& g = h->g;
  const bool dev_t = is_device_ptr(u_target), dev_f = is_device_ptr(f);
  const bool dev_0 = u0 ? is_device_ptr(u0) : true;
  const double* dt_ = u_target;
  const double* d0 = u0;
  double* df = f;
  if (!dev_t) {
    KKT_CUDA_TRY(cudaMemcpyAsync(h->spec, u_target, g.V * sizeof(double), cudaMemcpyHostToDevice, st));
    dt_ = h->spec;
  }
  if (u0 && !dev_0) {
    KKT_CUDA_TRY(cudaMemcpyAsync(h->spec2, u0, g.N * sizeof(double), cudaMemcpyHostToDevice, st));
    d0 = h->spec2;
  }
  if (!dev_f) {
    KKT_TRY(dev_alloc(h, &h->kf, 3 * static_cast<size_t>(g.V)));
    df = h->kf;
  }
  KKT_TRY(launch_build_rhs(h, dt_, d0, df, st));
  if (!dev_f) {
    KKT_CUDA_TRY(cudaMemcpyAsync(f, df, 3 * g.V * sizeof(double), cudaMemcpyDeviceToHost, st));
  }
  if (!dev_t || !dev_f || !dev_0) KKT_CUDA_TRY(cudaStreamSynchronize(st));
  return KKT_OK;
}

int kkt_matvec(kkt_handle* h, const double* x, double* y, void* stream) {
  KKT_TRY(check_handle(h));
  KKT_TRY(check_ptrs({x, y}));
  const long long V = h->g.V;
  return launch_matvec(h, x, 1.0, x + V, 1.0, x + 2 * V, 1.0, y, as_stream(stream));
}

int kkt_precond_apply(kkt_handle* h, const double* r, double* y, void* stream) {
  KKT_TRY(check_handle(h));
  KKT_TRY(check_ptrs({r, y}));
  cudaStream_t st = as_stream(stream);
  const Geometry& g = h->g;
  KKT_TRY(launch_scale2(r, 1.0 / g.h, y, r + g.V, 1.0 / (g.omega * g.h), y + g.V, g.V, st));
  return schur_precond_w(h, r + 2 * g.V, 1.0, y + 2 * g.V, st);
}

int kkt_dst2d(kkt_handle* h, const double* in, double* out, void* stream) {
  KKT_TRY(check_handle(h));
  KKT_TRY(check_ptrs({in, out}));
  cudaStream_t st = as_stream(stream);
  if (h->opt.precision == KKT_PREC_FP64) return dst2d(h, in, out, st);
  // reduced precision: the tensor-core transforms (operands rounded to BF16 / TF32, FP32 sums)
  const TcPlan& t = h->tc;
  const int valid = h->g.nx - 1;
  const bool sp = h->opt.tc_split != 0;
  KKT_TRY(tc_pack(t, in, valid, st));
  KKT_TRY(tc_gemm(t, 0, sp ? 3 : (t.bf16 ? 0 : 1), t.x1, valid, st, sp, t.x1_lo));
  return tc_gemm(t, 1, 2, out, valid, st, sp);
}

int kkt_schur_apply(kkt_handle* h, const double* x, double* y, void* stream) {
  KKT_TRY(check_handle(h));
  KKT_TRY(check_ptrs({x, y}));
  cudaStream_t st = as_stream(stream);
  KKT_TRY(launch_jhat_time(h, x, h->spec, +1, 1.0, st));           // Jhat^T x
  return launch_jhat_time(h, h->spec, y, -1, 1.0 / h->g.h, st);    // Jhat (.) / h
}

int kkt_schur_precond_apply(kkt_handle* h, const double* r, double* y, void* stream) {
  KKT_TRY(check_handle(h));
  KKT_TRY(check_ptrs({r, y}));
  return schur_precond_w(h, r, 1.0, y, as_stream(stream));
}

int kkt_coarse_apply(kkt_handle* h, const double* r, double* x0, void* stream) {
  KKT_TRY(check_handle(h));
  KKT_TRY(check_ptrs({r, x0}));
  if (h->opt.coarse != KKT_COARSE_EXACT) return set_error(KKT_ERR_INVALID_ARG, "coarse apply needs the exact coarse level");
  cudaStream_t st = as_stream(stream);
  KKT_TRY(dst2d(h, r, h->spec, st));
  KKT_TRY(spectral_coarse_only(h, h->spec, h->spec2, st));
  return dst2d(h, h->spec2, x0, st);
}

int kkt_attach_mlp(kkt_handle* h, kkt_mlp* m, int mode) {
  KKT_TRY(check_handle(h));
  if (!m) return set_error(KKT_ERR_INVALID_ARG, "null network");
  if (mode < 0 || mode > 2)
    return set_error(KKT_ERR_INVALID_ARG, "mode must be 0 (learned, guarded), 1 (none) or 2 (network only)");
  int d_in = 0, width = 0, d_out = 0;
  KKT_TRY(mlp_dims(m, &d_in, &width, &d_out));
  const Geometry& g = h->g;
  if (d_out != 2 * g.n_sub) return set_error(KKT_ERR_INVALID_ARG, "network output width != 2 n_sub of this problem");
  const int K = kkt::mlp_config(m).modes;
  if (K < 1 || K > std::min(g.Mx, g.My)) return set_error(KKT_ERR_INVALID_ARG, "learned modes exceed the grid");
  const size_t nl = static_cast<size_t>(K) * K;
  KKT_TRY(dev_alloc(h, &h->learn_c, nl * d_out));
  KKT_TRY(dev_alloc(h, &h->learn_feat, nl * 2));
  KKT_TRY(dev_alloc(h, &h->learn_x, nl * d_in));
  KKT_TRY(dev_alloc(h, &h->learn_count, 2));
  KKT_CUDA_TRY(cudaMemset(h->learn_count, 0, 2 * sizeof(long long)));
  // features of the learned modes: log(dt nu lambda_kl), log(a - 1) = log(dt / sqrt(omega))
  const double pi = 3.14159265358979323846;
  std::vector<double> feat(nl * 2);
  for (int l = 0; l < K; ++l)
    for (int k = 0; k < K; ++k) {
      const double sx = std::sin((k + 1) * pi / (2.0 * g.nx)), sy = std::sin((l + 1) * pi / (2.0 * g.ny));
      const double lam = 4.0 / (g.dx * g.dx) * sx * sx + 4.0 / (g.dy * g.dy) * sy * sy;
      feat[2 * (l * K + k)] = std::log(g.dtnu * lam);
      feat[2 * (l * K + k) + 1] = std::log(g.dt / std::sqrt(g.omega));
    }
  KKT_CUDA_TRY(cudaMemcpy(h->learn_feat, feat.data(), feat.size() * sizeof(double), cudaMemcpyHostToDevice));
  h->mlp = m;
  h->mlp_mode = mode;
  h->learn_k = K;
  return KKT_OK;
}

int kkt_inject_tc_timeout(kkt_handle* h) {
  KKT_TRY(check_handle(h));
  if (h->opt.precision == KKT_PREC_FP64 || !h->tc.err)
    return set_error(KKT_ERR_INVALID_ARG, "the handle has no tensor-core transforms (FP64 precision)");
  return tc_set_flag(h->tc);
}

int kkt_learned_stats(kkt_handle* h, long long* kept, long long* fallback, int reset) {
  KKT_TRY(check_handle(h));
  long long c[2] = {0, 0};
  if (h->learn_count) {
    KKT_CUDA_TRY(cudaMemcpy(c, h->learn_count, sizeof(c), cudaMemcpyDeviceToHost));
    if (reset) KKT_CUDA_TRY(cudaMemset(h->learn_count, 0, sizeof(c)));
  }
  if (kept) *kept = c[0];
  if (fallback) *fallback = c[1];
  return KKT_OK;
}

int kkt_multidot(kkt_handle* h, const double* V, long long stride, int count, const double* w, long long n,
                 double* out, void* stream) {
  KKT_TRY(check_handle(h));
  KKT_TRY(check_ptrs({V, w, out}));
  if (count < 1 || count > 32) return set_error(KKT_ERR_INVALID_ARG, "count must be in [1, 32]");
  if (n < 1 || stride < n) return set_error(KKT_ERR_INVALID_ARG, "need n >= 1 and stride >= n");
  return krylov_multidot(h, V, stride, count, w, n, as_stream(stream), out);
}

static int solve_impl(kkt_handle* h, const double* f, double* x, double tol, int maxit, kkt_stats* stats,
                      void* stream, bool zero_guess);

int kkt_solve(kkt_handle* h, const double* f, double* x, double tol, int maxit, kkt_stats* stats, void* stream) {
  return solve_impl(h, f, x, tol, maxit, stats, stream, false);
}

int kkt_set_dst_method(kkt_handle* h, int method) {
  KKT_TRY(check_handle(h));
  if (method < KKT_DST_AUTO || method > KKT_DST_TENSOR) return set_error(KKT_ERR_INVALID_ARG, "dst method out of range");
  return dst_set_method(h, method);
}

int kkt_get_dst_method(const kkt_handle* h, int* method) {
  KKT_TRY(check_handle(h));
  if (!method) return set_error(KKT_ERR_INVALID_ARG, "null method");
  *method = h->dst_tensor ? KKT_DST_TENSOR
                          : ((h->dst_x.lane_direct || h->dst_y.lane_direct) ? KKT_DST_LANE : KKT_DST_TILES);
  return KKT_OK;
}

int kkt_set_staging(kkt_handle* h, int mode) {
  KKT_TRY(check_handle(h));
  if (mode != KKT_STAGING_AUTO && mode != KKT_STAGING_COPY_ENGINE)
    return set_error(KKT_ERR_INVALID_ARG, "staging mode out of range");
  h->staging = mode;
  return KKT_OK;
}

int kkt_solve_zero_guess(kkt_handle* h, const double* f, double* x, double tol, int maxit, kkt_stats* stats,
                         void* stream) {
  return solve_impl(h, f, x, tol, maxit, stats, stream, true);
}

static int solve_impl(kkt_handle* h, const double* f, double* x, double tol, int maxit, kkt_stats* stats,
                      void* stream, bool zero_guess) {
  KKT_TRY(check_handle(h));
  if (!f || !x) return set_error(KKT_ERR_INVALID_ARG, "null pointer");
  if (!(tol > 0.0) || !std::isfinite(tol)) return set_error(KKT_ERR_INVALID_ARG, "tol must be positive");
  if (maxit < 1) return set_error(KKT_ERR_INVALID_ARG, "maxit must be >= 1");
  const auto t0 = std::chrono::steady_clock::now();
  cudaStream_t st = as_stream(stream);
  const Geometry& g = h->g;
  const long long V = g.V, n3 = 3 * V;
  KKT_TRY(ensure_krylov(h));
  const bool spectral = h->opt.basis == KKT_BASIS_SPECTRAL;
  const bool dev_f = is_device_ptr(f), dev_x = is_device_ptr(x);
  const double* df = f;
  double* dx = x;
  if (!dev_f) {
    if (!h->kf) KKT_TRY(dev_alloc(h, &h->kf, n3));
    KKT_TRY(stage_copy(h, h->kf, f, n3, cudaMemcpyHostToDevice, st));
    df = h->kf;
  }
  if (!dev_x) {
    if (!h->kx) KKT_TRY(dev_alloc(h, &h->kx, n3));
    if (zero_guess)   // x is output only: nothing to upload
      KKT_CUDA_TRY(cudaMemsetAsync(h->kx, 0, n3 * sizeof(double), st));
    else
      KKT_TRY(stage_copy(h, h->kx, x, n3, cudaMemcpyHostToDevice, st));
    dx = h->kx;
  } else if (zero_guess) {
    KKT_CUDA_TRY(cudaMemsetAsync(x, 0, n3 * sizeof(double), st));
  }
  // physical-space f and x on the device; in the spectral basis the iteration runs on their
  // sine-mode coefficients (every block through the orthonormal 2D DST-I, which is its own
  // inverse), and x is transformed back once at exit
  const double* pf = df;
  double* px = dx;
  if (spectral) {
    if (!h->ks_f) KKT_TRY(dev_alloc(h, &h->ks_f, n3));
    if (!h->ks_x) KKT_TRY(dev_alloc(h, &h->ks_x, n3));
    for (int b = 0; b < 3; ++b) {
      KKT_TRY(dst2d(h, pf + b * V, h->ks_f + b * V, st));
      KKT_TRY(dst2d(h, px + b * V, h->ks_x + b * V, st));
    }
    df = h->ks_f;
    dx = h->ks_x;
  }
  auto matvec = [&](const double* u, double su, const double* z, double sz, const double* w, double sw, double* y,
                    double ou, double oz, double ow) -> int {
    return spectral ? launch_matvec_spectral(h, u, su, z, sz, w, sw, y, st, ou, oz, ow)
                    : launch_matvec(h, u, su, z, sz, w, sw, y, st, ou, oz, ow);
  };
  auto precond_w = [&](const double* rw, double scale, double* yw) -> int {
    return spectral ? spectral_schur_precond(h, rw, yw, scale, st) : schur_precond_w(h, rw, scale, yw, st);
  };
  const int m = h->opt.restart;
  double* Vb = h->kV;
  double* Zw = h->kZw;
  double* hr = h->h_red;            // [0,128): reductions
  double* hc = h->h_red + 128;      // coefficient staging, 4 x 128
  std::vector<double> H((m + 1) * m), cs(m), sn(m), gv(m + 1), eta(m + 1), yv(m);
  auto Hs = [&](int i, int j) -> double& { return H[static_cast<size_t>(i) * m + j]; };
  kkt_stats local;
  std::memset(&local, 0, sizeof(local));
  double fnorm_plain = 0.0;
  std::function<double()> euclid_residual;
  auto finish = [&](int status, double rel) -> int {
    if (spectral)
      for (int b = 0; b < 3; ++b)
        if (dst2d(h, dx + b * V, px + b * V, st) < 0 && status >= 0) status = KKT_ERR_CUDA;
    if (status >= 0 && std::isfinite(rel) && fnorm_plain > 0.0 && euclid_residual)
      local.rel_residual_euclid = euclid_residual();
    if (status >= 0 && h->opt.precision != KKT_PREC_FP64 && tc_check(h->tc, st) < 0) status = KKT_ERR_TIMEOUT;
    if (status >= 0 && h->dst_tensor && oz_check(h->oz, st) < 0) status = KKT_ERR_TIMEOUT;
    if (!dev_x) {
      if (stage_copy(h, x, px, n3, cudaMemcpyDeviceToHost, st) < 0 && status >= 0) status = KKT_ERR_CUDA;
      cudaStreamSynchronize(st);
    }
    local.status = status;
    local.rel_residual = rel;
    local.time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (stats) *stats = local;
    return status;
  };
  auto fetch = [&](int count) -> int {
    KKT_CUDA_TRY(cudaMemcpyAsync(hr, h->red_out, count * sizeof(double), cudaMemcpyDeviceToHost, st));
    KKT_CUDA_TRY(cudaStreamSynchronize(st));
    return KKT_OK;
  };
  // residual weights D = diag(du, dz, dw) of the options' norm
  const bool l2 = h->opt.residual_norm == KKT_NORM_L2;
  const double du = l2 ? 1.0 / std::sqrt(g.h) : 1.0, dz = du, dw = l2 ? std::sqrt(g.h) : 1.0;
  const double dblk[3] = {du, dz, dw};
  // squared block norms of a full vector -> weighted and unweighted totals
  auto block_norms = [&](const double* v, double& weighted, double& plain) -> int {
    double b[3];
    for (int k = 0; k < 3; ++k) {
      KKT_TRY(krylov_norm2(h, v + k * V, V, st));
      KKT_TRY(fetch(1));
      b[k] = hr[0];
    }
    weighted = du * du * b[0] + dz * dz * b[1] + dw * dw * b[2];
    plain = b[0] + b[1] + b[2];
    return KKT_OK;
  };
  double fw2 = 0.0, fp2 = 0.0;
  KKT_TRY(block_norms(df, fw2, fp2));
  const double fnorm = std::sqrt(fw2);
  fnorm_plain = std::sqrt(fp2);
  if (!std::isfinite(fnorm)) return finish(set_error(KKT_ERR_NONFINITE, "right-hand side is not finite"), NAN);
  if (fnorm == 0.0) {
    KKT_CUDA_TRY(cudaMemsetAsync(dx, 0, n3 * sizeof(double), st));
    return finish(KKT_OK, 0.0);
  }
  // V_0 = D (f - K x), beta = ||V_0||
  auto residual = [&](double& beta) -> int {
    KKT_TRY(matvec(dx, 1.0, dx + V, 1.0, dx + 2 * V, 1.0, Vb, du, dz, dw));
    for (int k = 0; k < 3; ++k) KKT_TRY(launch_axpby(dblk[k], df + k * V, -1.0, Vb + k * V, Vb + k * V, V, st));
    KKT_TRY(krylov_norm2(h, Vb, n3, st));
    KKT_TRY(fetch(1));
    beta = std::sqrt(hr[0]);
    return KKT_OK;
  };
  // unweighted relative residual of x (physical space), into the stats (uses V_1 as scratch)
  euclid_residual = [&]() -> double {
    double* R = Vb + n3;
    if (launch_matvec(h, px, 1.0, px + V, 1.0, px + 2 * V, 1.0, R, st) < 0) return NAN;
    if (launch_axpby(1.0, pf, -1.0, R, R, n3, st) < 0) return NAN;
    if (krylov_norm2(h, R, n3, st) < 0 || fetch(1) < 0) return NAN;
    return std::sqrt(hr[0]) / fnorm_plain;
  };
  double beta = 0.0;
  KKT_TRY(residual(beta));
  if (!std::isfinite(beta)) return finish(set_error(KKT_ERR_NONFINITE, "initial residual is not finite"), NAN);
  if (beta / fnorm <= tol) return finish(KKT_OK, beta / fnorm);
  int its = 0;
  while (true) {
    std::fill(H.begin(), H.end(), 0.0);
    std::fill(gv.begin(), gv.end(), 0.0);
    gv[0] = beta;
    eta[0] = beta;   // V_0 holds r = beta v_0
    int jused = 0;
    bool stop = false;
    for (int j = 0; j < m; ++j) {
      double* Vj = Vb + static_cast<size_t>(j) * n3;
      double* W = Vb + static_cast<size_t>(j + 1) * n3;
      double* Zj = Zw + static_cast<size_t>(j) * V;
      // z_j = P^{-1} D^{-1} v_j: the u, z blocks are scalings (folded into the matvec), the
      // w block goes through S-hat_2level^{-1}; then W = D K z_j
      KKT_TRY(precond_w(Vj + 2 * V, 1.0 / (dw * eta[j]), Zj));
      local.precond_applies++;
      KKT_TRY(matvec(Vj, 1.0 / (g.h * du * eta[j]), Vj + V, 1.0 / (g.omega * g.h * dz * eta[j]), Zj, 1.0, W, du, dz,
                     dw));
      for (int k = 0; k <= j; ++k) Hs(k, j) = 0.0;
      double wnorm2 = 0.0;
      const int bs = orth_block(h->opt.orth);
      if (bs > 1) {
        // MGS over blocks of bs basis vectors: every dot of a block is taken on the same w (the
        // vectors of a block are orthogonal to working accuracy), and the block is subtracted
        // in one pass that also takes the next block's dots: 2 + 2 / bs vector passes per
        // basis vector
        const double* V0 = Vb;
        double sc[8];
        KKT_TRY(krylov_mgsb_step(h, bs, 0, nullptr, nullptr, nullptr, std::min(bs, j + 1), V0, n3, W, n3, h->red_out,
                                 st));
        for (int k = 0; k <= j;) {
          const int na = std::min(bs, j + 1 - k);
          const int nd = std::min(bs, j + 1 - (k + na));
          for (int a = 0; a < na; ++a) sc[a] = 1.0 / (eta[k + a] * eta[k + a]);
          KKT_TRY(krylov_mgsb_step(h, bs, na, V0 + static_cast<size_t>(k) * n3, h->red_out + k, sc, nd,
                                   V0 + static_cast<size_t>(k + na) * n3, n3, W, n3, h->red_out + k + na, st));
          k += na;
        }
        KKT_TRY(fetch(j + 2));
        for (int k = 0; k <= j; ++k) Hs(k, j) = hr[k] / eta[k];
        wnorm2 = hr[j + 1];
        if (!std::isfinite(wnorm2)) return finish(set_error(KKT_ERR_NONFINITE, "Krylov vector is not finite"), NAN);
      }
      if (h->opt.orth == KKT_ORTH_MGS) {
        // modified Gram-Schmidt: d_k = <V_k, w> on the w already orthogonalised against
        // V_0..V_k-1, then w -= (d_k / eta_k^2) V_k; the dots stay on the device (red_out[k])
        // and feed the next step's coefficient, so the host reads the column once
        KKT_TRY(krylov_mgs_step(h, nullptr, nullptr, 0.0, Vb, W, n3, h->red_out, st));
        for (int k = 0; k <= j; ++k) {
          const double* Vn = k < j ? Vb + static_cast<size_t>(k + 1) * n3 : nullptr;
          KKT_TRY(krylov_mgs_step(h, Vb + static_cast<size_t>(k) * n3, h->red_out + k, 1.0 / (eta[k] * eta[k]), Vn, W,
                                  n3, h->red_out + k + 1, st));
        }
        KKT_TRY(fetch(j + 2));
        for (int k = 0; k <= j; ++k) Hs(k, j) = hr[k] / eta[k];
        wnorm2 = hr[j + 1];
        if (!std::isfinite(wnorm2)) return finish(set_error(KKT_ERR_NONFINITE, "Krylov vector is not finite"), NAN);
      }
      // classical Gram-Schmidt with one conditional reorthogonalisation (||w'|| < ||w|| / sqrt 2)
      for (int pass = 0; pass < 2 && h->opt.orth == KKT_ORTH_CGS2; ++pass) {
        KKT_TRY(krylov_multidot(h, Vb, n3, j + 1, W, n3, st));
        KKT_TRY(fetch(j + 2));
        const double before = hr[j + 1];
        for (int k = 0; k <= j; ++k) {
          const double hk = hr[k] / eta[k];
          Hs(k, j) += hk;
          hc[k] = hk / eta[k];
        }
        KKT_CUDA_TRY(cudaMemcpyAsync(h->dcoef, hc, (j + 1) * sizeof(double), cudaMemcpyHostToDevice, st));
        KKT_TRY(krylov_update_norm(h, Vb, n3, j + 1, h->dcoef, W, n3, st));
        KKT_TRY(fetch(1));
        wnorm2 = hr[0];
        if (!std::isfinite(wnorm2)) return finish(set_error(KKT_ERR_NONFINITE, "Krylov vector is not finite"), NAN);
        if (wnorm2 >= 0.5 * before) break;
      }
      const double hn = std::sqrt(wnorm2);
      Hs(j + 1, j) = hn;
      eta[j + 1] = hn;
      for (int i = 0; i < j; ++i) {
        const double t = cs[i] * Hs(i, j) + sn[i] * Hs(i + 1, j);
        Hs(i + 1, j) = -sn[i] * Hs(i, j) + cs[i] * Hs(i + 1, j);
        Hs(i, j) = t;
      }
      const double d = std::hypot(Hs(j, j), Hs(j + 1, j));
      cs[j] = d > 0 ? Hs(j, j) / d : 1.0;
      sn[j] = d > 0 ? Hs(j + 1, j) / d : 0.0;
      Hs(j, j) = d;
      Hs(j + 1, j) = 0.0;
      gv[j + 1] = -sn[j] * gv[j];
      gv[j] = cs[j] * gv[j];
      ++its;
      jused = j + 1;
      const double est = std::fabs(gv[j + 1]) / fnorm;
      if (local.history_len < KKT_HISTORY_MAX) local.history[local.history_len++] = est;
      if (est <= tol || its >= maxit || hn == 0.0) {
        stop = true;
        break;
      }
    }
    // y = H^{-1} g (upper triangular), x += Z y
    for (int i = jused - 1; i >= 0; --i) {
      double s = gv[i];
      for (int k = i + 1; k < jused; ++k) s -= Hs(i, k) * yv[k];
      yv[i] = Hs(i, i) != 0.0 ? s / Hs(i, i) : 0.0;
    }
    for (int k = 0; k < jused; ++k) {
      hc[k] = yv[k] / (g.h * du * eta[k]);
      hc[128 + k] = yv[k] / (g.omega * g.h * dz * eta[k]);
      hc[256 + k] = yv[k];
    }
    KKT_CUDA_TRY(cudaMemcpyAsync(h->dcoef, hc, 3 * 128 * sizeof(double), cudaMemcpyHostToDevice, st));
    KKT_TRY(krylov_axpy_multi(Vb, n3, jused, h->dcoef, dx, V, st));
    KKT_TRY(krylov_axpy_multi(Vb + V, n3, jused, h->dcoef + 128, dx + V, V, st));
    KKT_TRY(krylov_axpy_multi(Zw, V, jused, h->dcoef + 256, dx + 2 * V, V, st));
    local.restarts++;
    KKT_TRY(residual(beta));
    const double rel = beta / fnorm;
    local.iterations = its;
    if (!std::isfinite(rel)) return finish(set_error(KKT_ERR_NONFINITE, "iterate is not finite"), rel);
    if (rel <= tol) return finish(KKT_OK, rel);
    if (its >= maxit) return finish(KKT_NOT_CONVERGED, rel);
    if (stop && eta[jused] == 0.0) return finish(set_error(KKT_ERR_BREAKDOWN, "Arnoldi breakdown before convergence"), rel);
  }
}

}  // extern "C"
