// Process-wide launch counters and optional CUDA-event timing of every kernel launch,
// exported as kkt_profile_enable / kkt_profile_read. Every launch scope is also an NVTX range
// named after its kernel class (header-only NVTX v3: a no-op unless a tool is attached), so an
// ncu or nsys capture can be filtered by phase.
#include <nvtx3/nvToolsExt.h>

#include <mutex>
#include <vector>

#include "kkt_internal.cuh"

namespace kkt {
namespace {

struct Pending {
  cudaEvent_t a, b;
  int cls;
  double flops, bytes;
};

std::mutex g_mu;
bool g_on = false;
long long g_launches[KKT_K_COUNT] = {};
double g_ms[KKT_K_COUNT] = {};
long long g_timed[KKT_K_COUNT] = {};
double g_flops[KKT_K_COUNT] = {};
double g_bytes[KKT_K_COUNT] = {};
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_pool;
thread_local cudaEvent_t t_open = nullptr;
thread_local ProfCapture* t_cap = nullptr;

cudaEvent_t take_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void drain_locked() {
  for (const Pending& p : g_pending) {
    float ms = 0.f;
    cudaEventSynchronize(p.b);
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      g_ms[p.cls] += ms;
      g_timed[p.cls] += 1;
      g_flops[p.cls] += p.flops;
      g_bytes[p.cls] += p.bytes;
    }
    g_pool.push_back(p.a);
    g_pool.push_back(p.b);
  }
  g_pending.clear();
}

const char* const kClassNames[KKT_K_COUNT] = {"kkt.dst",    "kkt.coarse", "kkt.sweep",  "kkt.matvec", "kkt.multidot",
                                               "kkt.update", "kkt.axpy",   "kkt.reduce", "kkt.graph",
                                               "kkt.pack"};

}  // namespace

void prof_begin(int cls, cudaStream_t st) {
  nvtxRangePushA(kClassNames[cls]);
  if (t_cap) {   // being captured into a graph: count the launch for every replay instead
    t_cap->launches[cls] += 1;
    return;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  g_launches[cls] += 1;
  if (!g_on) return;
  t_open = take_event();
  cudaEventRecord(t_open, st);
}

void prof_end(int cls, cudaStream_t st, double flops, double bytes) {
  nvtxRangePop();
  if (t_cap) {
    t_cap->flops += flops;
    t_cap->bytes += bytes;
    return;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_on || !t_open) return;
  cudaEvent_t b = take_event();
  cudaEventRecord(b, st);
  g_pending.push_back({t_open, b, cls, flops, bytes});
  t_open = nullptr;
  if (g_pending.size() > 4096) drain_locked();
}

void prof_capture(ProfCapture* acc) { t_cap = acc; }

int prof_graph_launch(cudaGraphExec_t g, const ProfCapture& acc, cudaStream_t st) {
  {
    std::lock_guard<std::mutex> lk(g_mu);
    for (int c = 0; c < KKT_K_COUNT; ++c) g_launches[c] += acc.launches[c];
  }
  ProfScope ps(KKT_K_GRAPH, st, acc.flops, acc.bytes);
  KKT_CUDA_TRY(cudaGraphLaunch(g, st));
  return KKT_OK;
}

}  // namespace kkt

extern "C" {

int kkt_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(kkt::g_mu);
  kkt::g_on = on != 0;
  return KKT_OK;
}

int kkt_profile_read(kkt_kernel_stats* out, int reset) {
  if (!out) return kkt::set_error(KKT_ERR_INVALID_ARG, "null stats");
  std::lock_guard<std::mutex> lk(kkt::g_mu);
  kkt::drain_locked();
  for (int c = 0; c < KKT_K_COUNT; ++c) {
    out->launches[c] = kkt::g_launches[c];
    out->ms[c] = kkt::g_ms[c];
    out->timed[c] = kkt::g_timed[c];
    out->flops[c] = kkt::g_flops[c];
    out->bytes[c] = kkt::g_bytes[c];
    if (reset) {
      kkt::g_launches[c] = 0;
      kkt::g_ms[c] = 0.0;
      kkt::g_timed[c] = 0;
      kkt::g_flops[c] = 0.0;
      kkt::g_bytes[c] = 0.0;
    }
  }
  return KKT_OK;
}

}  // extern "C"
