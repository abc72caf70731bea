// prof.cu -- launch accounting, optional per-kernel CUDA-event timing and the
// NVTX ranges of the entry points.
//
// Every kernel launch of the library goes through a LaunchScope, which counts
// it and, while profiling is on, records a CUDA event before and after it on
// the launching stream.  sz3g_profile_read() sums the elapsed times per kernel.
#include <atomic>
#include <cstring>
#include <mutex>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "internal.cuh"

namespace sz3g {

TraceRange::TraceRange(const char* name) { nvtxRangePushA(name); }
TraceRange::~TraceRange() { nvtxRangePop(); }

static const char* kKernelNames[kKernelCount] = {
    "range", "eb", "anchor", "lift", "pass_quantize", "pass_recover", "codebook", "encode", "finalize",
    "decode_tables", "decode", "scan", "zero_count", "pack_table", "level_quantize", "level_recover",
    "coarse_quantize", "coarse_recover", "decimate", "publish", "select", "mlp", "lossless", "report", "bitplane", "fixed_table",
};

namespace {
struct Rec {
  int kid;
  cudaEvent_t a, b;
};
std::mutex g_mu;
bool g_on = false;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;
std::atomic<unsigned long long> g_launches{0};

cudaEvent_t take_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}
}  // namespace

bool profiling_on() {
  std::lock_guard<std::mutex> lk(g_mu);
  return g_on;
}

void count_launches(unsigned long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

unsigned long long launch_total() { return g_launches.load(); }

LaunchScope::LaunchScope(int kid, cudaStream_t s) : kid_(kid), s_(s), a_(nullptr) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_on) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return;  // launches captured into a graph are not timed one by one
  }
  a_ = take_event();
  if (a_) cudaEventRecord((cudaEvent_t)a_, s);
}

LaunchScope::~LaunchScope() {
  if (!a_) return;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEvent_t b = take_event();
  if (!b) return;
  cudaEventRecord(b, s_);
  g_recs.push_back(Rec{kid_, (cudaEvent_t)a_, b});
}

}  // namespace sz3g

using namespace sz3g;

extern "C" {

int sz3g_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (Rec& r : g_recs) {
    g_pool.push_back(r.a);
    g_pool.push_back(r.b);
  }
  g_recs.clear();
  g_on = on != 0;
  return SZ3G_OK;
}

int sz3g_profile_read(const char* kernel, double* total_ms, uint64_t* launches) {
  if (!kernel || !total_ms || !launches) return SZ3G_E_INVAL;
  int kid = -1;
  for (int k = 0; k < kKernelCount; ++k)
    if (std::strcmp(kernel, kKernelNames[k]) == 0) kid = k;
  if (kid < 0) return SZ3G_E_INVAL;
  std::lock_guard<std::mutex> lk(g_mu);
  double t = 0;
  uint64_t n = 0;
  for (Rec& r : g_recs) {
    if (r.kid != kid) continue;
    if (cudaEventSynchronize(r.b) != cudaSuccess) {
      cudaGetLastError();
      return SZ3G_E_CUDA;
    }
    float ms = 0;
    if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) {
      cudaGetLastError();
      return SZ3G_E_CUDA;
    }
    t += ms;
    ++n;
  }
  *total_ms = t;
  *launches = n;
  return SZ3G_OK;
}

const char* sz3g_profile_kernel_name(int index) {
  return (index >= 0 && index < kKernelCount) ? kKernelNames[index] : nullptr;
}

int sz3g_launch_count(uint64_t* launches) {
  if (!launches) return SZ3G_E_INVAL;
  *launches = g_launches.load();
  return SZ3G_OK;
}

}  // extern "C"
