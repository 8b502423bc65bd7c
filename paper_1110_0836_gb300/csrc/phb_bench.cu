// FMA throughput probe used by the benchmark for the ALU roofline (see
// include/phurbas_bench.h).  16 independent accumulators per thread keep the
// FMA pipes busy; the constants keep values bounded.
#include <atomic>
#include <vector>

#include "phb_internal.cuh"
#include "../../include/phurbas_bench.h"

namespace phb {
namespace {
std::atomic<int64_t> g_launches{0};
struct Trace {
  bool armed = false;
  std::vector<cudaEvent_t> b, e;
  std::vector<int> id;
  int used = 0;
} g_trace;
}  // namespace

void note_launch(int count) { g_launches.fetch_add(count, std::memory_order_relaxed); }

int trace_begin(int kernel_id, cudaStream_t st) {
  if (!g_trace.armed || g_trace.used >= static_cast<int>(g_trace.b.size())) return -1;
  const int k = g_trace.used++;
  g_trace.id[k] = kernel_id;
  cudaEventRecord(g_trace.b[k], st);
  return k;
}

void trace_end(int slot, cudaStream_t st) {
  if (slot >= 0) cudaEventRecord(g_trace.e[slot], st);
}

}  // namespace phb

extern "C" int64_t phb_launch_count(void) { return phb::g_launches.load(); }

extern "C" int phb_trace_start(int32_t capacity) {
  using phb::g_trace;
  if (capacity <= 0 || g_trace.armed) return 1;
  g_trace.b.assign(capacity, nullptr);
  g_trace.e.assign(capacity, nullptr);
  g_trace.id.assign(capacity, 0);
  g_trace.used = 0;
  for (int k = 0; k < capacity; ++k)
    if (cudaEventCreate(&g_trace.b[k]) != cudaSuccess || cudaEventCreate(&g_trace.e[k]) != cudaSuccess)
      return 3;
  g_trace.armed = true;
  return 0;
}

extern "C" int phb_trace_read(float* ms, int32_t* kernel_ids, int32_t capacity) {
  using phb::g_trace;
  if (!g_trace.armed) return -1;
  const int n = g_trace.used;
  // a failed event query leaves a non-sticky error behind: consume it so that
  // the next launch check does not report it
  if (n > 0 && cudaEventSynchronize(g_trace.e[n - 1]) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  for (int k = 0; k < n && k < capacity; ++k) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, g_trace.b[k], g_trace.e[k]) != cudaSuccess) {
      cudaGetLastError();
      return -1;
    }
    if (ms) ms[k] = t;
    if (kernel_ids) kernel_ids[k] = g_trace.id[k];
  }
  return n < capacity ? n : capacity;
}

extern "C" int phb_trace_stop(float* ms, int32_t* kernel_ids, int32_t capacity) {
  using phb::g_trace;
  if (!g_trace.armed) return -1;
  g_trace.armed = false;
  int n = g_trace.used;
  int rc = n;
  if (n > 0 && cudaEventSynchronize(g_trace.e[n - 1]) != cudaSuccess) rc = -1;
  for (int k = 0; k < n && rc >= 0; ++k) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, g_trace.b[k], g_trace.e[k]) != cudaSuccess) { rc = -1; break; }
    if (k < capacity) {
      if (ms) ms[k] = t;
      if (kernel_ids) kernel_ids[k] = g_trace.id[k];
    }
  }
  for (size_t k = 0; k < g_trace.b.size(); ++k) {
    if (g_trace.b[k]) cudaEventDestroy(g_trace.b[k]);
    if (g_trace.e[k]) cudaEventDestroy(g_trace.e[k]);
  }
  g_trace.b.clear();
  g_trace.e.clear();
  g_trace.used = 0;
  if (rc < 0) cudaGetLastError();
  return rc < 0 ? -1 : (n < capacity ? n : capacity);
}

namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_fma(int iters, T* sink) {
  T a[16];
  const T x = T(0.999999), y = T(1e-7);
#pragma unroll
  for (int k = 0; k < 16; ++k) a[k] = T(threadIdx.x + k) * T(1e-3);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 16; ++k) a[k] = fma(a[k], x, y);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < 16; ++k) s += a[k];
  sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int phb_fma_peak(int32_t precision, int32_t blocks, int32_t iters, void* sink,
                            phb_stream_t stream) {
  if (blocks <= 0 || iters <= 0 || !sink || (precision != 0 && precision != 1)) return 1;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (precision == 1)
    k_fma<float><<<blocks, 256, 0, st>>>(iters, static_cast<float*>(sink));
  else
    k_fma<double><<<blocks, 256, 0, st>>>(iters, static_cast<double*>(sink));
  phb::note_launch();
  return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

extern "C" int phb_record_region(const phb_plan* plan, size_t* offset, size_t* bytes) {
  if (!plan || !offset || !bytes || plan->ws_bytes == 0 || plan->n <= 0) return 1;
  *offset = plan->ws_off[phb::R_REC];
  *bytes = static_cast<size_t>(plan->n) * 24 * sizeof(float);
  return 0;
}

extern "C" int phb_workspace_stats(const phb_plan* plan, const void* ws, int32_t* out, int32_t count,
                                   phb_stream_t stream) {
  if (!plan || !ws || !out || count < 0 || count > 5 || plan->ws_bytes == 0) return 1;
  int32_t tmp[6] = {0, 0, 0, 0, 0, 0};
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int32_t* misc = phb::region<int32_t>(plan, ws, phb::R_MISC);
  if (cudaMemcpyAsync(tmp, misc, sizeof(tmp), cudaMemcpyDeviceToHost, st) != cudaSuccess) return 3;
  if (cudaStreamSynchronize(st) != cudaSuccess) return 3;
  const int32_t v[5] = {tmp[0], tmp[1], tmp[2], plan->ntiles, tmp[5]};
  for (int k = 0; k < count; ++k) out[k] = v[k];
  return 0;
}
