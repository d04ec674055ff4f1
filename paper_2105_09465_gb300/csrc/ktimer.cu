// Launch timer: CUDA events recorded on the launching stream around the
// pair-sweep kernels, so a caller can read each kernel's own device time
// (without the pre-pass and merge launches of the same entry point).
// Off by default; while off, ktimer_begin/ktimer_end cost one load each.
#include <atomic>
#include <mutex>
#include <vector>
#include "common.cuh"

namespace lr {
namespace {

constexpr int kMaxRecords = 8192;

struct Record {
  int id;
  bool closed;  // the end event was recorded (a failed launch leaves it open)
  cudaEvent_t a, b;
};

std::mutex g_mu;
std::atomic<bool> g_on{false};
int g_dev = -1;
std::vector<Record> g_rec;         // recorded this session, in launch order
std::vector<cudaEvent_t> g_pool;   // events created on g_dev, reused
size_t g_pool_next = 0;
int64_t g_dropped = 0;
// The record opened by this thread's last ktimer_begin (begin and end of one
// launch are issued back to back by the same host thread).
thread_local int t_open = -1;

cudaEvent_t take_event() {
  if (g_pool_next < g_pool.size()) return g_pool[g_pool_next++];
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  g_pool.push_back(e);
  ++g_pool_next;
  return e;
}

bool capturing(cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return true;
  return cs != cudaStreamCaptureStatusNone;
}

}  // namespace

void ktimer_begin(int id, cudaStream_t s) {
  t_open = -1;
  if (!g_on.load(std::memory_order_relaxed)) return;
  std::lock_guard<std::mutex> lk(g_mu);
  int dev = -1;
  if (!g_on || cudaGetDevice(&dev) != cudaSuccess || dev != g_dev || capturing(s)) return;
  if ((int)g_rec.size() >= kMaxRecords) {
    ++g_dropped;
    return;
  }
  cudaEvent_t a = take_event(), b = take_event();
  if (!a || !b || cudaEventRecord(a, s) != cudaSuccess) {
    ++g_dropped;
    return;
  }
  g_rec.push_back(Record{id, false, a, b});
  t_open = (int)g_rec.size() - 1;
}

void ktimer_end(int id, cudaStream_t s) {
  if (t_open < 0) return;
  std::lock_guard<std::mutex> lk(g_mu);
  if (t_open < 0 || t_open >= (int)g_rec.size() || g_rec[t_open].id != id) return;
  if (cudaEventRecord(g_rec[t_open].b, s) == cudaSuccess)
    g_rec[t_open].closed = true;
  else
    ++g_dropped;
  t_open = -1;
}

}  // namespace lr

extern "C" lr_status lr_kernel_timer_enable(int32_t enable) {
  using namespace lr;
  std::lock_guard<std::mutex> lk(g_mu);
  if (enable) {
    int dev = 0;
    LR_CHECK_CUDA(cudaGetDevice(&dev));
    if (dev != g_dev) {
      // events belong to the device they were created on
      for (cudaEvent_t e : g_pool) cudaEventDestroy(e);
      g_pool.clear();
      g_dev = dev;
    }
    g_rec.clear();
    g_pool_next = 0;
    g_dropped = 0;
  }
  g_on.store(enable != 0);
  return LR_OK;
}

extern "C" lr_status lr_kernel_timer_read(int32_t kernel, int64_t* launches, double* total_ms, int64_t* dropped) {
  using namespace lr;
  LR_REQUIRE(kernel >= 0 && kernel < LR_KT_COUNT, "lr_kernel_timer_read: unknown kernel id %d", kernel);
  LR_REQUIRE(launches && total_ms, "lr_kernel_timer_read: NULL output");
  std::lock_guard<std::mutex> lk(g_mu);
  int64_t cnt = 0;
  double tot = 0.0;
  for (const Record& r : g_rec) {
    if (r.id != kernel || !r.closed) continue;
    LR_CHECK_CUDA(cudaEventSynchronize(r.b));
    float ms = 0.f;
    LR_CHECK_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
    ++cnt;
    tot += ms;
  }
  *launches = cnt;
  *total_ms = tot;
  if (dropped) *dropped = g_dropped;
  return LR_OK;
}

// ---------------------------------------------------------------------------
// Fork and join of a second stream for independent branches of one entry
// point (see common.cuh). The side stream is per device and non-blocking;
// the events are per call, so concurrent callers never share one.
namespace lr {

cudaStream_t side_stream() {
  static std::mutex mu;
  static cudaStream_t streams[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(mu);
  if (!streams[dev] && cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking) != cudaSuccess)
    streams[dev] = nullptr;
  return streams[dev];
}

lr_status fork_begin(cudaStream_t s, Fork* f) {
  f->side = s;
  f->join = nullptr;
  cudaStream_t side = side_stream();
  if (!side) return LR_OK;  // no second stream: the branch runs on s
  cudaEvent_t e = nullptr;
  LR_CHECK_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  cudaError_t r = cudaEventRecord(e, s);
  if (r == cudaSuccess) r = cudaStreamWaitEvent(side, e, 0);
  cudaEventDestroy(e);
  if (r != cudaSuccess) return cuda_status(r, "fork_begin");
  LR_CHECK_CUDA(cudaEventCreateWithFlags(&f->join, cudaEventDisableTiming));
  f->side = side;
  return LR_OK;
}

lr_status fork_end(cudaStream_t s, Fork* f) {
  if (!f->join) return LR_OK;
  cudaError_t r = cudaEventRecord(f->join, f->side);
  if (r == cudaSuccess) r = cudaStreamWaitEvent(s, f->join, 0);
  cudaEventDestroy(f->join);
  f->join = nullptr;
  f->side = s;
  return r == cudaSuccess ? LR_OK : cuda_status(r, "fork_end");
}

}  // namespace lr
