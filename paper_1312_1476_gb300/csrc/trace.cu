// trace.cu -- see trace.h.
#include <cuda_runtime.h>

#include <mutex>
#include <vector>

#include "../../include/gmrf.h"
#include "trace.h"

namespace gmrf {
namespace {

struct Pending {
  int kc;
  cudaEvent_t a, b;
};

struct Registry {
  bool timing = false;
  int64_t launches[KC_COUNT] = {};
  int64_t timed[KC_COUNT] = {};
  double ms[KC_COUNT] = {};
  std::vector<cudaEvent_t> pool;
  std::vector<Pending> pending;
};

Registry& reg() {
  static Registry r;
  return r;
}

// Per host thread: the graph being captured by this thread (captures are
// thread-local), and the class of the launch between trace_begin/trace_end.
thread_local GraphTrace* g_sink = nullptr;
thread_local int g_open_kc = -1;
thread_local Pending t_open = {-1, nullptr, nullptr};
std::mutex g_mu;  // guards the registry

cudaEvent_t take() {
  Registry& r = reg();
  if (!r.pool.empty()) {
    cudaEvent_t e = r.pool.back();
    r.pool.pop_back();
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

void trace_begin(int kc, cudaStream_t s, int nkernels) {
  Registry& r = reg();
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_sink) {
    g_sink->launches[kc] += nkernels;
    g_open_kc = -1;
    if (g_sink->timed && g_sink->npairs < 4096) {
      const int i = g_sink->npairs;
      g_sink->a[i] = g_sink->b[i] = nullptr;
      if (cudaEventCreate(&g_sink->a[i]) == cudaSuccess && cudaEventCreate(&g_sink->b[i]) == cudaSuccess &&
          cudaEventRecordWithFlags(g_sink->a[i], s, cudaEventRecordExternal) == cudaSuccess) {
        g_sink->kc[i] = kc;
        g_open_kc = kc;
      } else {
        cudaGetLastError();
        if (g_sink->a[i]) cudaEventDestroy(g_sink->a[i]);
        if (g_sink->b[i]) cudaEventDestroy(g_sink->b[i]);
      }
    }
    return;
  }
  r.launches[kc] += nkernels;
  if (!r.timing) return;
  t_open.kc = kc;
  t_open.a = take();
  t_open.b = take();
  if (t_open.a) cudaEventRecord(t_open.a, s);
}

void trace_end(int kc, cudaStream_t s) {
  Registry& r = reg();
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_sink) {
    if (g_open_kc == kc) {
      const int i = g_sink->npairs;
      if (cudaEventRecordWithFlags(g_sink->b[i], s, cudaEventRecordExternal) == cudaSuccess) g_sink->npairs++;
      else cudaGetLastError();
    }
    g_open_kc = -1;
    return;
  }
  if (!r.timing || t_open.kc != kc) return;
  if (t_open.a && t_open.b) {
    cudaEventRecord(t_open.b, s);
    r.pending.push_back(t_open);
  }
  t_open.kc = -1;
}

void trace_collect() {
  Registry& r = reg();
  std::lock_guard<std::mutex> lock(g_mu);
  for (Pending& p : r.pending) {
    if (cudaEventSynchronize(p.b) == cudaSuccess) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) {
        r.ms[p.kc] += t;
        r.timed[p.kc] += 1;
      }
    }
    cudaGetLastError();
    r.pool.push_back(p.a);
    r.pool.push_back(p.b);
  }
  r.pending.clear();
}

bool trace_timing_enabled() {
  std::lock_guard<std::mutex> lock(g_mu);
  return reg().timing;
}

void GraphTrace::release() {
  for (int i = 0; i < npairs; ++i) {
    cudaEventDestroy(a[i]);
    cudaEventDestroy(b[i]);
  }
  npairs = 0;
  for (int k = 0; k < KC_COUNT; ++k) launches[k] = 0;
}

void trace_capture_begin(GraphTrace* g) {
  g->release();
  std::lock_guard<std::mutex> lock(g_mu);
  g->timed = reg().timing;
  g_sink = g;
  g_open_kc = -1;
}

void trace_capture_end() {
  g_sink = nullptr;
  g_open_kc = -1;
}

void trace_replayed(const GraphTrace* g, int useful_pairs) {
  Registry& r = reg();
  std::lock_guard<std::mutex> lock(g_mu);
  for (int k = 0; k < KC_COUNT; ++k) r.launches[k] += g->launches[k];
  if (!r.timing || !g->timed) return;
  const int np = useful_pairs < g->npairs ? useful_pairs : g->npairs;
  for (int i = 0; i < np; ++i) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, g->a[i], g->b[i]) == cudaSuccess) {
      r.ms[g->kc[i]] += t;
      r.timed[g->kc[i]] += 1;
    } else {
      cudaGetLastError();
    }
  }
}

}  // namespace gmrf

extern "C" int gmrf_trace(int32_t op, int32_t kclass, double* total_ms, int64_t* launches, int64_t* timed) {
  using namespace gmrf;
  Registry& r = reg();
  switch (op) {
    case 0: {
      trace_collect();
      std::lock_guard<std::mutex> lock(g_mu);
      for (int k = 0; k < KC_COUNT; ++k) {
        r.launches[k] = 0;
        r.timed[k] = 0;
        r.ms[k] = 0.0;
      }
      return GMRF_OK;
    }
    case 1: {
      std::lock_guard<std::mutex> lock(g_mu);
      r.timing = true;
      return GMRF_OK;
    }
    case 2: {
      trace_collect();
      std::lock_guard<std::mutex> lock(g_mu);
      r.timing = false;
      return GMRF_OK;
    }
    case 3: {
      if (kclass < -1 || kclass >= KC_COUNT) return GMRF_ERR_INVALID;
      trace_collect();
      std::lock_guard<std::mutex> lock(g_mu);
      double ms = 0.0;
      int64_t l = 0, t = 0;
      for (int k = 0; k < KC_COUNT; ++k) {
        if (kclass != -1 && k != kclass) continue;
        ms += r.ms[k];
        l += r.launches[k];
        t += r.timed[k];
      }
      if (total_ms) *total_ms = ms;
      if (launches) *launches = l;
      if (timed) *timed = t;
      return GMRF_OK;
    }
    default:
      return GMRF_ERR_INVALID;
  }
}
