// trace.h -- kernel launch counting and per-kernel-class CUDA-event timing.
//
// Every kernel launch of the library goes through trace_begin / trace_end.
// Launch counts are always kept.  When event timing is enabled
// (gmrf_trace(1, ...)), a pair of events is recorded around the launch on
// its own stream and the elapsed times are accumulated at the next host
// synchronisation point (trace_collect).  Thread-safe: the registry is
// guarded by a mutex and a graph capture only sees launches of the thread
// that captures.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gmrf {

enum KernelClass {
  KC_STENCIL_STEP = 0,  // fused stencil + Lanczos step
  KC_PRE_ROW_FWD = 1,   // preconditioned step: form v_j + row forward transform
  KC_PRE_COL = 2,       // column transform * symbol * inverse
  KC_PRE_ROW_MID = 3,   // inverse rows, R, forward rows
  KC_PRE_ROW_LAST = 4,  // inverse rows, A v, recurrence, reductions
  KC_INIT = 5,          // ||z||
  KC_RNG = 6,           // Philox streams
  KC_TM = 7,            // T_m functions (nodes, poles, sums, log)
  KC_ASSEMBLE = 8,      // x = ||z|| V_m y
  KC_PRE_APPLY = 9,     // plain M^{-1/2} / A applies, final M^{-1/2} u
  KC_OTHER = 10,        // scale, convert, field statistics, log det M
  KC_SPARSE_STEP = 11,  // Lanczos step with a CSR Q (and incomplete-Cholesky solves)
  KC_COUNT = 12
};

void trace_begin(int kc, cudaStream_t s, int nkernels = 1);
void trace_end(int kc, cudaStream_t s);
void trace_collect();
bool trace_timing_enabled();

// Launches and event pairs recorded while a CUDA graph is being captured.
// The events become external event-record nodes of the graph, so every replay
// re-records them; trace_replayed() accounts one completed replay.
struct GraphTrace {
  bool timed = false;
  int64_t launches[KC_COUNT] = {};
  int kc[4096];
  cudaEvent_t a[4096];
  cudaEvent_t b[4096];
  int npairs = 0;
  void release();
};
void trace_capture_begin(GraphTrace* g);  // route trace_begin/end into g
void trace_capture_end();
// After a replay has completed: adds its launches, and the times of its
// first `useful_pairs` timed launches (launches of steps in which some
// vector was still iterating; later steps exit at entry and are not timed).
void trace_replayed(const GraphTrace* g, int useful_pairs);

template <typename F>
inline cudaError_t traced(int kc, cudaStream_t s, int nkernels, F f) {
  trace_begin(kc, s, nkernels);
  cudaError_t e = f();
  trace_end(kc, s);
  return e;
}

}  // namespace gmrf
