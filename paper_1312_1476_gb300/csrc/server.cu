// server.cu -- continuous batching of sample and log-det requests over one
// problem (include/gmrf.h, gmrf_server_*).
//
// The samples of Algorithm 1 and the probes of Section 6 are independent
// Lanczos runs, and every step kernel of this library reads the step index of
// each vector from that vector's own state.  So vectors at different steps can
// share one launch: the server keeps a fixed table of `nslots` vector slots
// (basis V_m, alpha/beta, state) resident on the device, captures one CUDA
// graph of c steps over the whole table, and between replays
//   * admits waiting vectors into free slots (FIFO over requests): z or the
//     probe from the request's Philox stream, ||z||, a fresh state;
//   * finishes every vector that stopped: a sample gets T_m^{-1/2} e_1,
//     x = ||z|| V_m y (M^{-1/2} u when preconditioned), tau^{-1/2} and the
//     accuracy check of gmrf_sample (with its extra steps where the check asks
//     for them); a probe gets its quadrature term;
//   * completes a request when its last vector has finished (log det: the
//     reduction over its probes).
// Idle slots cost one early-exit block per kernel.  A vector's arithmetic
// never depends on its slot or on the other slots, so every result is bitwise
// the one gmrf_sample / gmrf_logdet return for the same request.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <deque>
#include <map>
#include <vector>

#include "host.h"

using namespace gmrf;
using namespace host;

namespace {

enum { KIND_SAMPLE = 0, KIND_LOGDET = 1 };

struct Req {
  int kind = 0, count = 0;
  uint64_t seed = 0;
  double tau = 1.0;
  void* x = nullptr;          // samples: device [count][n]
  int admitted = 0, finished = 0;
  std::vector<VecState> st;   // final state of each vector
  DevBuf q;                   // log det: [count] quadrature terms + 2 results
  double logdet = NAN, std_err = NAN;
  bool done = false;
};

struct Slot {
  int64_t req = -1;     // owning request, -1: free
  int vec = 0;          // vector index within the request
  int round = 0;        // resumptions asked by the accuracy check so far
  double est_prev = 0.0;
};

}  // namespace

struct gmrf_server {
  gmrf_problem* p = nullptr;
  gmrf_server_opts o{};
  LanczosBufs b;
  std::vector<Slot> slots;
  std::vector<VecState> hst;      // host copy of the slot states after a replay
  std::map<int64_t, Req> reqs;
  std::deque<int64_t> pending;    // requests with vectors still to admit (FIFO)
  int64_t next_id = 1;
  DevBuf mmin;                    // [nslots] zeros: fresh states have no minimum step count
};

namespace {

// Marks the problem as driven by its server for the duration of a server call.
struct Inside {
  gmrf_problem* p;
  explicit Inside(gmrf_problem* q) : p(q) { p->in_server = true; }
  ~Inside() { p->in_server = false; }
};

// Admits waiting vectors into free slots, in request order.
int admit(gmrf_server* sv) {
  gmrf_problem* p = sv->p;
  const size_t n = p->g.n, es = esize(p);
  const int ns = sv->o.nslots;
  cudaStream_t s = p->ws;
  int a = 0;  // search position for free slots
  while (!sv->pending.empty()) {
    Req& r = sv->reqs[sv->pending.front()];
    while (r.admitted < r.count) {
      while (a < ns && sv->slots[a].req >= 0) ++a;
      if (a >= ns) return GMRF_OK;  // no free slot: the rest waits
      int len = 0;
      while (a + len < ns && sv->slots[a + len].req < 0) ++len;
      const int cnt = std::min(len, r.count - r.admitted);
      LanczosBufs bs = sub_batch(sv->b, a, cnt, n, es);
      bs.m_min = (const int*)sv->mmin.p;
      // the z (or probe) streams of gmrf_sample (gmrf_logdet): vector k of the
      // request is Philox stream k of its seed
      CK(traced(KC_RNG, s, 1, [&] {
        return launch_rng(r.kind == KIND_SAMPLE ? 0 : 1, p->fp64, cnt, (int64_t)n, r.seed, r.admitted, bs.W[0], s);
      }));
      CK(traced(KC_INIT, s, 1, [&] { return launch_lanczos_init(p->fp64, n, bs, s); }));
      for (int i = 0; i < cnt; ++i) {
        Slot& sl = sv->slots[a + i];
        sl.req = sv->pending.front();
        sl.vec = r.admitted + i;
        sl.round = 0;
        sl.est_prev = 0.0;
      }
      r.admitted += cnt;
      a += cnt;
    }
    sv->pending.pop_front();
  }
  return GMRF_OK;
}

// Finishes the sample vectors of slots [a, a + k) (one request, consecutive
// vectors); vectors the accuracy check sends back for more steps stay in
// their slots.
int finish_samples(gmrf_server* sv, int a, int k, Req& r) {
  gmrf_problem* p = sv->p;
  const size_t n = p->g.n, es = esize(p);
  const int m_max = sv->o.m_max;
  cudaStream_t s = p->ws;
  const LanczosBufs bs = sub_batch(sv->b, a, k, n, es);
  const int vec0 = sv->slots[a].vec;
  void* dst = (char*)r.x + (size_t)vec0 * n * es;
  const double xs = 1.0 / std::sqrt(p->tau * r.tau);
  CK(traced(KC_TM, s, 3, [&] {
    return launch_tm_inv_sqrt(bs, p->fp64, (TmNodes*)p->nodes.p, (double*)p->scratch.p, (double*)p->y.p, s);
  }));
  CKR(check_tm(p, bs, s));
  CKR(ensure(p->ucg, (size_t)k * n * es, p->ws));
  CKR(ensure(p->zre, (size_t)k * n * es, p->ws));
  const double* y = (const double*)p->y.p;
  const double* ycg = (const double*)p->ycg.p;
  // the same arithmetic as gmrf_sample for each kind of problem
  if (sparse_f(p) || (!p->sp && p->precond != GMRF_PREC_NONE)) {
    CKR(ensure(p->work, (size_t)k * n * es, p->ws));
    CK(traced(KC_ASSEMBLE, s, 1,
              [&] { return launch_assemble_dual(p->fp64, n, bs, y, m_max, 1.0, p->work.p, ycg, p->ucg.p, s); }));
    if (p->sp)
      CK(traced(KC_PRE_APPLY, s, 1, [&] { return launch_sparse_ops(*p->sp, 2, p->work.p, dst, k, s); }));
    else
      CK(traced(KC_PRE_APPLY, s, 3,
                [&] { return launch_precond_apply(p->pre, p->g, p->fp64, PRE_INV_SQRT, p->work.p, dst, k, s); }));
    CK(traced(KC_OTHER, s, 1, [&] { return launch_scale(p->fp64, dst, (size_t)k * n, xs, s); }));
  } else {
    CK(traced(KC_ASSEMBLE, s, 1,
              [&] { return launch_assemble_dual(p->fp64, n, bs, y, m_max, xs, dst, ycg, p->ucg.p, s); }));
  }
  // the accuracy check of gmrf_sample, on z regenerated from the request's stream
  CK(traced(KC_RNG, s, 1, [&] { return launch_rng(0, p->fp64, k, (int64_t)n, r.seed, vec0, p->zre.p, s); }));
  std::vector<double> ests((size_t)k);
  CKR(check_vectors(p, k, p->zre.p, p->ucg.p, sv->b.st + a, sv->hst.data() + a, sv->o.tol, ests.data(), s));
  bool resumed = false;
  for (int i = 0; i < k; ++i) {
    Slot& sl = sv->slots[a + i];
    VecState& v = sv->hst[a + i];
    double est = ests[i], prev = sl.est_prev;
    int mm = 0;
    // one vector's round of gmrf_sample's rule
    if (check_resume(&v, &est, &prev, &mm, 1, sv->o.tol, m_max, sl.round)) {
      sl.round += 1;
      sl.est_prev = est;
      resumed = true;
      continue;
    }
    check_apply(&v, &est, 1, sv->o.tol);
    r.st[sl.vec] = v;
    r.finished += 1;
    sl.req = -1;
  }
  if (resumed) CK(cudaMemcpyAsync(sv->b.st + a, sv->hst.data() + a, sizeof(VecState) * k, cudaMemcpyHostToDevice, s));
  return GMRF_OK;
}

// Finishes the probe vectors of slots [a, a + k): their quadrature terms.
int finish_probes(gmrf_server* sv, int a, int k, Req& r) {
  gmrf_problem* p = sv->p;
  const size_t n = p->g.n, es = esize(p);
  cudaStream_t s = p->ws;
  const LanczosBufs bq = sub_batch(sv->b, a, k, n, es);
  const int vec0 = sv->slots[a].vec;
  CK(traced(KC_TM, s, 2, [&] { return launch_tm_log(bq, p->fp64, (TmNodes*)p->nodes.p, (double*)r.q.p + vec0, s); }));
  for (int i = 0; i < k; ++i) {
    Slot& sl = sv->slots[a + i];
    r.st[sl.vec] = sv->hst[a + i];
    r.finished += 1;
    sl.req = -1;
  }
  return GMRF_OK;
}

int complete(gmrf_server* sv, Req& r) {
  gmrf_problem* p = sv->p;
  cudaStream_t s = p->ws;
  if (r.kind == KIND_LOGDET) {
    // log det (tau Q) = mean q + log det M + n log tau  (Section 6.2, plus sign)
    const double shift = p->logdet_M + (double)p->g.n * std::log(p->tau * r.tau);
    double* q = (double*)r.q.p;
    CK(traced(KC_TM, s, 1, [&] { return launch_logdet_reduce(q, r.count, 1, shift, q + r.count, s); }));
    double res[2];
    CK(cudaMemcpyAsync(res, q + r.count, sizeof(res), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    r.logdet = res[0];
    r.std_err = res[1];
    release(r.q, s);
  }
  r.done = true;
  return GMRF_OK;
}

int step_body(gmrf_server* sv, int32_t* active) {
  gmrf_problem* p = sv->p;
  cudaStream_t s = p->ws;
  const int ns = sv->o.nslots;
  CKR(admit(sv));
  int running = 0, hw = 0;
  for (int i = 0; i < ns; ++i)
    if (sv->slots[i].req >= 0) {  // admitted or resumed: the replay runs them
      ++running;
      hw = i + 1;
    }
  if (running) {
    // The replay covers the slots up to the highest one in use (admission
    // fills the lowest free slots), rounded up to 8 so that the step graph is
    // recaptured only when that prefix grows or shrinks by a block of slots:
    // idle slots beyond it would cost an early-exit block per kernel each.
    const int hw8 = std::min(ns, (hw + 7) / 8 * 8);
    const LanczosBufs bp = sub_batch(sv->b, 0, hw8, p->g.n, esize(p));
    const StepParams P = step_params(p, bp, sv->o.tol, sv->o.m_max, false);
    const int c = std::min(sv->o.check_every > 0 ? sv->o.check_every : 16, sv->o.m_max);
    if (p->precond != GMRF_PREC_NONE && !p->sp) CKR(precond_prepare(p->pre, hw8, s));
    CKR(capture_steps(p, bp, P, c));
    CK(cudaGraphLaunch(p->graph.exec, s));
    trace_replayed(&p->graph.tr, c * p->graph.kernels_per_step);
  }
  CK(cudaMemcpyAsync(sv->hst.data(), sv->b.st, sizeof(VecState) * ns, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  // vectors that stopped, in runs of consecutive slots of one request with
  // consecutive vector indices
  for (int i = 0; i < ns;) {
    const Slot& sl = sv->slots[i];
    if (sl.req < 0 || sv->hst[i].status == VS_RUNNING) {
      ++i;
      continue;
    }
    int k = 1;
    while (i + k < ns && sv->slots[i + k].req == sl.req && sv->slots[i + k].vec == sl.vec + k &&
           sv->hst[i + k].status != VS_RUNNING)
      ++k;
    Req& r = sv->reqs[sl.req];
    CKR(r.kind == KIND_SAMPLE ? finish_samples(sv, i, k, r) : finish_probes(sv, i, k, r));
    if (r.finished == r.count && !r.done) CKR(complete(sv, r));
    i += k;
  }
  trace_collect();
  int act = 0;
  for (int i = 0; i < ns; ++i) act += sv->slots[i].req >= 0;
  for (int64_t id : sv->pending) act += sv->reqs[id].count - sv->reqs[id].admitted;
  if (active) *active = act;
  return GMRF_OK;
}

}  // namespace

extern "C" {

int gmrf_server_create(gmrf_problem* p, const gmrf_server_opts* o, gmrf_server** out) {
  if (!p || !o || !out) return GMRF_ERR_INVALID;
  *out = nullptr;
  if (o->nslots < 1 || o->nslots > 65535 || o->m_max < 1 || o->m_max > 8192 || !(o->tol > 0.0) ||
      !std::isfinite(o->tol) || o->reserved != 0)
    return GMRF_ERR_INVALID;
  if (p->server) return GMRF_ERR_INVALID;
  gmrf_server* sv = new (std::nothrow) gmrf_server();
  if (!sv) return GMRF_ERR_OOM;
  sv->p = p;
  sv->o = *o;
  const int ns = o->nslots;
  int rc = enter(p);
  if (rc == GMRF_OK) rc = ensure_lanczos(p, ns, o->m_max + 1, o->m_max, true, sv->b);
  if (rc == GMRF_OK) rc = ensure_host_states(p, ns);
  if (rc == GMRF_OK) rc = ensure(sv->mmin, sizeof(int) * ns, p->ws);
  if (rc == GMRF_OK && cudaMemsetAsync(sv->mmin.p, 0, sizeof(int) * ns, p->ws) != cudaSuccess) rc = GMRF_ERR_CUDA;
  // every slot starts free: a finished state, which the step kernels skip
  std::vector<VecState> idle((size_t)ns);
  for (auto& v : idle) {
    v = VecState{};
    v.status = VS_DONE;
  }
  if (rc == GMRF_OK && cudaMemcpyAsync(sv->b.st, idle.data(), sizeof(VecState) * ns, cudaMemcpyHostToDevice, p->ws) !=
                           cudaSuccess)
    rc = GMRF_ERR_CUDA;
  if (rc == GMRF_OK && cudaStreamSynchronize(p->ws) != cudaSuccess) rc = GMRF_ERR_CUDA;
  leave(p);
  if (rc != GMRF_OK) {
    cudaGetLastError();
    release(sv->mmin, p->ws);
    delete sv;
    return rc;
  }
  sv->slots.assign((size_t)ns, Slot{});
  sv->hst.assign((size_t)ns, VecState{});
  p->server = sv;
  *out = sv;
  return GMRF_OK;
}

int gmrf_server_submit(gmrf_server* sv, int32_t kind, int32_t count, uint64_t seed, double tau, void* x_out,
                       int64_t* req) {
  if (!sv || !req || count < 1 || count > (1 << 24) || !(tau > 0.0) || !std::isfinite(tau)) return GMRF_ERR_INVALID;
  if (kind != KIND_SAMPLE && kind != KIND_LOGDET) return GMRF_ERR_INVALID;
  if (kind == KIND_SAMPLE && (!x_out || !is_device_ptr(x_out))) return GMRF_ERR_INVALID;
  Req r;
  r.kind = kind;
  r.count = count;
  r.seed = seed;
  r.tau = tau;
  r.x = x_out;
  r.st.assign((size_t)count, VecState{});
  if (kind == KIND_LOGDET) {
    Inside in(sv->p);
    CKR(ensure(r.q, sizeof(double) * ((size_t)count + 2), sv->p->ws));
  }
  const int64_t id = sv->next_id++;
  sv->reqs.emplace(id, std::move(r));
  sv->pending.push_back(id);
  *req = id;
  return GMRF_OK;
}

int gmrf_server_step(gmrf_server* sv, int32_t* active) {
  if (!sv) return GMRF_ERR_INVALID;
  Inside in(sv->p);
  CKR(enter(sv->p));
  const int rc = step_body(sv, active);
  const int rl = leave(sv->p);
  return rc != GMRF_OK ? rc : rl;
}

int gmrf_server_poll(gmrf_server* sv, int64_t req, int32_t* done, int32_t* result, gmrf_result_info* info,
                     double* logdet, double* std_err) {
  if (!sv || !done) return GMRF_ERR_INVALID;
  auto it = sv->reqs.find(req);
  if (it == sv->reqs.end()) return GMRF_ERR_INVALID;
  Req& r = it->second;
  *done = r.done ? 1 : 0;
  if (!r.done) return GMRF_OK;
  if (result) *result = worst_status(r.st.data(), r.count);
  fill_info(r.st.data(), r.count, info);
  if (logdet) *logdet = r.logdet;
  if (std_err) *std_err = r.std_err;
  sv->reqs.erase(it);
  return GMRF_OK;
}

void gmrf_server_destroy(gmrf_server* sv) {
  if (!sv) return;
  gmrf_problem* p = sv->p;
  if (p->ws) cudaStreamSynchronize(p->ws);
  for (auto& kv : sv->reqs) release(kv.second.q, p->ws);
  release(sv->mmin, p->ws);
  if (p->ws) cudaStreamSynchronize(p->ws);
  p->server = nullptr;
  delete sv;
}

}  // extern "C"
