// async.cu -- the asynchronous form of the calls (include/gmrf.h,
// gmrf_submit_* / gmrf_poll / gmrf_wait): each problem that receives a submit
// gets one library-owned host worker thread that runs its submitted calls in
// order, each exactly as the synchronous call would run it.  Host code only.
#include <cuda_runtime.h>

#include <condition_variable>
#include <deque>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <thread>

#include "internal.h"

namespace {

struct Worker {
  std::thread th;
  std::mutex mu;
  std::condition_variable cv;                 // queue changes and results
  std::deque<std::pair<int64_t, std::function<int()>>> q;
  std::map<int64_t, int> done;                // ticket -> return code
  int64_t next = 1;
  bool stop = false;
  int dev = 0;

  void run() {
    cudaSetDevice(dev);
    for (;;) {
      std::pair<int64_t, std::function<int()>> job;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv.wait(lk, [&] { return stop || !q.empty(); });
        if (q.empty()) return;  // stop requested and nothing left
        job = std::move(q.front());
        q.pop_front();
      }
      const int rc = job.second();
      {
        std::lock_guard<std::mutex> lk(mu);
        done[job.first] = rc;
      }
      cv.notify_all();
    }
  }
};

std::mutex g_mu;
std::map<const gmrf_problem*, std::shared_ptr<Worker>> g_workers;

std::shared_ptr<Worker> worker_of(const gmrf_problem* p, bool create) {
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_workers.find(p);
  if (it != g_workers.end()) return it->second;
  if (!create) return nullptr;
  auto w = std::make_shared<Worker>();
  if (cudaGetDevice(&w->dev) != cudaSuccess) {
    cudaGetLastError();
    w->dev = 0;
  }
  w->th = std::thread([w] { w->run(); });
  g_workers[p] = w;
  return w;
}

int submit(gmrf_problem* p, std::function<int()> job, int64_t* ticket) {
  std::shared_ptr<Worker> w;
  try {
    w = worker_of(p, true);
  } catch (...) {
    return GMRF_ERR_OOM;
  }
  {
    std::lock_guard<std::mutex> lk(w->mu);
    *ticket = w->next++;
    w->q.emplace_back(*ticket, std::move(job));
  }
  w->cv.notify_all();
  return GMRF_OK;
}

}  // namespace

namespace gmrf {
// Called by gmrf_destroy before the problem is freed: runs what was submitted,
// then joins the worker.
void async_shutdown(const gmrf_problem* p) {
  std::shared_ptr<Worker> w;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_workers.find(p);
    if (it == g_workers.end()) return;
    w = it->second;
    g_workers.erase(it);
  }
  {
    std::lock_guard<std::mutex> lk(w->mu);
    w->stop = true;
  }
  w->cv.notify_all();
  if (w->th.joinable()) w->th.join();
}
}  // namespace gmrf

extern "C" {

int gmrf_submit_sample(gmrf_problem* p, const gmrf_sample_opts* opts, void* x_out, gmrf_result_info* info,
                       int64_t* ticket) {
  if (!p || !opts || !ticket) return GMRF_ERR_INVALID;
  const gmrf_sample_opts o = *opts;  // copied: the caller's struct may go away
  return submit(p, [=] { return gmrf_sample(p, &o, x_out, info); }, ticket);
}

int gmrf_submit_logdet(gmrf_problem* p, const gmrf_logdet_opts* opts, double* logdet, double* std_err,
                       double* q_out, gmrf_result_info* info, int64_t* ticket) {
  if (!p || !opts || !ticket) return GMRF_ERR_INVALID;
  const gmrf_logdet_opts o = *opts;
  return submit(p, [=] { return gmrf_logdet(p, &o, logdet, std_err, q_out, info); }, ticket);
}

int gmrf_submit_solve(gmrf_problem* p, const gmrf_solve_opts* opts, const void* b, void* x, gmrf_result_info* info,
                      int64_t* ticket) {
  if (!p || !opts || !ticket) return GMRF_ERR_INVALID;
  const gmrf_solve_opts o = *opts;
  return submit(p, [=] { return gmrf_solve(p, &o, b, x, info); }, ticket);
}

int gmrf_poll(gmrf_problem* p, int64_t ticket, int32_t* done, int32_t* result) {
  if (!p || !done) return GMRF_ERR_INVALID;
  auto w = worker_of(p, false);
  if (!w) return GMRF_ERR_INVALID;
  std::lock_guard<std::mutex> lk(w->mu);
  if (ticket < 1 || ticket >= w->next) return GMRF_ERR_INVALID;
  auto it = w->done.find(ticket);
  *done = it != w->done.end();
  if (*done && result) *result = it->second;
  return GMRF_OK;
}

int gmrf_wait(gmrf_problem* p, int64_t ticket, int32_t* result) {
  if (!p) return GMRF_ERR_INVALID;
  auto w = worker_of(p, false);
  if (!w) return GMRF_ERR_INVALID;
  std::unique_lock<std::mutex> lk(w->mu);
  if (ticket < 1 || ticket >= w->next) return GMRF_ERR_INVALID;
  w->cv.wait(lk, [&] { return w->done.count(ticket) != 0; });
  if (result) *result = w->done[ticket];
  return GMRF_OK;
}

}  // extern "C"
