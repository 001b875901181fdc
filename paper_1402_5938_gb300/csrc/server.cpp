// Solve server: continuous batching of independent solves on one GPU.
//
// Requests (a problem descriptor, a nodal right-hand side on the host, a tolerance) enter a
// FIFO queue. `max_slots` worker threads, each with its own CUDA stream, take requests as
// soon as a slot is free and the request's peak device memory fits the budget next to what
// is resident, so work of different requests overlaps on the device. Hierarchies stay
// resident after their solve in an LRU cache keyed by the descriptor: a later request with
// the same problem skips the setup; idle cached hierarchies are evicted when an admission
// needs their memory. Every request records its latency from submit to completion.
#include <string.h>

#include "common.cuh"

#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/hmg.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  unsigned long long ticket = 0;
  hmg_desc desc{};
  std::string key;
  std::vector<double> f;
  double rtol = 1e-8;
  int mode = HMG_MODE_PCG;
  int maxit = 1000;
  size_t need = 0;  // admission reservation (peak bytes of a setup; 0 when served from cache)
  Clock::time_point t_submit, t_done;
  std::vector<double> u;
  int iters = 0;
  double res0 = 0, res_final = 0;
  hmg_status status = HMG_EBUSY;
  bool done = false;
  bool cache_hit = false;
};

struct Cached {
  hmg_problem* prob = nullptr;
  size_t bytes = 0;
  bool busy = false;
  unsigned long long last_used = 0;
};

struct Worker {
  cudaStream_t stream = nullptr;
  double *d_f = nullptr, *d_b = nullptr, *d_u = nullptr;
  double *h_f = nullptr, *h_u = nullptr;
  size_t cap = 0;  // entries of the buffers
};

std::string key_of(const hmg_desc& d) { return std::string(reinterpret_cast<const char*>(&d), sizeof(d)); }

}  // namespace

struct hmg_server {
  int device = 0;
  size_t budget = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Request>> queue;
  std::unordered_map<unsigned long long, std::shared_ptr<Request>> tickets;
  std::unordered_map<std::string, Cached> cache;
  std::unordered_map<std::string, int> pending;  // problems whose setup is running
  size_t resident = 0;  // cached hierarchies + worker buffers
  size_t reserved = 0;  // admitted setups not yet resident
  unsigned long long next_ticket = 1, tick = 0;
  long long completed = 0, cache_hits = 0;
  int inflight = 0;
  bool admitting = false;  // a worker is inside admit(), which may drop the lock to evict
  bool stop = false;
  std::vector<std::thread> threads;
  std::vector<Worker> workers;

  void run(int w);
  bool admit(std::shared_ptr<Request>& r, std::unique_lock<std::mutex>& lk);
};

// Called with the lock held: decide whether the head request can start now.
bool hmg_server::admit(std::shared_ptr<Request>& r, std::unique_lock<std::mutex>& lk) {
  if (pending.count(r->key)) return false;  // its hierarchy is being built: reuse it when ready
  auto it = cache.find(r->key);
  if (it != cache.end()) {
    if (it->second.busy) return false;  // same problem in use: wait for it (keeps FIFO order)
    it->second.busy = true;
    r->cache_hit = true;
    r->need = 0;
    return true;
  }
  size_t res = 0, peak = 0;
  if (hmg_estimate_bytes(&r->desc, &res, &peak) != HMG_OK) peak = 0;
  peak += 3 * hmg_desc_ndof(&r->desc) * sizeof(double);  // the worker's vectors may grow
  // evict idle cached hierarchies, least recently used first, until the request fits
  while (resident + reserved + peak > budget) {
    auto victim = cache.end();
    for (auto c = cache.begin(); c != cache.end(); ++c)
      if (!c->second.busy && (victim == cache.end() || c->second.last_used < victim->second.last_used)) victim = c;
    if (victim == cache.end()) break;
    hmg_problem* p = victim->second.prob;
    resident -= victim->second.bytes;
    cache.erase(victim);
    lk.unlock();
    hmg_destroy(p);
    lk.lock();
  }
  if (resident + reserved + peak > budget) return false;
  reserved += peak;
  r->need = peak;
  pending[r->key] = 1;
  return true;
}

void hmg_server::run(int w) {
  cudaSetDevice(device);
  Worker& W = workers[w];
  std::unique_lock<std::mutex> lk(mu);
  for (;;) {
    std::shared_ptr<Request> r;
    cv_work.wait(lk, [&] {
      if (stop) return true;
      if (admitting) return false;  // one admission at a time: admit() may unlock to evict
      bool got = false;
      admitting = true;
      while (!queue.empty()) {
        std::shared_ptr<Request> head = queue.front();
        if (admit(head, lk)) {
          r = head;
          queue.pop_front();
          got = true;
          break;
        }
        // nothing running or cached could make room: this request can never start
        if (inflight == 0 && cache.empty()) {
          queue.pop_front();
          head->status = HMG_ENOMEM;
          head->done = true;
          head->t_done = Clock::now();
          cv_done.notify_all();
          continue;
        }
        break;
      }
      admitting = false;
      cv_work.notify_all();  // let waiting workers look at the new queue head
      return got;
    });
    if (stop && !r) return;
    if (!r) continue;
    ++inflight;
    hmg_problem* P = nullptr;
    if (r->cache_hit) {
      P = cache[r->key].prob;
      ++cache_hits;
    }
    lk.unlock();

    hmg_status st = HMG_OK;
    const size_t n = hmg_desc_ndof(&r->desc);
    size_t grow = 0;
    if (!P) st = hmg_setup(&r->desc, W.stream, &P);
    if (st == HMG_OK && n > W.cap) {
      // stream-ordered device memory and pooled pinned memory: no implicit device barrier
      if (W.d_f) {
        hmg::dev_free(W.d_f, W.stream);
        hmg::dev_free(W.d_b, W.stream);
        hmg::dev_free(W.d_u, W.stream);
        hmg::pinned_free(W.h_f, W.cap * 8);
        hmg::pinned_free(W.h_u, W.cap * 8);
      }
      W.d_f = W.d_b = W.d_u = W.h_f = W.h_u = nullptr;
      grow = (n - W.cap) * 3 * sizeof(double);
      W.h_f = static_cast<double*>(hmg::pinned_alloc(n * 8));
      W.h_u = static_cast<double*>(hmg::pinned_alloc(n * 8));
      if (hmg::dev_alloc((void**)&W.d_f, n * 8, W.stream) != cudaSuccess ||
          hmg::dev_alloc((void**)&W.d_b, n * 8, W.stream) != cudaSuccess ||
          hmg::dev_alloc((void**)&W.d_u, n * 8, W.stream) != cudaSuccess || !W.h_f || !W.h_u) {
        st = HMG_ENOMEM;
        W.cap = 0;
      } else {
        W.cap = n;
      }
    }
    std::vector<double> hist((size_t)r->maxit + 1, 0.0);
    int iters = 0;
    if (st == HMG_OK) {
      memcpy(W.h_f, r->f.data(), n * sizeof(double));
      if (cudaMemcpyAsync(W.d_f, W.h_f, n * 8, cudaMemcpyHostToDevice, W.stream) != cudaSuccess) st = HMG_EDEVICE;
      if (st == HMG_OK) st = hmg_rhs(P, W.d_f, W.d_b, W.stream);
      if (st == HMG_OK) {
        st = hmg_solve(P, r->mode, W.d_b, W.d_u, r->rtol, r->maxit, &iters, hist.data(), W.stream);
        if (st == HMG_OK || st == HMG_ENOCONV) {
          r->u.resize(n);
          if (cudaMemcpyAsync(W.h_u, W.d_u, n * 8, cudaMemcpyDeviceToHost, W.stream) != cudaSuccess ||
              cudaStreamSynchronize(W.stream) != cudaSuccess)
            st = HMG_EDEVICE;
          else
            memcpy(r->u.data(), W.h_u, n * sizeof(double));
        }
      }
    }

    lk.lock();
    --inflight;
    resident += grow;
    if (r->cache_hit) {
      Cached& c = cache[r->key];
      c.busy = false;
      c.last_used = ++tick;
    } else {
      reserved -= r->need;
      pending.erase(r->key);
      if (P && (st == HMG_OK || st == HMG_ENOCONV)) {
        Cached c;
        c.prob = P;
        c.bytes = hmg_device_bytes(P);
        c.last_used = ++tick;
        resident += c.bytes;
        cache[r->key] = c;
      } else if (P) {
        lk.unlock();
        hmg_destroy(P);
        lk.lock();
      }
    }
    r->iters = iters;
    r->res0 = hist[0];
    r->res_final = hist[(size_t)std::min(iters, r->maxit)];
    r->status = st;
    r->t_done = Clock::now();
    r->done = true;
    ++completed;
    cv_done.notify_all();
    cv_work.notify_all();
  }
}

extern "C" {

hmg_status hmg_server_create(int device, size_t hbm_budget, int max_slots, hmg_server** out) {
  if (!out || max_slots < 1 || max_slots > 256 || hbm_budget == 0) return HMG_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return HMG_EDEVICE;
  hmg_server* s = new (std::nothrow) hmg_server();
  if (!s) return HMG_ENOMEM;
  s->device = device;
  s->budget = hbm_budget;
  s->workers.resize(max_slots);
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(device);
  for (auto& w : s->workers) {
    if (cudaStreamCreateWithFlags(&w.stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaSetDevice(prev);
      for (auto& w2 : s->workers)
        if (w2.stream) cudaStreamDestroy(w2.stream);
      delete s;
      return HMG_EDEVICE;
    }
  }
  cudaSetDevice(prev);
  for (int i = 0; i < max_slots; ++i) s->threads.emplace_back([s, i] { s->run(i); });
  *out = s;
  return HMG_OK;
}

hmg_status hmg_server_submit(hmg_server* s, const hmg_desc* desc, const double* f_host, double rtol, int mode,
                             int maxit, unsigned long long* ticket) {
  if (!s || !desc || !f_host || !ticket || !(rtol >= 0.0) || maxit < 0 || (mode != HMG_MODE_MG && mode != HMG_MODE_PCG))
    return HMG_EINVAL;
  const size_t n = hmg_desc_ndof(desc);
  if (n == 0) return HMG_EINVAL;
  if (desc->node_xyz || desc->mu_fn) return HMG_EINVAL;  // the server caches by descriptor values only
  size_t res = 0, peak = 0;
  hmg_status st = hmg_estimate_bytes(desc, &res, &peak);
  if (st != HMG_OK) return st;
  auto r = std::make_shared<Request>();
  r->desc = *desc;
  r->key = key_of(*desc);
  r->f.assign(f_host, f_host + n);
  r->rtol = rtol;
  r->mode = mode;
  r->maxit = maxit;
  r->t_submit = Clock::now();
  std::lock_guard<std::mutex> lk(s->mu);
  if (peak + 3 * n * sizeof(double) > s->budget) return HMG_ENOMEM;  // can never be admitted
  r->ticket = s->next_ticket++;
  *ticket = r->ticket;
  s->tickets[r->ticket] = r;
  s->queue.push_back(r);
  s->cv_work.notify_all();
  return HMG_OK;
}

static hmg_status take_result(hmg_server* s, std::unordered_map<unsigned long long, std::shared_ptr<Request>>::iterator it,
                              double* u_host, int* iters, double* res_final, double* latency_s) {
  std::shared_ptr<Request> r = it->second;
  s->tickets.erase(it);
  if (u_host && !r->u.empty()) memcpy(u_host, r->u.data(), r->u.size() * sizeof(double));
  if (iters) *iters = r->iters;
  if (res_final) *res_final = r->res0 > 0 ? r->res_final / r->res0 : 0.0;
  if (latency_s) *latency_s = std::chrono::duration<double>(r->t_done - r->t_submit).count();
  return r->status;
}

hmg_status hmg_server_poll(hmg_server* s, unsigned long long ticket, double* u_host, int* iters, double* res_final,
                           double* latency_s) {
  if (!s) return HMG_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->tickets.find(ticket);
  if (it == s->tickets.end()) return HMG_EINVAL;
  if (!it->second->done) return HMG_EBUSY;
  return take_result(s, it, u_host, iters, res_final, latency_s);
}

hmg_status hmg_server_wait(hmg_server* s, unsigned long long ticket, double timeout_s, double* u_host, int* iters,
                           double* res_final, double* latency_s) {
  if (!s) return HMG_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->tickets.find(ticket);
  if (it == s->tickets.end()) return HMG_EINVAL;
  std::shared_ptr<Request> r = it->second;
  const bool ok = s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] { return r->done; });
  if (!ok) return HMG_ETIMEOUT;
  return take_result(s, s->tickets.find(ticket), u_host, iters, res_final, latency_s);
}

hmg_status hmg_server_stats(hmg_server* s, long long* completed, long long* cache_hits, size_t* resident_bytes,
                            int* queued) {
  if (!s) return HMG_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (completed) *completed = s->completed;
  if (cache_hits) *cache_hits = s->cache_hits;
  if (resident_bytes) *resident_bytes = s->resident;
  if (queued) *queued = (int)s->queue.size();
  return HMG_OK;
}

hmg_status hmg_server_destroy(hmg_server* s) {
  if (!s) return HMG_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv_work.notify_all();
  }
  for (auto& t : s->threads) t.join();
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(s->device);
  for (auto& c : s->cache) hmg_destroy(c.second.prob);
  for (auto& w : s->workers) {
    if (w.d_f) {
      hmg::dev_free(w.d_f, w.stream);
      hmg::dev_free(w.d_b, w.stream);
      hmg::dev_free(w.d_u, w.stream);
      hmg::pinned_free(w.h_f, w.cap * 8);
      hmg::pinned_free(w.h_u, w.cap * 8);
    }
    if (w.stream) {
      cudaStreamSynchronize(w.stream);
      cudaStreamDestroy(w.stream);
    }
  }
  cudaSetDevice(prev);
  delete s;
  return HMG_OK;
}

}  // extern "C"
