// fv_server.cu — continuous-batching server for solve requests.
//
// Requests (one initial state, a grid size, a horizon, plain or learned) are
// queued by fv_submit().  A worker thread admits them in arrival order as slots
// and device memory free up (admission by device-memory footprint), keeps
// every admitted state resident on the device, and advances all of them in
// rounds: each admitted request has its own stream and gets the next chunk of
// its steps enqueued as graph replays as soon as its previous chunk is done,
// so the work of requests that arrived at different times overlaps on the
// GPU.  A finished request's state is copied to host memory and its device
// memory released for the next waiting request.  fv_poll() reports a ticket's
// result and its latency (submit to completion, host clock).  A request's
// arithmetic does not depend on what else runs: each has its own buffers,
// control block and deterministic kernels, so its result is the same alone
// and in the mix.
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "fv_common.cuh"
#include "fv_internal.h"
#include "stencil_net.cuh"

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Req {
  unsigned long long ticket = 0;
  fv_request r{};
  std::vector<float> q0, result;
  double t_submit = 0, t_admit = 0, t_done = 0;
  int status = FV_PENDING;
  fv_state* st = nullptr;
  long steps_done = 0;
  long chunk_steps = 0;
  bool in_flight = false;
  cudaEvent_t ev = nullptr;
  size_t footprint = 0;
  bool done = false;
  bool fell_back = false;   // learned run became unstable: rerun with the plain step
};

size_t footprint_bytes(const fv_request& r) {
  const size_t cells = (size_t)r.nx * r.ny;
  const size_t C = r.eq == FV_EQ_SWE ? 3 : 4;
  size_t b = 2 * C * 4 * cells + (1 << 20);        // q^n, q^(1), control, diagnostics scratch
  if (r.learned) b += cells * (36 * 4 + 3 * 64);   // coefficients + CNN activations
  return b;
}

}  // namespace

struct fv_server {
  size_t budget = 0, used = 0;
  int max_slots = 1;
  long chunk = 64;
  const fv_net* net = nullptr;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Req*> pending;
  std::vector<Req*> active;
  std::unordered_map<unsigned long long, Req*> all;
  std::thread worker;
  std::atomic<bool> stop{false};
  unsigned long long next_ticket = 1;
  int device = 0;
  long long fallbacks = 0;
};

namespace {

void finish(fv_server* S, Req* q, int status) {
  q->status = status;
  q->t_done = now_s();
  q->done = true;
  if (q->st) fv_destroy_state(q->st);
  q->st = nullptr;
  if (q->ev) cudaEventDestroy(q->ev);
  q->ev = nullptr;
  S->used -= q->footprint;
}

// Create the device state of an admitted request (worker thread, no lock).
int start_request(fv_server* S, Req* q) {
  fv_grid g{q->r.nx, q->r.ny, 1, 1.0, 1.0};
  int rc;
  if (q->r.eq == FV_EQ_SWE) {
    fv_swe_params p{9.81, q->r.cfl, FV_DT_ADAPTIVE, 0.0};
    rc = swe_init(&g, &p, q->q0.data(), FV_HOST, nullptr, &q->st);
  } else {
    fv_euler_params p{1.4, q->r.cfl, FV_DT_ADAPTIVE, 0.0};
    rc = euler_init(&g, &p, q->q0.data(), FV_HOST, nullptr, &q->st);
  }
  if (rc != FV_OK) return rc;
  if (cudaEventCreateWithFlags(&q->ev, cudaEventDisableTiming) != cudaSuccess) return FV_ECUDA;
  if (q->r.learned) {
    rc = fvs::learned_prepare(q->st, S->net);
    if (rc != FV_OK) return rc;
  }
  return FV_OK;
}

void worker_loop(fv_server* S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lock(S->mu);
  while (!S->stop) {
    // admission: arrival order, while a slot and the memory are free
    while (!S->pending.empty() && (int)S->active.size() < S->max_slots &&
           S->used + S->pending.front()->footprint <= S->budget) {
      Req* q = S->pending.front();
      S->pending.pop_front();
      S->used += q->footprint;
      S->active.push_back(q);
      lock.unlock();
      q->t_admit = now_s();
      int rc = start_request(S, q);
      lock.lock();
      if (rc != FV_OK) {
        finish(S, q, rc);
        S->active.pop_back();
      }
    }
    bool progressed = false;
    for (size_t i = 0; i < S->active.size();) {
      Req* q = S->active[i];
      if (q->in_flight) {
        cudaError_t e = cudaEventQuery(q->ev);
        if (e == cudaErrorNotReady) {
          ++i;
          continue;
        }
        q->in_flight = false;
        progressed = true;
        if (e != cudaSuccess) {
          finish(S, q, FV_ECUDA);
          S->active.erase(S->active.begin() + i);
          continue;
        }
        q->steps_done += q->chunk_steps;
        unsigned flags = 0;
        if (fv_health(q->st, &flags) != FV_OK || flags) {
          if (q->r.learned) {
            // the plain step is the learned step's fallback: rerun the request
            // with MUSCL-minmod from its initial state
            fv_destroy_state(q->st);
            q->st = nullptr;
            cudaEventDestroy(q->ev);
            q->ev = nullptr;
            q->r.learned = 0;
            q->fell_back = true;
            q->steps_done = 0;
            ++S->fallbacks;
            lock.unlock();
            int rc = start_request(S, q);
            lock.lock();
            if (rc != FV_OK) {
              finish(S, q, rc);
              S->active.erase(S->active.begin() + i);
              continue;
            }
          } else {
            finish(S, q, FV_EUNSTABLE);
            S->active.erase(S->active.begin() + i);
            continue;
          }
        }
        if (q->steps_done >= q->r.nsteps) {
          q->result.resize(q->q0.size());
          int rc = fv_get_state(q->st, q->result.data(), FV_HOST);
          finish(S, q, rc);
          S->active.erase(S->active.begin() + i);
          continue;
        }
      }
      // next chunk of this request
      const long k = q->r.nsteps - q->steps_done < S->chunk ? q->r.nsteps - q->steps_done : S->chunk;
      lock.unlock();
      int rc = fv_enqueue_steps(q->st, q->r.learned ? S->net : nullptr, k);
      if (rc == FV_OK) {
        void* stream = nullptr;
        fv_state_stream(q->st, &stream);
        if (cudaEventRecord(q->ev, (cudaStream_t)stream) != cudaSuccess) rc = FV_ECUDA;
      }
      lock.lock();
      if (rc != FV_OK) {
        finish(S, q, rc);
        S->active.erase(S->active.begin() + i);
        continue;
      }
      q->chunk_steps = k;
      q->in_flight = true;
      progressed = true;
      ++i;
    }
    if (progressed) S->cv.notify_all();
    if (!progressed) S->cv.wait_for(lock, std::chrono::microseconds(200));
  }
  // shut down: drop whatever is still running (fv_destroy_state waits for it)
  for (Req* q : S->active) finish(S, q, FV_ETIMEOUT);
  S->active.clear();
}

}  // namespace

extern "C" int fv_server_create(size_t hbm_budget_bytes, int max_slots, const fv_net* net,
                                fv_server** out) {
  if (!out || hbm_budget_bytes == 0 || max_slots < 1) return fvh::fail(FV_EINVAL, "bad server arguments");
  fv_server* S = new fv_server();
  S->budget = hbm_budget_bytes;
  S->max_slots = max_slots;
  S->net = net;
  cudaGetDevice(&S->device);
  S->worker = std::thread(worker_loop, S);
  *out = S;
  return FV_OK;
}

extern "C" int fv_server_destroy(fv_server* S) {
  if (!S) return FV_OK;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    S->stop = true;
  }
  S->cv.notify_all();
  if (S->worker.joinable()) S->worker.join();
  for (auto& kv : S->all) delete kv.second;   // every request not yet polled
  delete S;
  return FV_OK;
}

extern "C" int fv_submit(fv_server* S, const fv_request* r, unsigned long long* ticket) {
  if (!S || !r || !ticket || !r->q0) return fvh::fail(FV_EINVAL, "null argument");
  if (r->eq != FV_EQ_SWE && r->eq != FV_EQ_EULER) return fvh::fail(FV_EINVAL, "unknown equation set");
  if (r->nx < 1 || r->ny < 1 || r->nsteps < 1) return fvh::fail(FV_EINVAL, "bad request sizes");
  if (r->learned && (r->eq != FV_EQ_SWE || !S->net))
    return fvh::fail(FV_EINVAL, "learned requests need shallow water and a server network");
  if (r->learned && (!snk::grid_supported(r->nx) || ((long long)r->nx * r->ny) % snk::TILE))
    return fvh::fail(FV_EINVAL, "learned request grid not supported by the network kernels");
  if (!(r->cfl > 0)) return fvh::fail(FV_EINVAL, "cfl must be > 0");
  Req* q = new Req();
  q->r = *r;
  const size_t n = (size_t)r->nx * r->ny * (r->eq == FV_EQ_SWE ? 3 : 4);
  q->q0.assign(r->q0, r->q0 + n);
  q->r.q0 = nullptr;
  q->footprint = footprint_bytes(*r);
  if (q->footprint > S->budget) {
    delete q;
    return fvh::fail(FV_EBUSY, "request needs more device memory than the server budget");
  }
  {
    std::lock_guard<std::mutex> lock(S->mu);
    q->ticket = S->next_ticket++;
    q->t_submit = now_s();
    S->pending.push_back(q);
    S->all[q->ticket] = q;
    *ticket = q->ticket;
  }
  S->cv.notify_all();
  return FV_OK;
}

extern "C" int fv_poll(fv_server* S, unsigned long long ticket, float* q_out, double* latency_s) {
  if (!S) return fvh::fail(FV_EINVAL, "null server");
  std::lock_guard<std::mutex> lock(S->mu);
  auto it = S->all.find(ticket);
  if (it == S->all.end()) return fvh::fail(FV_ENOTFOUND, "unknown ticket");
  Req* q = it->second;
  if (!q->done) return FV_PENDING;
  if (latency_s) *latency_s = q->t_done - q->t_submit;
  const int status = q->status;
  if (status == FV_OK && q_out) std::copy(q->result.begin(), q->result.end(), q_out);
  S->all.erase(it);
  delete q;
  if (status != FV_OK) return fvh::fail(status, "request failed on the device");
  return FV_OK;
}

extern "C" int fv_server_stats(fv_server* S, int* active, int* pending, size_t* used_bytes,
                               long long* fallbacks) {
  if (!S) return fvh::fail(FV_EINVAL, "null server");
  std::lock_guard<std::mutex> lock(S->mu);
  if (active) *active = (int)S->active.size();
  if (pending) *pending = (int)S->pending.size();
  if (used_bytes) *used_bytes = S->used;
  if (fallbacks) *fallbacks = S->fallbacks;
  return FV_OK;
}
