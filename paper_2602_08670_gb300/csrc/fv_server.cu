// fv_server.cu — continuous-batching server for solve requests.
//
// Requests (one initial state, a grid size, a horizon in steps, plain or
// learned) are queued by fv_submit() and admitted in arrival order by a worker
// thread.  Requests of one shape class (equations, plain or learned, grid
// size, CFL number) share a bucket: one resident state of `cap` member slots,
// created once and reused, whose members are advanced together by the same
// kernel launches (one launch per Runge-Kutta stage for all of them, replayed
// from a captured graph chunk of 32 steps).  A request enters a free slot of
// its bucket between two chunks (its initial state copied into the slot, its
// control block reset with its own step limit and time step); a member that
// reaches its step limit stops inside the chunk (the stage kernels skip it),
// and its result is copied out after the chunk, freeing the slot for the next
// waiting request.  Buckets of different shapes run on their own streams, so
// their chunks overlap on the GPU.  Admission: a request is admitted while
// the number of active requests is below max_slots and its bucket has a free
// slot, or a new bucket's device memory (its state's actual allocations) fits
// the budget next to the existing buckets; empty buckets are released when
// the budget is needed.  In steady state nothing is allocated or freed.
// A learned member whose state leaves the physical states (health word) is
// restarted from its initial state on the plain step, the learned step's
// fallback.  fv_poll() reports a ticket's result and its latency (submit to
// result on the host, host clock).  A member's arithmetic does not depend on
// its slot or on the other members (per-member control blocks, kernels that
// never mix members), so a result is the same alone and in the mix.
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

constexpr long CHUNK = 32;                  // steps per graph replay
constexpr long long BUCKET_CELLS = 1 << 22;  // member slots x cells per bucket (at most)
constexpr int MAX_CAP = 64;

struct Bucket;

struct Req {
  unsigned long long ticket = 0;
  fv_request r{};
  std::vector<float> q0, result;
  double t_submit = 0, t_admit = 0, t_done = 0;
  int status = FV_PENDING;
  bool done = false;
  bool fell_back = false;     // learned run became unstable: rerun with the plain step
  Bucket* bucket = nullptr;
  int slot = -1;
  bool started = false;       // its slot has been initialised on the device
  float hmin = 0.f;           // learned positivity threshold (host copy, read by an async copy)
};

struct Key {
  int eq, learned, nx, ny;
  double cfl;
  bool operator==(const Key& o) const {
    return eq == o.eq && learned == o.learned && nx == o.nx && ny == o.ny && cfl == o.cfl;
  }
};

struct Bucket {
  Key key{};
  int cap = 0;
  fv_state* st = nullptr;
  size_t bytes = 0;           // device memory of the state and its learned workspace
  std::vector<Req*> slot;     // nullptr = free
  int used = 0;
  fvk::Ctrl* host_ctrl = nullptr;   // pinned copy of the control blocks after a chunk
  cudaEvent_t ev = nullptr;
  bool in_flight = false;
};

Key key_of(const fv_request& r) { return Key{r.eq, r.learned, r.nx, r.ny, r.cfl}; }

int capacity_for(const fv_request& r) {
  const long long cells = (long long)r.nx * r.ny;
  long long cap = BUCKET_CELLS / (cells > 0 ? cells : 1);
  if (cap < 1) cap = 1;
  if (cap > MAX_CAP) cap = MAX_CAP;
  return (int)cap;
}

// Device memory of a bucket with `cap` slots before it exists (admission
// test): per slot two state buffers (q^n, the stage state), a control block,
// the reduction scratch of the diagnostics and, for learned requests, the
// network's workspace (none for the fused stencil kernel; coefficients and
// activations for the two-pass one; side states and activations for a
// face-state network); plus a fixed part.  Once the bucket exists, the sum of
// its actual allocations replaces the estimate.
size_t slot_bytes(const fv_request& r, const fv_net* net) {
  const size_t cells = (size_t)r.nx * r.ny;
  const size_t C = r.eq == FV_EQ_SWE ? 3 : 4;
  size_t b = 2 * C * 4 * cells + sizeof(fvk::Ctrl) + (C + 1) * (256 + 1) * sizeof(double);
  if (r.learned) {
    const bool face = net && net->n.kind == snk::NET_FACE;
    const bool fused = !face && fvk::learned_fused_supported(r.nx, r.ny);
    if (face) b += cells * (12 * 4 + 3 * 64);
    else if (!fused) b += cells * (36 * 4 + 3 * 64);
    b += sizeof(float);
  }
  return b;
}

constexpr size_t BUCKET_FIXED_BYTES = 4096;

__global__ void park_kernel(fvk::Ctrl* c, int B) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  c[b].done = 1u;
  c[b].health = 0u;
  c[b].step_end = 0;
}

// Stop stepping one member (a slot whose request left it unfinished).
__global__ void park_member_kernel(fvk::Ctrl* ctrl, int b) {
  ctrl[b].done = 1u;
  ctrl[b].step_end = 0;
}

__global__ void reset_member_kernel(fvk::Ctrl* ctrl, int b, long long step_end) {
  fvk::Ctrl* c = ctrl + b;
  c->t = 0.0;
  c->dt = 0.0;
  c->t_end = 0.0;
  c->amax_last = 0.0;
  c->step = 0;
  c->amax_bits = 0u;
  c->blocks_done = 0u;
  c->health = 0u;
  c->done = 0u;
  c->exhausted = 0u;
  c->step_end = step_end;
}

}  // namespace

struct fv_server {
  size_t budget = 0, used = 0;    // bytes held by buckets
  int max_slots = 1;
  int active = 0;                 // admitted requests not yet finished
  const fv_net* net = nullptr;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Req*> pending;
  std::vector<Bucket*> buckets;
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
  if (q->bucket) {
    q->bucket->slot[q->slot] = nullptr;
    q->bucket->used -= 1;
    q->bucket = nullptr;
  }
  S->active -= 1;
}

void bucket_free(Bucket* b) {
  if (b->st) fv_destroy_state(b->st);
  if (b->host_ctrl) cudaFreeHost(b->host_ctrl);
  if (b->ev) cudaEventDestroy(b->ev);
  delete b;
}

// Create a bucket (worker thread, no lock held): a state of `cap` parked
// members, its learned workspace, pinned control-block mirror and event.
int bucket_create(fv_server* S, const fv_request& r, int cap, Bucket** out) {
  Bucket* b = new Bucket();
  b->key = key_of(r);
  b->cap = cap;
  b->slot.assign(b->cap, nullptr);
  const int C = r.eq == FV_EQ_SWE ? 3 : 4;
  std::vector<float> zero((size_t)b->cap * C * r.nx * r.ny, 1.f);   // placeholder state (h, rho = 1)
  for (size_t i = 0; i < zero.size(); ++i) {
    const size_t v = (i / ((size_t)r.nx * r.ny)) % C;
    if (v == 1 || v == 2) zero[i] = 0.f;                             // at rest (Euler: E = 1)
  }
  fv_grid g{r.nx, r.ny, b->cap, 1.0, 1.0};
  int rc;
  if (r.eq == FV_EQ_SWE) {
    fv_swe_params p{9.81, r.cfl, FV_DT_ADAPTIVE, 0.0};
    rc = swe_init(&g, &p, zero.data(), FV_HOST, nullptr, &b->st);
  } else {
    fv_euler_params p{1.4, r.cfl, FV_DT_ADAPTIVE, 0.0};
    rc = euler_init(&g, &p, zero.data(), FV_HOST, nullptr, &b->st);
  }
  if (rc == FV_OK && r.learned) {
    std::vector<double> h(b->cap, 0.0);
    rc = fvs::learned_set_hmin_values(b->st, h.data());
    if (rc == FV_OK) rc = fvs::learned_prepare(b->st, S->net);
  }
  if (rc == FV_OK && cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming) != cudaSuccess) rc = FV_ECUDA;
  if (rc == FV_OK &&
      cudaHostAlloc(reinterpret_cast<void**>(&b->host_ctrl), sizeof(fvk::Ctrl) * b->cap, cudaHostAllocDefault) !=
          cudaSuccess)
    rc = FV_ECUDA;
  if (rc == FV_OK) {
    park_kernel<<<(b->cap + 127) / 128, 128, 0, b->st->stream>>>(b->st->ctrl, b->cap);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(b->st->stream) != cudaSuccess) rc = FV_ECUDA;
  }
  if (rc != FV_OK) {
    bucket_free(b);
    return rc;
  }
  b->bytes = (size_t)fvs::state_device_bytes(b->st);
  *out = b;
  return FV_OK;
}

// Initialise request q in its slot (bucket idle): initial state, control
// block with its step limit, time step from its own wave speeds, and the
// learned positivity threshold.  Stream-ordered before the bucket's next chunk.
int start_member(Bucket* b, Req* q) {
  fv_state* s = b->st;
  const size_t n = (size_t)s->g.member();
  cudaStream_t st = s->stream;
  if (cudaMemcpyAsync(s->qA + (size_t)q->slot * n, q->q0.data(), n * sizeof(float), cudaMemcpyHostToDevice, st) !=
      cudaSuccess)
    return FV_ECUDA;
  reset_member_kernel<<<1, 1, 0, st>>>(s->ctrl, q->slot, q->r.nsteps);
  if (cudaGetLastError() != cudaSuccess) return FV_ECUDA;
  if (fvk::launch_wavespeed_init(s->g, s->qA, s->ctrl, s->dp, st, q->slot) != cudaSuccess) return FV_ECUDA;
  if (q->r.learned) {
    // h_min = 1e-3 x the member's mean depth (as a standalone learned state)
    double sum = 0.0;
    const size_t plane = (size_t)s->g.plane();
    for (size_t i = 0; i < plane; ++i) sum += q->q0[i];
    q->hmin = (float)(1e-3 * sum / (double)plane);
    float* hm = fvs::learned_hmin_ptr(s);
    if (!hm || cudaMemcpyAsync(hm + q->slot, &q->hmin, sizeof(float), cudaMemcpyHostToDevice, st) != cudaSuccess)
      return FV_ECUDA;
  }
  q->started = true;
  return FV_OK;
}

Bucket* find_bucket(fv_server* S, const Key& k, bool need_free) {
  for (Bucket* b : S->buckets)
    if (b->key == k && (!need_free || b->used < b->cap)) return b;
  return nullptr;
}

// Release empty, idle buckets until `need` more bytes fit the budget.
void release_empty(fv_server* S, size_t need) {
  for (size_t i = 0; i < S->buckets.size() && S->used + need > S->budget;) {
    Bucket* b = S->buckets[i];
    if (b->used == 0 && !b->in_flight) {
      S->used -= b->bytes;
      bucket_free(b);
      S->buckets.erase(S->buckets.begin() + i);
    } else {
      ++i;
    }
  }
}

void worker_loop(fv_server* S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lock(S->mu);
  while (!S->stop) {
    bool progressed = false;
    // admission: arrival order, while a slot is free and the memory fits
    while (!S->pending.empty() && S->active < S->max_slots) {
      Req* q = S->pending.front();
      const Key k = key_of(q->r);
      Bucket* b = find_bucket(S, k, true);
      if (!b) {
        // a new bucket: as many slots as its shape takes, within the budget left
        const size_t per = slot_bytes(q->r, S->net);
        int cap = capacity_for(q->r);
        release_empty(S, BUCKET_FIXED_BYTES + per * cap);
        const size_t room = S->budget > S->used + BUCKET_FIXED_BYTES ? S->budget - S->used - BUCKET_FIXED_BYTES : 0;
        if ((size_t)cap * per > room) cap = (int)(room / per);
        if (cap < 1) break;                     // wait for memory (the head keeps its place)
        lock.unlock();
        int rc = bucket_create(S, q->r, cap, &b);
        lock.lock();
        if (rc != FV_OK) {
          S->pending.pop_front();
          S->active += 1;
          finish(S, q, rc);
          progressed = true;
          continue;
        }
        S->used += b->bytes;
        S->buckets.push_back(b);
      }
      S->pending.pop_front();
      int slot = 0;
      while (b->slot[slot]) ++slot;
      b->slot[slot] = q;
      b->used += 1;
      q->bucket = b;
      q->slot = slot;
      q->started = false;
      q->t_admit = now_s();
      S->active += 1;
      progressed = true;
    }
    for (Bucket* b : S->buckets) {
      if (b->in_flight) {
        const cudaError_t e = cudaEventQuery(b->ev);
        if (e == cudaErrorNotReady) continue;
        b->in_flight = false;
        progressed = true;
        for (int i = 0; i < b->cap; ++i) {
          Req* q = b->slot[i];
          if (!q || !q->started) continue;
          if (e != cudaSuccess) {
            finish(S, q, FV_ECUDA);
            continue;
          }
          const fvk::Ctrl& c = b->host_ctrl[i];
          if (c.health) {
            // the slot leaves the chunks until a new request starts in it
            park_member_kernel<<<1, 1, 0, b->st->stream>>>(b->st->ctrl, i);
            if (q->r.learned) {
              // the plain step is the learned step's fallback: rerun the
              // request with MUSCL-minmod from its initial state, first in line
              q->bucket->slot[q->slot] = nullptr;
              q->bucket->used -= 1;
              q->bucket = nullptr;
              q->r.learned = 0;
              q->fell_back = true;
              S->active -= 1;
              ++S->fallbacks;
              S->pending.push_front(q);
            } else {
              finish(S, q, FV_EUNSTABLE);
            }
            continue;
          }
          if (c.step >= q->r.nsteps) {
            q->result.resize(q->q0.size());
            const size_t n = (size_t)b->st->g.member();
            lock.unlock();
            const cudaError_t ce = cudaMemcpyAsync(q->result.data(), b->st->qA + (size_t)i * n, n * sizeof(float),
                                                   cudaMemcpyDeviceToHost, b->st->stream);
            const cudaError_t se = ce == cudaSuccess ? cudaStreamSynchronize(b->st->stream) : ce;
            lock.lock();
            finish(S, q, se == cudaSuccess ? FV_OK : FV_ECUDA);
          }
        }
      }
      if (b->in_flight || b->used == 0) continue;
      // idle bucket with members: start the newcomers, then the next chunk
      lock.unlock();
      int rc = FV_OK;
      std::vector<Req*> failed;
      for (int i = 0; i < b->cap; ++i) {
        Req* q = b->slot[i];
        if (q && !q->started && start_member(b, q) != FV_OK) failed.push_back(q);
      }
      rc = fv_enqueue_steps(b->st, b->key.learned ? S->net : nullptr, CHUNK);
      if (rc == FV_OK &&
          cudaMemcpyAsync(b->host_ctrl, b->st->ctrl, sizeof(fvk::Ctrl) * b->cap, cudaMemcpyDeviceToHost,
                          b->st->stream) != cudaSuccess)
        rc = FV_ECUDA;
      if (rc == FV_OK && cudaEventRecord(b->ev, b->st->stream) != cudaSuccess) rc = FV_ECUDA;
      lock.lock();
      for (Req* q : failed) finish(S, q, FV_ECUDA);
      if (rc != FV_OK) {
        for (int i = 0; i < b->cap; ++i)
          if (b->slot[i]) finish(S, b->slot[i], rc);
        continue;
      }
      b->in_flight = true;
      progressed = true;
    }
    if (progressed) S->cv.notify_all();
    else S->cv.wait_for(lock, std::chrono::microseconds(200));
  }
  // shut down: fail whatever is still admitted, release every bucket
  for (Bucket* b : S->buckets) {
    for (int i = 0; i < b->cap; ++i)
      if (b->slot[i]) finish(S, b->slot[i], FV_ETIMEOUT);
    bucket_free(b);
  }
  S->buckets.clear();
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
  if (BUCKET_FIXED_BYTES + slot_bytes(*r, S->net) > S->budget)
    return fvh::fail(FV_EBUSY, "request needs more device memory than the server budget");
  Req* q = new Req();
  q->r = *r;
  const size_t n = (size_t)r->nx * r->ny * (r->eq == FV_EQ_SWE ? 3 : 4);
  q->q0.assign(r->q0, r->q0 + n);
  q->r.q0 = nullptr;
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
  if (active) *active = S->active;
  if (pending) *pending = (int)S->pending.size();
  if (used_bytes) *used_bytes = S->used;
  if (fallbacks) *fallbacks = S->fallbacks;
  return FV_OK;
}
