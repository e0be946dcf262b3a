// Batched applies and the serving runtime (no counterpart in the paper; they run many independent
// mobility products, each exactly the product of dpstokes_apply, concurrently on one GPU).
//
// dpstokes_apply_batch: every request's pipeline is enqueued on one of a pool of library-owned
// streams (requests that share a plan go to the same stream, in order), forked from and joined
// back to the caller's stream with events.  Concurrent small systems fill the GPU that a single
// small system leaves idle.  Nothing synchronises the host and nothing allocates, so a batch can
// be captured into a CUDA graph and replayed.
//
// dps server: a worker thread admits queued requests to a fixed number of slots (streams) as
// slots and device memory free up, oldest first among those whose plan is available; plans are
// cached by their full parameter key (one plan per key), used by one request at a time, and
// evicted least-recently-used when the memory budget would be exceeded.  Each request copies its host inputs in, runs the product and copies the
// outputs back on its slot's stream, so requests that arrive while others run overlap with them.
#include <string.h>
#include <time.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "dps_internal.cuh"

namespace dps {
namespace {

// ---------------------------------------------------------------------------------------------
// stream pool of the batched apply (one per device, created on first use)
// ---------------------------------------------------------------------------------------------
constexpr int kBatchStreams = 8;
constexpr size_t kAdmitWindow = 64;  // queued requests the server's admission looks at
constexpr int kMaxDevices = 64;

struct StreamPool {
  std::mutex enqueue;  // one batch at a time records and waits on the pool's fork/join events
  bool ready = false;
  cudaStream_t s[kBatchStreams];
  cudaEvent_t fork;
  cudaEvent_t join[kBatchStreams];
};
std::mutex g_pool_mutex;
StreamPool g_pool[kMaxDevices];

dps_status pool_for_device(StreamPool** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DPS_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_pool_mutex);
  StreamPool& p = g_pool[dev];
  if (!p.ready) {
    for (int i = 0; i < kBatchStreams; ++i) {
      if (cudaStreamCreateWithFlags(&p.s[i], cudaStreamNonBlocking) != cudaSuccess) return DPS_ERR_CUDA;
      if (cudaEventCreateWithFlags(&p.join[i], cudaEventDisableTiming) != cudaSuccess) return DPS_ERR_CUDA;
    }
    if (cudaEventCreateWithFlags(&p.fork, cudaEventDisableTiming) != cudaSuccess) return DPS_ERR_CUDA;
    p.ready = true;
  }
  *out = &p;
  return DPS_OK;
}

// move the plan's status word to the request's status slot and clear it for the next apply
__global__ void take_status_kernel(int* plan_status, int32_t* out) {
  const int v = *plan_status;
  *plan_status = 0;
  int32_t code = DPS_OK;
  if (v & kStatNonfinite) code = DPS_ERR_NONFINITE;
  else if (v & kStatDomain) code = DPS_ERR_OUT_OF_DOMAIN;
  else if (v & kStatInternal) code = DPS_ERR_CUDA;
  *out = code;
}

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// ---------------------------------------------------------------------------------------------
// server
// ---------------------------------------------------------------------------------------------
struct PlanKey {
  double Lx, Ly, zmin, zmax;
  int32_t mode, nx, ny, nz, m_M, m_D, with_torque, precision;
  double beta_M, beta_D, eta;
  int64_t max_n;
  dps_wall_params walls;
  bool operator==(const PlanKey& o) const { return memcmp(this, &o, sizeof(PlanKey)) == 0; }
};

PlanKey key_of(const dps_serve_request& r) {
  PlanKey k;
  memset(&k, 0, sizeof(k));  // padding takes part in the comparison
  k.Lx = r.Lx; k.Ly = r.Ly; k.zmin = r.zmin; k.zmax = r.zmax;
  k.mode = r.wall_mode; k.nx = r.grid.nx; k.ny = r.grid.ny; k.nz = r.grid.nz;
  k.m_M = r.kp.m_M; k.m_D = r.kp.with_torque ? r.kp.m_D : 0; k.with_torque = r.kp.with_torque;
  k.precision = r.kp.precision; k.beta_M = r.kp.beta_M; k.beta_D = r.kp.with_torque ? r.kp.beta_D : 0.0;
  k.eta = r.kp.eta; k.max_n = r.kp.max_n;
  k.walls = r.walls;
  return k;
}

struct CachedPlan {
  PlanKey key;
  dps_plan_t plan = nullptr;
  int64_t bytes = 0;
  bool in_use = false;
  uint64_t last_use = 0;
};

struct Pending {
  dps_serve_request r;
  int64_t ticket;
  double t_submit;
};

struct Slot {
  cudaStream_t s = nullptr;
  cudaEvent_t done = nullptr;
  int32_t* h_status = nullptr;  // pinned
  bool busy = false;
  int64_t ticket = -1;
  CachedPlan* cp = nullptr;
  double t_submit = 0, t_start = 0;
  // pinned staging of the outputs when the caller's buffers are pageable (a device-to-host copy
  // into pageable memory would block the worker until the product finished); copied into the
  // caller's buffers when the slot retires
  double* h_out = nullptr;
  size_t h_cap = 0;  // doubles
  double* user_U = nullptr;
  double* user_W = nullptr;
  size_t out_bytes = 0;
  bool staged = false;
};

// page-locked (or device-accessible) host memory: copies to it are asynchronous
bool copies_async_to(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeManaged;
}

}  // namespace

struct Server {
  int device = 0;
  int64_t budget = 0, used = 0;
  std::vector<Slot> slots;
  std::vector<CachedPlan*> cache;
  std::deque<Pending> queue;
  std::unordered_map<int64_t, dps_serve_result> done;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::thread worker;
  bool stop = false;
  int64_t next_ticket = 0;
  uint64_t clock = 0;
  int64_t created = 0, evicted = 0, rejected = 0;
  int64_t max_queued = 0;  // 0: unbounded queue

  // plan sizing before creation, following the plan's own allocations: grid, particle records and
  // bins, solve workspace, spectra, staging buffers and tables (an upper bound, plus 1/8)
  static int64_t estimate_bytes(const dps_serve_request& r) {
    const int64_t ts = r.kp.precision == DPS_MIXED ? 4 : 8;
    const int64_t nx = r.grid.nx, ny = r.grid.ny, nz = r.grid.nz;
    const int64_t nkx = nx / 2 + 1, pitch = (nkx + 31) / 32 * 32, K = nkx * ny;
    const int route = r.kp.with_torque;  // record slabs: M, plus D, plus D' for the derivative route
    const int64_t nf = route == DPS_TORQUE_SPECTRAL_CURL ? 6 : 3;
    const int64_t nk = route == DPS_TORQUE_NONE ? 1 : (route == DPS_TORQUE_KERNEL_DERIVATIVE ? 3 : 2);
    const int64_t nmax = std::max<int64_t>(r.kp.max_n, 1);
    const int64_t rec = 4 * (8 + (6 + nk * (2 * (kMaxM + 1) + nz)) * ts / 4 + 3);
    const int64_t nbins = ((nx + kTileX - 1) / kTileX) * ((ny + kTileY - 1) / kTileY);
    const int64_t blocks = std::min<int64_t>(152 * 4, (K + kBvpThreads - 1) / kBvpThreads);
    int64_t b = nf * nz * ny * pitch * 2 * ts;                          // grid
    b += nmax * (rec + 8 + 15 * 8) + 3 * nbins * 4;                      // records, bins, staging
    b += blocks * kBvpThreads * nz * (3 * 16 + 3 * 8 + 2 * ts);          // solve workspace
    b += 3 * nz * K * 2 * ts + 12 * K * 2 * ts;                          // kbuf, kaux
    b += nkx * (ny / 2 + 1) * nz * 4 * 8;                                // factorisation table (FP64)
    // partial sums of the tile-gather interpolation (forces only, or equal supports with the
    // spectral curl): slots of the tiles a support can overlap x fields x particles
    const int64_t ifields = route == DPS_TORQUE_NONE ? 3
                          : (route == DPS_TORQUE_SPECTRAL_CURL && r.kp.m_M == r.kp.m_D ? 6 : 0);
    if (ifields) {
      const int64_t px = r.kp.m_M + 1;
      const int64_t nbx = (nx + kTileX - 1) / kTileX, nby = (ny + kTileY - 1) / kTileY;
      const int64_t sxn = std::min<int64_t>(nbx, (px - 1) / kTileX + 2 + (nx % kTileX ? 1 : 0));
      const int64_t syn = std::min<int64_t>(nby, (px - 1) / kTileY + 2 + (ny % kTileY ? 1 : 0));
      b += sxn * syn * ifields * nmax * ts;
    }
    b += 8 * nz * (nz + 32) * ts + 3 * (nx + ny) * 16 + 16 * nz * 8;     // tables (twiddles: length n + stages <= 2 n)
    return b + b / 8 + (256 << 10);
  }

  CachedPlan* find_free(const PlanKey& k) {
    for (CachedPlan* c : cache)
      if (!c->in_use && c->key == k) return c;
    return nullptr;
  }

  CachedPlan* find_any(const PlanKey& k) {
    for (CachedPlan* c : cache)
      if (c->key == k) return c;
    return nullptr;
  }

  // evict least-recently-used idle plans until `need` more bytes fit; false if they cannot
  bool make_room(int64_t need) {
    while (used + need > budget) {
      CachedPlan* lru = nullptr;
      for (CachedPlan* c : cache)
        if (!c->in_use && (!lru || c->last_use < lru->last_use)) lru = c;
      if (!lru) return false;
      used -= lru->bytes;
      dpstokes_destroy(lru->plan);
      cache.erase(std::find(cache.begin(), cache.end(), lru));
      delete lru;
      ++evicted;
    }
    return true;
  }

  void finish(Slot& sl, dps_status st) {
    if (sl.staged) {  // the slot's copies have completed (its event or a stream synchronisation)
      if (st == DPS_OK) {
        memcpy(sl.user_U, sl.h_out, sl.out_bytes);
        if (sl.user_W) memcpy(sl.user_W, sl.h_out + sl.out_bytes / sizeof(double), sl.out_bytes);
      }
      sl.staged = false;
    }
    dps_serve_result res;
    res.status = st;
    res.t_submit = sl.t_submit;
    res.t_start = sl.t_start;
    res.t_done = now_s();
    done[sl.ticket] = res;
    if (sl.cp) sl.cp->in_use = false;
    sl.cp = nullptr;
    sl.busy = false;
    sl.ticket = -1;
  }

  void fail(const Pending& q, dps_status st) {
    dps_serve_result res;
    res.status = st;
    res.t_submit = q.t_submit;
    res.t_start = res.t_done = now_s();
    done[q.ticket] = res;
  }

  // enqueue one request on a slot: copies in, product, copies out, status, completion event
  dps_status launch(Slot& sl, CachedPlan* cp, const dps_serve_request& r) {
    Plan* p = reinterpret_cast<Plan*>(cp->plan);
    dps_status st = check_apply_args(p, r.n, r.positions, r.forces, r.torques, r.out_vel, r.out_angvel);
    if (st != DPS_OK) return st;
    cudaStream_t s = sl.s;
    double* dpos = p->stage_in;
    double* dF = dpos + 3 * (size_t)p->max_n;
    double* dT = p->g.with_torque ? dF + 3 * (size_t)p->max_n : nullptr;
    double* dU = p->stage_out;
    double* dW = p->g.with_torque ? dU + 3 * (size_t)p->max_n : nullptr;
    const size_t b = 3 * (size_t)r.n * sizeof(double);
    if (r.n > 0) {
      if (cudaMemcpyAsync(dpos, r.positions, b, cudaMemcpyHostToDevice, s) != cudaSuccess) return DPS_ERR_CUDA;
      if (cudaMemcpyAsync(dF, r.forces, b, cudaMemcpyHostToDevice, s) != cudaSuccess) return DPS_ERR_CUDA;
      if (dT && cudaMemcpyAsync(dT, r.torques, b, cudaMemcpyHostToDevice, s) != cudaSuccess) return DPS_ERR_CUDA;
    }
    st = run(p, r.n, dpos, dF, dT, dU, dW, s, 99);
    if (st != DPS_OK) return st;
    if (r.n > 0) {
      double* oU = r.out_vel;
      double* oW = r.out_angvel;
      if (!copies_async_to(r.out_vel) || (dW && !copies_async_to(r.out_angvel))) {
        const size_t need = 6 * (size_t)r.n;  // the slot is idle: nothing uses its staging buffer
        if (sl.h_cap < need) {
          const size_t cap = std::max<size_t>(need, 2 * sl.h_cap);
          if (sl.h_out) cudaFreeHost(sl.h_out);
          sl.h_out = nullptr;
          sl.h_cap = 0;
          if (cudaMallocHost((void**)&sl.h_out, cap * sizeof(double)) != cudaSuccess) return DPS_ERR_OOM;
          sl.h_cap = cap;
        }
        oU = sl.h_out;
        oW = dW ? sl.h_out + 3 * (size_t)r.n : nullptr;
        sl.user_U = r.out_vel;
        sl.user_W = dW ? r.out_angvel : nullptr;
        sl.out_bytes = b;
        sl.staged = true;
      }
      if (cudaMemcpyAsync(oU, dU, b, cudaMemcpyDeviceToHost, s) != cudaSuccess) return DPS_ERR_CUDA;
      if (dW && cudaMemcpyAsync(oW, dW, b, cudaMemcpyDeviceToHost, s) != cudaSuccess) return DPS_ERR_CUDA;
    }
    if (cudaMemcpyAsync(sl.h_status, p->status, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess)
      return DPS_ERR_CUDA;
    if (cudaMemsetAsync(p->status, 0, sizeof(int32_t), s) != cudaSuccess) return DPS_ERR_CUDA;
    if (cudaEventRecord(sl.done, s) != cudaSuccess) return DPS_ERR_CUDA;
    return DPS_OK;
  }

  static dps_status decode(int32_t v) {
    if (v & kStatNonfinite) return DPS_ERR_NONFINITE;
    if (v & kStatDomain) return DPS_ERR_OUT_OF_DOMAIN;
    if (v & kStatInternal) return DPS_ERR_CUDA;
    return DPS_OK;
  }

  void loop() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lock(mu);
    for (;;) {
      bool progress = false;
      // retire finished slots
      for (Slot& sl : slots) {
        if (!sl.busy) continue;
        const cudaError_t q = cudaEventQuery(sl.done);
        if (q == cudaErrorNotReady) continue;
        finish(sl, q == cudaSuccess ? decode(*sl.h_status) : DPS_ERR_CUDA);
        progress = true;
      }
      if (progress) cv_done.notify_all();
      // Admission, while a slot is free, over the oldest kAdmitWindow queued requests: first the
      // oldest whose plan is cached and idle; otherwise the oldest whose key has no plan at all
      // (created now, after evicting idle plans if the budget needs it).  A key never holds two
      // plans, and no request waits behind another one's busy plan.
      while (!queue.empty()) {
        Slot* free_slot = nullptr;
        bool any_busy = false;
        for (Slot& sl : slots) {
          if (sl.busy) any_busy = true;
          else if (!free_slot) free_slot = &sl;
        }
        if (!free_slot) break;
        const size_t window = std::min<size_t>(queue.size(), kAdmitWindow);
        size_t pick = window;
        CachedPlan* cp = nullptr;
        for (size_t i = 0; i < window && !cp; ++i) {
          cp = find_free(key_of(queue[i].r));
          if (cp) pick = i;
        }
        if (!cp) {
          for (size_t i = 0; i < window; ++i)
            if (!find_any(key_of(queue[i].r))) { pick = i; break; }
          if (pick == window) break;  // every candidate's plan is busy: wait for a completion
          Pending q = queue[pick];
          const int64_t need = estimate_bytes(q.r);
          if (need > budget) {  // can never fit
            queue.erase(queue.begin() + pick);
            fail(q, DPS_ERR_OOM);
            cv_done.notify_all();
            continue;
          }
          if (!make_room(need)) {
            if (any_busy) break;  // wait for running requests to release plans
            queue.erase(queue.begin() + pick);
            fail(q, DPS_ERR_OOM);
            cv_done.notify_all();
            continue;
          }
          dps_plan_t plan = nullptr;
          const dps_status st = dpstokes_plan_create_ex(&plan, q.r.Lx, q.r.Ly, q.r.zmin, q.r.zmax, q.r.wall_mode,
                                                        &q.r.grid, &q.r.kp, &q.r.walls);
          if (st != DPS_OK) {
            queue.erase(queue.begin() + pick);
            fail(q, st);
            cv_done.notify_all();
            continue;
          }
          cp = new CachedPlan();
          cp->key = key_of(q.r);
          cp->plan = plan;
          dps_plan_info info;
          dpstokes_plan_info(plan, &info);
          cp->bytes = info.device_bytes;
          used += cp->bytes;
          cache.push_back(cp);
          ++created;
        }
        const Pending q = queue[pick];
        queue.erase(queue.begin() + pick);
        cp->in_use = true;
        cp->last_use = ++clock;
        free_slot->busy = true;
        free_slot->cp = cp;
        free_slot->ticket = q.ticket;
        free_slot->t_submit = q.t_submit;
        free_slot->t_start = now_s();
        const dps_status st = launch(*free_slot, cp, q.r);
        if (st != DPS_OK) {
          cudaStreamSynchronize(free_slot->s);  // nothing of this request may still run
          finish(*free_slot, st);
          cv_done.notify_all();
        }
        progress = true;
      }
      bool busy = false;
      for (Slot& sl : slots) busy = busy || sl.busy;
      if (stop && queue.empty() && !busy) break;
      if (!progress) {
        // poll the running slots; new submissions wake the loop at once
        cv_work.wait_for(lock, std::chrono::microseconds(busy ? 20 : 2000));
      }
    }
  }
};

}  // namespace dps

extern "C" {

dps_status dpstokes_apply_batch(const dps_request* reqs, int32_t count, void* stream) {
  using namespace dps;
  if (count < 0 || (count > 0 && !reqs)) return DPS_ERR_INVALID_ARG;
  for (int32_t i = 0; i < count; ++i) {
    const Plan* p = reinterpret_cast<const Plan*>(reqs[i].plan);
    const dps_status st = check_apply_args(p, reqs[i].n, reqs[i].positions, reqs[i].forces, reqs[i].torques,
                                           reqs[i].out_vel, reqs[i].out_angvel);
    if (st != DPS_OK) return st;
  }
  if (count == 0) return DPS_OK;
  StreamPool* pool = nullptr;
  dps_status st = pool_for_device(&pool);
  if (st != DPS_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  // batches from several host threads enqueue one after another: each one's fork record and waits
  // and its join records and waits must not interleave with another's on the shared events
  std::lock_guard<std::mutex> guard(pool->enqueue);
  // requests of one plan share a stream (they use the plan's buffers in turn)
  std::vector<int> lane(count, -1);
  std::vector<dps_plan_t> owner(kBatchStreams, nullptr);
  int used = 0, rr = 0;
  for (int32_t i = 0; i < count; ++i) {
    for (int32_t j = 0; j < i; ++j)
      if (reqs[j].plan == reqs[i].plan) { lane[i] = lane[j]; break; }
    if (lane[i] < 0) {
      lane[i] = rr;
      rr = (rr + 1) % kBatchStreams;
      used = std::max(used, lane[i] + 1);
    }
  }
  if (cudaEventRecord(pool->fork, s) != cudaSuccess) return DPS_ERR_CUDA;
  for (int l = 0; l < used; ++l)
    if (cudaStreamWaitEvent(pool->s[l], pool->fork, 0) != cudaSuccess) return DPS_ERR_CUDA;
  for (int32_t i = 0; i < count; ++i) {
    const dps_request& r = reqs[i];
    Plan* p = reinterpret_cast<Plan*>(r.plan);
    cudaStream_t ws = pool->s[lane[i]];
    st = run(p, r.n, r.positions, r.forces, r.torques, r.out_vel, r.out_angvel, ws, 99);
    if (st != DPS_OK) return st;
    if (r.status) take_status_kernel<<<1, 1, 0, ws>>>(p->status, r.status);
  }
  for (int l = 0; l < used; ++l) {
    if (cudaEventRecord(pool->join[l], pool->s[l]) != cudaSuccess) return DPS_ERR_CUDA;
    if (cudaStreamWaitEvent(s, pool->join[l], 0) != cudaSuccess) return DPS_ERR_CUDA;
  }
  return cudaGetLastError() == cudaSuccess ? DPS_OK : DPS_ERR_CUDA;
}

dps_status dpstokes_batch_prepare(void) {
  dps::StreamPool* pool = nullptr;
  return dps::pool_for_device(&pool);
}

dps_status dpstokes_server_create(dps_server_t* out, int64_t memory_budget_bytes, int32_t slots) {
  using namespace dps;
  if (!out) return DPS_ERR_INVALID_ARG;
  *out = nullptr;
  if (memory_budget_bytes <= 0 || slots < 1 || slots > 64) return DPS_ERR_INVALID_ARG;
  Server* sv = new Server();
  if (cudaGetDevice(&sv->device) != cudaSuccess) { delete sv; return DPS_ERR_CUDA; }
  sv->budget = memory_budget_bytes;
  sv->slots.resize(slots);
  for (Slot& sl : sv->slots) {
    if (cudaStreamCreateWithFlags(&sl.s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess ||
        cudaMallocHost((void**)&sl.h_status, sizeof(int32_t)) != cudaSuccess) {
      for (Slot& t : sv->slots) {
        if (t.s) cudaStreamDestroy(t.s);
        if (t.done) cudaEventDestroy(t.done);
        if (t.h_status) cudaFreeHost(t.h_status);
      }
      delete sv;
      return DPS_ERR_CUDA;
    }
  }
  sv->worker = std::thread([sv] { sv->loop(); });
  *out = reinterpret_cast<dps_server_t>(sv);
  return DPS_OK;
}

dps_status dpstokes_server_submit(dps_server_t server, const dps_serve_request* req, int64_t* ticket) {
  using namespace dps;
  Server* sv = reinterpret_cast<Server*>(server);
  if (!sv || !req || !ticket) return DPS_ERR_INVALID_ARG;
  if (req->n < 0 || req->n > req->kp.max_n) return DPS_ERR_INVALID_ARG;
  const double t_submit = now_s();
  {
    std::lock_guard<std::mutex> lock(sv->mu);
    if (sv->stop) return DPS_ERR_INVALID_ARG;
    if (sv->max_queued > 0 && (int64_t)sv->queue.size() >= sv->max_queued) {
      ++sv->rejected;
      return DPS_ERR_BUSY;
    }
    Pending q;
    q.r = *req;
    q.ticket = sv->next_ticket++;
    q.t_submit = t_submit;
    sv->queue.push_back(q);
    *ticket = q.ticket;
  }
  sv->cv_work.notify_one();
  return DPS_OK;
}

dps_status dpstokes_server_wait(dps_server_t server, int64_t ticket, double timeout_s, dps_serve_result* result) {
  using namespace dps;
  Server* sv = reinterpret_cast<Server*>(server);
  if (!sv || !result || ticket < 0) return DPS_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lock(sv->mu);
  if (ticket >= sv->next_ticket) return DPS_ERR_INVALID_ARG;
  const auto until = std::chrono::steady_clock::now() + std::chrono::duration<double>(std::max(0.0, timeout_s));
  for (;;) {
    auto it = sv->done.find(ticket);
    if (it != sv->done.end()) {
      *result = it->second;
      sv->done.erase(it);
      return DPS_OK;
    }
    if (sv->cv_done.wait_until(lock, until) == std::cv_status::timeout && sv->done.find(ticket) == sv->done.end())
      return DPS_ERR_TIMEOUT;
  }
}

dps_status dpstokes_server_stats(dps_server_t server, dps_server_stats* out) {
  using namespace dps;
  Server* sv = reinterpret_cast<Server*>(server);
  if (!sv || !out) return DPS_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(sv->mu);
  out->queued = (int64_t)sv->queue.size();
  int running = 0;
  for (const Slot& sl : sv->slots) running += sl.busy ? 1 : 0;
  out->running = running;
  out->plans_resident = (int64_t)sv->cache.size();
  out->plans_created = sv->created;
  out->plans_evicted = sv->evicted;
  out->bytes_resident = sv->used;
  out->rejected = sv->rejected;
  return DPS_OK;
}

dps_status dpstokes_server_set_queue_limit(dps_server_t server, int64_t max_queued) {
  using namespace dps;
  Server* sv = reinterpret_cast<Server*>(server);
  if (!sv || max_queued < 0) return DPS_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(sv->mu);
  sv->max_queued = max_queued;
  return DPS_OK;
}

void dpstokes_server_destroy(dps_server_t server) {
  using namespace dps;
  Server* sv = reinterpret_cast<Server*>(server);
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lock(sv->mu);
    sv->stop = true;
  }
  sv->cv_work.notify_one();
  if (sv->worker.joinable()) sv->worker.join();
  for (Slot& sl : sv->slots) {
    cudaStreamSynchronize(sl.s);
    cudaStreamDestroy(sl.s);
    cudaEventDestroy(sl.done);
    cudaFreeHost(sl.h_status);
    if (sl.h_out) cudaFreeHost(sl.h_out);
  }
  for (CachedPlan* c : sv->cache) {
    dpstokes_destroy(c->plan);
    delete c;
  }
  delete sv;
}

}  // extern "C"
