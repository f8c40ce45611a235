// Request server: continuous batching of ordering requests on one GPU.
//
// Every slot is a host worker with its own non-blocking stream.  A free slot
// admits the oldest queued requests that fit the memory budget (by estimate)
// and the batch limits, copies their patterns to the device and orders them
// as one batch; requests arriving meanwhile are admitted by the next free
// slot and run concurrently with the batches already on the device.  The
// batch path makes every per-problem decision from the problem alone, so a
// request's permutation does not depend on the batch it ran in.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "vmo_internal.cuh"

namespace vmo {

vmo_status batch_order(const vmo_csr* mats, int32_t count, const float* coords, const vmo_params* p, int32_t sbd,
                       int32_t* perm, cudaStream_t s);
vmo_status ensure_device_public();
vmo_status check_params_public(const vmo_params* p);

namespace {

struct Req {
  int32_t n = 0;
  int64_t nnz = 0;
  const int32_t* rowptr = nullptr;
  const int32_t* colidx = nullptr;
  int32_t* out = nullptr;
  bool cancel_requested = false;  // cancelled while running: becomes terminal when its batch ends
  vmo_request_info info{};
};

}  // namespace

struct ServerImpl {
  vmo_server_config cfg{};
  int device = 0;
  std::chrono::steady_clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, Req> reqs;
  uint64_t next_id = 1;
  bool stopping = false;
  int64_t in_use = 0, peak = 0, batches = 0;
  int64_t submitted = 0, completed = 0, failed = 0, cancelled = 0, running = 0, nnz_done = 0;
  std::vector<std::thread> workers;

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  void worker(int slot);
  void run_batch(int slot, const std::vector<uint64_t>& ids, cudaStream_t s, int32_t*& stage, size_t& stage_cap);
};

namespace {

vmo_status validate_host_csr(int32_t n, const int32_t* rowptr, const int32_t* colidx, int64_t* nnz) {
  if (n < 0) return invalid("server: negative n");
  if (!rowptr) return invalid("server: rowptr is null");
  if (rowptr[0] != 0) return invalid("server: rowptr[0] != 0");
  for (int32_t i = 0; i < n; ++i)
    if (rowptr[i + 1] < rowptr[i]) return invalid("server: rowptr decreases at row " + std::to_string(i));
  const int64_t z = rowptr[n];
  if (z > 0 && !colidx) return invalid("server: colidx is null");
  for (int64_t t = 0; t < z; ++t)
    if (colidx[t] < 0 || colidx[t] >= n) return invalid("server: column index out of range at entry " + std::to_string(t));
  *nnz = z;
  return VMO_OK;
}

}  // namespace

void ServerImpl::worker(int slot) {
  cudaSetDevice(device);
  cudaStream_t s = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
    (void)cudaGetLastError();
    s = nullptr;
  }
  DevArrayStreamScope scope(s);
  int32_t* stage = nullptr;  // pinned staging of the permutations
  size_t stage_cap = 0;
  for (;;) {
    std::vector<uint64_t> ids;
    {
      std::unique_lock<std::mutex> lk(mu);
      for (;;) {
        if (stopping && queue.empty()) break;
        if (!queue.empty() && s) {
          const int32_t look = (int32_t)std::min<size_t>(queue.size(), (size_t)cfg.max_batch);
          std::vector<int64_t> b(look), z(look);
          for (int32_t i = 0; i < look; ++i) {
            const Req& r = reqs[queue[i]];
            b[i] = r.info.bytes;
            z[i] = r.nnz;
          }
          const int32_t take = vmo_server_plan(b.data(), z.data(), look, cfg.budget_bytes - in_use, cfg.max_batch,
                                               cfg.max_batch_nnz);
          if (take > 0) {
            const int64_t seq = batches++;
            const double t = now();
            for (int32_t i = 0; i < take; ++i) {
              Req& r = reqs[queue.front()];
              ids.push_back(queue.front());
              queue.pop_front();
              r.info.state = VMO_REQ_RUNNING;
              r.info.t_admit = t;
              r.info.batch = seq;
              r.info.batch_size = take;
              r.info.slot = slot;
              in_use += r.info.bytes;
            }
            running += take;
            peak = std::max(peak, in_use);
            break;
          }
        }
        cv_work.wait(lk);
      }
    }
    if (ids.empty()) break;
    run_batch(slot, ids, s, stage, stage_cap);
  }
  if (stage) cudaFreeHost(stage);
  if (s) {
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }
}

void ServerImpl::run_batch(int slot, const std::vector<uint64_t>& ids, cudaStream_t s, int32_t*& stage,
                           size_t& stage_cap) {
  (void)slot;
  // the records stay where they are while running (an unordered_map keeps
  // its elements in place; release refuses records that are not terminal,
  // and cancel only sets a flag)
  std::vector<Req*> rs;
  {
    std::lock_guard<std::mutex> lk(mu);
    for (uint64_t id : ids) rs.push_back(&reqs[id]);
  }
  const int count = (int)rs.size();
  int64_t rows = 0, ents = 0;
  for (Req* r : rs) {
    rows += r->n + 1;
    ents += r->nnz;
  }
  int64_t nperm = 0;
  for (Req* r : rs) nperm += r->n;
  vmo_status st = VMO_OK;
  int32_t* dbuf = nullptr;
  const size_t words = (size_t)(rows + ents + nperm);
  cudaError_t e = cudaMallocAsync((void**)&dbuf, std::max<size_t>(words, 4) * sizeof(int32_t), s);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    st = VMO_ERR_OOM;
    dbuf = nullptr;
  } else {
    g_device_allocs.fetch_add(1, std::memory_order_relaxed);
  }
  if (st == VMO_OK && (size_t)nperm > stage_cap) {
    if (stage) cudaFreeHost(stage);
    stage = nullptr;
    stage_cap = 0;
    if (cudaMallocHost((void**)&stage, (size_t)nperm * sizeof(int32_t)) != cudaSuccess) {
      (void)cudaGetLastError();
      stage = nullptr;
      st = VMO_ERR_OOM;
    } else {
      stage_cap = (size_t)nperm;
    }
  }
  if (st == VMO_OK) {
    std::vector<vmo_csr> mats(count);
    int32_t* p = dbuf;
    for (int i = 0; i < count; ++i) {
      Req* r = rs[i];
      int32_t* rp = p;
      p += r->n + 1;
      int32_t* ci = p;
      p += r->nnz;
      if (cudaMemcpyAsync(rp, r->rowptr, (size_t)(r->n + 1) * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
          (r->nnz > 0 && cudaMemcpyAsync(ci, r->colidx, (size_t)r->nnz * 4, cudaMemcpyHostToDevice, s) != cudaSuccess)) {
        (void)cudaGetLastError();
        st = VMO_ERR_CUDA;
        break;
      }
      mats[i] = vmo_csr{r->n, r->n, r->nnz, rp, ci};
    }
    int32_t* dperm = p;
    if (st == VMO_OK) st = batch_order(mats.data(), count, nullptr, &cfg.params, cfg.sbd, dperm, s);
    if (st == VMO_OK && nperm > 0) {
      if (cudaMemcpyAsync(stage, dperm, (size_t)nperm * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess) {
        (void)cudaGetLastError();
        st = VMO_ERR_CUDA;
      }
    }
  }
  if (dbuf) cudaFreeAsync(dbuf, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) {
    (void)cudaGetLastError();
    if (st == VMO_OK) st = VMO_ERR_CUDA;
  }
  {
    std::lock_guard<std::mutex> lk(mu);
    const double t = now();
    int64_t off = 0;
    for (Req* r : rs) {
      if (r->cancel_requested) {
        // cancelled while running: its inputs are no longer read, nothing is written
        r->info.state = VMO_REQ_CANCELLED;
        ++cancelled;
      } else if (st == VMO_OK) {
        if (r->n > 0) memcpy(r->out, stage + off, (size_t)r->n * 4);
        r->info.state = VMO_REQ_DONE;
        ++completed;
        nnz_done += r->nnz;
      } else {
        r->info.state = VMO_REQ_FAILED;
        r->info.status = st;
        ++failed;
      }
      r->info.t_done = t;
      off += r->n;
      in_use -= r->info.bytes;
      --running;
    }
  }
  cv_done.notify_all();
  cv_work.notify_all();
}

}  // namespace vmo

using namespace vmo;

struct vmo_server_s {
  ServerImpl impl;
};

extern "C" {

void vmo_server_default_config(vmo_server_config* cfg) {
  if (!cfg) return;
  memset(cfg, 0, sizeof(*cfg));
  vmo_default_params(&cfg->params);
  cfg->sbd = 0;
  cfg->slots = 4;
  cfg->max_batch = 256;
  cfg->max_batch_nnz = 8000000;
  cfg->budget_bytes = 0;
}

int64_t vmo_server_estimate_bytes(int64_t n, int64_t nnz) {
  return 512 * std::max<int64_t>(n, 0) + 64 * std::max<int64_t>(nnz, 0) + (int64_t(1) << 20);
}

int32_t vmo_server_plan(const int64_t* bytes, const int64_t* nnz, int32_t count, int64_t budget_free,
                        int32_t max_batch, int64_t max_batch_nnz) {
  if (!bytes || !nnz || count <= 0 || max_batch <= 0) return 0;
  int64_t b = 0, z = 0;
  int32_t take = 0;
  for (int32_t i = 0; i < count && take < max_batch; ++i) {
    if (b + bytes[i] > budget_free) break;
    if (take > 0 && z + nnz[i] > max_batch_nnz) break;
    b += bytes[i];
    z += nnz[i];
    ++take;
  }
  return take;
}

vmo_status vmo_server_create(const vmo_server_config* cfg, vmo_server* out) {
  if (!cfg || !out) return invalid("server: null argument");
  *out = nullptr;
  VMO_TRY(ensure_device_public());
  VMO_TRY(check_params_public(&cfg->params));
  if (cfg->slots < 1 || cfg->slots > 64) return invalid("server: slots must be 1..64");
  if (cfg->max_batch < 1) return invalid("server: max_batch must be >= 1");
  if (cfg->max_batch_nnz < 1) return invalid("server: max_batch_nnz must be >= 1");
  if (cfg->budget_bytes < 0) return invalid("server: negative budget");
  if (cfg->sbd != 0 && cfg->sbd != 1) return invalid("server: sbd must be 0 or 1");
  auto* srv = new vmo_server_s();
  ServerImpl& S = srv->impl;
  S.cfg = *cfg;
  S.t0 = std::chrono::steady_clock::now();
  cudaGetDevice(&S.device);
  if (S.cfg.budget_bytes == 0) {
    size_t fr = 0, tot = 0;
    cudaError_t e = cudaMemGetInfo(&fr, &tot);
    if (e != cudaSuccess) {
      delete srv;
      return cuda_fail(e, "cudaMemGetInfo", __FILE__, __LINE__);
    }
    S.cfg.budget_bytes = (int64_t)(fr / 2);
  }
  for (int i = 0; i < S.cfg.slots; ++i) S.workers.emplace_back([&S, i] { S.worker(i); });
  *out = srv;
  return VMO_OK;
}

vmo_status vmo_server_submit(vmo_server srv, int32_t n, const int32_t* rowptr, const int32_t* colidx,
                             int32_t* perm_out, uint64_t* id) {
  if (!srv || !id) return invalid("server: null argument");
  ServerImpl& S = srv->impl;
  int64_t nnz = 0;
  VMO_TRY(validate_host_csr(n, rowptr, colidx, &nnz));
  if (n > 0 && !perm_out) return invalid("server: perm_out is null");
  const int64_t bytes = vmo_server_estimate_bytes(n, nnz);
  if (bytes > S.cfg.budget_bytes) {
    set_error("server: request needs about " + std::to_string(bytes) + " bytes, over the budget of " +
              std::to_string(S.cfg.budget_bytes));
    return VMO_ERR_BUDGET;
  }
  {
    std::lock_guard<std::mutex> lk(S.mu);
    if (S.stopping) return invalid("server: shutting down");
    const uint64_t rid = S.next_id++;
    Req& r = S.reqs[rid];
    r.n = n;
    r.nnz = nnz;
    r.rowptr = rowptr;
    r.colidx = colidx;
    r.out = perm_out;
    r.info.state = VMO_REQ_QUEUED;
    r.info.status = VMO_OK;
    r.info.n = n;
    r.info.nnz = nnz;
    r.info.bytes = bytes;
    r.info.t_submit = S.now();
    r.info.batch = -1;
    r.info.slot = -1;
    ++S.submitted;
    *id = rid;
    if (n == 0) {  // nothing to order
      r.info.state = VMO_REQ_DONE;
      r.info.t_admit = r.info.t_done = r.info.t_submit;
      ++S.completed;
    } else {
      S.queue.push_back(rid);
    }
  }
  S.cv_work.notify_one();
  if (n == 0) S.cv_done.notify_all();
  return VMO_OK;
}

vmo_status vmo_server_poll(vmo_server srv, uint64_t id, vmo_request_info* info) {
  if (!srv || !info) return invalid("server: null argument");
  ServerImpl& S = srv->impl;
  std::lock_guard<std::mutex> lk(S.mu);
  auto it = S.reqs.find(id);
  if (it == S.reqs.end()) return invalid("server: unknown request id");
  *info = it->second.info;
  return VMO_OK;
}

vmo_status vmo_server_wait(vmo_server srv, uint64_t id, double timeout_s, vmo_request_info* info) {
  if (!srv) return invalid("server: null argument");
  ServerImpl& S = srv->impl;
  std::unique_lock<std::mutex> lk(S.mu);
  if (S.reqs.find(id) == S.reqs.end()) return invalid("server: unknown request id");
  // the record is looked up again after every wake-up: the mutex is released
  // while waiting, and another thread may insert (rehash) or release it
  auto terminal = [&] {
    auto it = S.reqs.find(id);
    return it == S.reqs.end() || it->second.info.state >= VMO_REQ_DONE;
  };
  bool ok = true;
  if (timeout_s < 0) {
    S.cv_done.wait(lk, terminal);
  } else {
    ok = S.cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), terminal);
  }
  auto it = S.reqs.find(id);
  if (it == S.reqs.end()) return invalid("server: request released while waiting");
  if (info) *info = it->second.info;
  if (!ok) {
    set_error("server: wait timed out");
    return VMO_ERR_TIMEOUT;
  }
  return VMO_OK;
}

vmo_status vmo_server_cancel(vmo_server srv, uint64_t id) {
  if (!srv) return invalid("server: null argument");
  ServerImpl& S = srv->impl;
  {
    std::lock_guard<std::mutex> lk(S.mu);
    auto it = S.reqs.find(id);
    if (it == S.reqs.end()) return invalid("server: unknown request id");
    Req& r = it->second;
    if (r.info.state == VMO_REQ_QUEUED) {
      S.queue.erase(std::find(S.queue.begin(), S.queue.end(), id));
      r.info.state = VMO_REQ_CANCELLED;
      r.info.t_done = S.now();
      ++S.cancelled;
    } else if (r.info.state == VMO_REQ_RUNNING) {
      // the batch may still read the request's host arrays: it stays running
      // and turns cancelled (nothing written) when the batch ends
      r.cancel_requested = true;
    }
  }
  S.cv_done.notify_all();
  S.cv_work.notify_all();
  return VMO_OK;
}

vmo_status vmo_server_release(vmo_server srv, uint64_t id) {
  if (!srv) return invalid("server: null argument");
  ServerImpl& S = srv->impl;
  {
    std::lock_guard<std::mutex> lk(S.mu);
    auto it = S.reqs.find(id);
    if (it == S.reqs.end()) return invalid("server: unknown request id");
    if (it->second.info.state < VMO_REQ_DONE) return invalid("server: request is not terminal");
    S.reqs.erase(it);
  }
  S.cv_done.notify_all();
  return VMO_OK;
}

vmo_status vmo_server_get_stats(vmo_server srv, vmo_server_stats* out) {
  if (!srv || !out) return invalid("server: null argument");
  ServerImpl& S = srv->impl;
  memset(out, 0, sizeof(*out));
  {
    std::lock_guard<std::mutex> lk(S.mu);
    out->submitted = S.submitted;
    out->completed = S.completed;
    out->failed = S.failed;
    out->cancelled = S.cancelled;
    out->queued = (int64_t)S.queue.size();
    out->running = S.running;
    out->batches = S.batches;
    out->nnz_completed = S.nnz_done;
    out->budget_bytes = S.cfg.budget_bytes;
    out->bytes_in_use = S.in_use;
    out->bytes_peak = S.peak;
  }
  cudaMemPool_t pool;
  uint64_t hi = 0;
  if (cudaDeviceGetDefaultMemPool(&pool, S.device) == cudaSuccess &&
      cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &hi) == cudaSuccess)
    out->pool_peak_bytes = (int64_t)hi;
  else
    (void)cudaGetLastError();
  return VMO_OK;
}

void vmo_server_destroy(vmo_server srv) {
  if (!srv) return;
  ServerImpl& S = srv->impl;
  {
    std::lock_guard<std::mutex> lk(S.mu);
    S.stopping = true;
    const double t = S.now();
    for (uint64_t id : S.queue) {
      Req& r = S.reqs[id];
      r.info.state = VMO_REQ_CANCELLED;
      r.info.t_done = t;
      ++S.cancelled;
    }
    S.queue.clear();
  }
  S.cv_work.notify_all();
  S.cv_done.notify_all();
  for (auto& w : S.workers) w.join();
  delete srv;
}

}  // extern "C"
