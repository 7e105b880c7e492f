// Serving loop of libapiccontact: resident simulations, a request queue,
// worker threads that batch ready requests into one batched contact step,
// admission by an HBM budget, and per-request latency.
//
// Each worker owns an apic_ctx and a non-blocking CUDA stream.  A worker
// takes, in FIFO order, every queued request whose simulation has no step in
// flight (and that shares flags and n_iter with the first one it took), up to
// max_batch requests and a scratch estimate that fits the budget, and runs
// them as one apic_contact_step_batched call with the simulations' resident
// arrays as inputs and outputs.  While it waits for its batch, other workers
// take the requests that arrived meanwhile, so batches overlap on the GPU.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <iterator>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <utility>
#include <vector>

#include "../../include/apiccontact.h"
#include "apic_internal.h"

using Clock = std::chrono::steady_clock;

namespace {

// Scratch the pipeline holds per particle of a batch, as an admission
// estimate (sort keys and values, sorted planes, Delta, item tables and the
// grid share; FP32 path).
constexpr size_t kScratchPerParticle = 640;

// Latency samples kept for the percentiles (the most recent ones).
constexpr size_t kMaxLatencySamples = size_t(1) << 20;

apic_status sfail(apic_status code, const char* msg) {
  apic::set_last_error(msg);
  return code;
}

}  // namespace

struct apic_sim {
  apic_server* srv = nullptr;
  int64_t n = 0;
  int32_t n_bodies = 1, n_iter = 0;
  uint32_t flags = 0;  // without APIC_HOST_PTRS
  double h = 0, mu = 0;
  std::vector<double> mu_pair;
  size_t esize = 4;
  double* x = nullptr;
  int32_t* body = nullptr;
  void *v = nullptr, *C = nullptr, *m = nullptr, *nrm = nullptr;
  size_t bytes = 0;
  bool busy = false;   // a step in flight
  int64_t queued = 0;  // steps waiting in the queue
};

namespace {

struct Ticket {
  apic_sim* sim = nullptr;
  double dt = 0;
  Clock::time_point t_submit, t_done;
  int state = 0;  // 0 queued, 1 running, 2 done
  apic_status status = APIC_OK;
  std::string error;  // the failed call's message
};

}  // namespace

struct apic_server {
  int device = 0;
  size_t budget = 0;
  int max_batch = 64;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, Ticket> tickets;
  uint64_t next_ticket = 1;
  std::vector<std::thread> workers;
  std::vector<size_t> worker_scratch;
  bool stop = false;
  int variant = -1;  // launch policy of the workers' contexts
  int graphs = 1;
  size_t resident = 0;
  int64_t open = 0;
  std::unordered_set<apic_sim*> sims;  // open simulations
  // statistics
  std::vector<double> lat_ms;
  int64_t completed = 0, failed = 0, batches = 0, particle_iters = 0, batch_scenes = 0;
};

namespace {

size_t scratch_total(const apic_server* s) {
  size_t t = 0;
  for (size_t b : s->worker_scratch) t += b;
  return t;
}

void worker_main(apic_server* srv, int wid) {
  cudaSetDevice(srv->device);
  apic_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  const bool ok = apic_create(&ctx, srv->device, 0) == APIC_OK &&
                  cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) == cudaSuccess;
  std::vector<uint64_t> batch;
  std::vector<apic_step_args> args;
  int variant = -1, graphs = 1;  // the context's current policy
  for (;;) {
    batch.clear();
    int want_variant, want_graphs;
    {
      std::unique_lock<std::mutex> lk(srv->mu);
      auto runnable = [&] {
        for (uint64_t t : srv->queue)
          if (!srv->tickets[t].sim->busy) return true;
        return false;
      };
      srv->cv_work.wait(lk, [&] { return srv->stop || runnable(); });
      if (srv->stop && !runnable()) break;
      want_variant = srv->variant;
      want_graphs = srv->graphs;
      // Budget left for this batch's scratch beyond what the workers hold.
      size_t room = SIZE_MAX;
      if (srv->budget) {
        const size_t held = srv->resident + scratch_total(srv);
        room = srv->budget > held ? srv->budget - held + srv->worker_scratch[wid] : 0;
      }
      uint32_t flags = 0;
      int32_t n_iter = 0;
      size_t particles = 0;
      for (auto it = srv->queue.begin(); it != srv->queue.end() && (int)batch.size() < srv->max_batch;) {
        Ticket& tk = srv->tickets[*it];
        apic_sim* sm = tk.sim;
        const size_t need = (particles + (size_t)sm->n) * kScratchPerParticle * (sm->esize / 4);
        const bool first = batch.empty();
        if (!sm->busy && (first || (sm->flags == flags && sm->n_iter == n_iter)) && (first || need <= room)) {
          if (first) {
            flags = sm->flags;
            n_iter = sm->n_iter;
          }
          sm->busy = true;
          sm->queued -= 1;
          tk.state = 1;
          particles += (size_t)sm->n;
          batch.push_back(*it);
          it = srv->queue.erase(it);
        } else {
          ++it;
        }
      }
    }
    if (batch.empty()) continue;
    if (ctx && want_variant != variant) {
      apic_set_variant(ctx, want_variant);
      variant = want_variant;
    }
    if (ctx && want_graphs != graphs) {
      apic_set_graphs(ctx, want_graphs);
      graphs = want_graphs;
    }
    args.assign(batch.size(), apic_step_args{});
    double dts[1024];
    {
      std::lock_guard<std::mutex> lk(srv->mu);
      for (size_t i = 0; i < batch.size(); ++i) {
        const Ticket& tk = srv->tickets[batch[i]];
        apic_sim* sm = tk.sim;
        apic_step_args& a = args[i];
        a.n = sm->n;
        a.n_bodies = sm->n_bodies;
        a.n_iter = sm->n_iter;
        a.body = sm->body;
        a.x = sm->x;
        a.v = sm->v;
        a.C = sm->C;
        a.m = sm->m;
        a.nrm = sm->nrm;
        a.v_out = sm->v;  // V_hat replaces the resident velocity state
        a.C_out = sm->C;
        a.h = sm->h;
        a.mu = sm->mu;
        a.mu_pair = sm->mu_pair.empty() ? nullptr : sm->mu_pair.data();
        a.flags = sm->flags;
        dts[i % 1024] = tk.dt;
      }
    }
    const apic_status st = ok ? apic_contact_step_batched(ctx, args.data(), (int32_t)args.size(), stream, nullptr)
                              : APIC_ERR_CUDA;
    std::vector<apic_status> each(args.size(), st);
    std::vector<std::string> why(args.size(), st == APIC_OK ? std::string() : std::string(apic_last_error()));
    if (st == APIC_ERR_INVALID_ARG && args.size() > 1) {
      // Some simulation's data is invalid.  A call that fails that way
      // leaves every scene as it was, so step them one by one: only the
      // offending requests fail.
      for (size_t i = 0; i < args.size(); ++i) {
        each[i] = apic_contact_step_batched(ctx, &args[i], 1, stream, nullptr);
        why[i] = each[i] == APIC_OK ? std::string() : std::string(apic_last_error());
      }
    }
    bool any_ok = false;
    for (apic_status e : each) any_ok = any_ok || e == APIC_OK;
    if (any_ok) {
      for (size_t i = 0; i < args.size(); ++i) {
        const double dt = dts[i % 1024];
        if (each[i] != APIC_OK || dt == 0.0 || args[i].n == 0) continue;
        cudaError_t e = (args[i].flags & APIC_FP64)
                            ? apic::launch_advect<double>(args[i].n, const_cast<double*>(args[i].x),
                                                          static_cast<const double*>(args[i].v), dt, stream)
                            : apic::launch_advect<float>(args[i].n, const_cast<double*>(args[i].x),
                                                         static_cast<const float*>(args[i].v), dt, stream);
        if (e != cudaSuccess) each[i] = APIC_ERR_CUDA;
      }
      if (cudaStreamSynchronize(stream) != cudaSuccess)
        for (apic_status& e : each) e = APIC_ERR_CUDA;
    }
    size_t held = 0;
    if (ctx) apic_scratch_bytes(ctx, &held);
    {
      std::lock_guard<std::mutex> lk(srv->mu);
      const auto now = Clock::now();
      srv->worker_scratch[wid] = held;
      srv->batches += 1;
      srv->batch_scenes += (int64_t)batch.size();
      for (size_t i = 0; i < batch.size(); ++i) {
        Ticket& tk = srv->tickets[batch[i]];
        tk.state = 2;
        tk.status = each[i];
        tk.error = each[i] == APIC_OK ? std::string() : (why[i].empty() ? std::string("CUDA error") : why[i]);
        tk.t_done = now;
        tk.sim->busy = false;
        if (each[i] == APIC_OK) {
          srv->completed += 1;
          srv->particle_iters += tk.sim->n * (int64_t)(tk.sim->n_iter + 1);
          if (srv->lat_ms.size() >= kMaxLatencySamples)  // keep the most recent half
            srv->lat_ms.erase(srv->lat_ms.begin(), srv->lat_ms.begin() + kMaxLatencySamples / 2);
          srv->lat_ms.push_back(std::chrono::duration<double, std::milli>(now - tk.t_submit).count());
        } else {
          srv->failed += 1;
        }
      }
    }
    srv->cv_done.notify_all();
    srv->cv_work.notify_all();
  }
  if (stream) cudaStreamDestroy(stream);
  if (ctx) apic_destroy(ctx);
}

void free_sim_memory(apic_sim* s) {
  cudaFree(s->x);
  cudaFree(s->body);
  cudaFree(s->v);
  cudaFree(s->C);
  cudaFree(s->m);
  cudaFree(s->nrm);
}

// Wait (lock held) until the simulation has nothing queued or in flight.
void wait_idle(apic_server* srv, std::unique_lock<std::mutex>& lk, apic_sim* s) {
  srv->cv_done.wait(lk, [&] { return !s->busy && s->queued == 0; });
}

}  // namespace

extern "C" {

apic_status apic_server_create(apic_server** out, int32_t device, size_t hbm_budget_bytes, int32_t n_workers,
                               int32_t max_batch_scenes) {
  if (!out) return sfail(APIC_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (n_workers < 1 || n_workers > 16) return sfail(APIC_ERR_INVALID_ARG, "n_workers must be in [1, 16]");
  if (max_batch_scenes < 1 || max_batch_scenes > 1024)
    return sfail(APIC_ERR_INVALID_ARG, "max_batch_scenes must be in [1, 1024]");
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count)
    return sfail(APIC_ERR_INVALID_ARG, "no such CUDA device");
  apic_server* srv = new apic_server();
  srv->device = device;
  srv->budget = hbm_budget_bytes;
  srv->max_batch = max_batch_scenes;
  srv->worker_scratch.assign(n_workers, 0);
  for (int w = 0; w < n_workers; ++w) srv->workers.emplace_back(worker_main, srv, w);
  *out = srv;
  return APIC_OK;
}

apic_status apic_server_set_policy(apic_server* srv, int32_t variant, int32_t graphs) {
  if (!srv) return sfail(APIC_ERR_INVALID_ARG, "server is NULL");
  if (variant < -1 || variant >= apic_variant_count())
    return sfail(APIC_ERR_INVALID_ARG, "variant out of range (-1 tunes per size class)");
  std::lock_guard<std::mutex> lk(srv->mu);
  srv->variant = variant;
  srv->graphs = graphs != 0;
  return APIC_OK;
}

apic_status apic_server_destroy(apic_server* srv) {
  if (!srv) return APIC_OK;
  {
    std::unique_lock<std::mutex> lk(srv->mu);
    srv->cv_done.wait(lk, [&] {
      if (!srv->queue.empty()) return false;
      for (auto& kv : srv->tickets)
        if (kv.second.state != 2) return false;
      return true;
    });
    srv->stop = true;
  }
  srv->cv_work.notify_all();
  for (auto& t : srv->workers) t.join();
  cudaSetDevice(srv->device);
  for (apic_sim* sm : srv->sims) {  // simulations the caller did not close
    free_sim_memory(sm);
    delete sm;
  }
  delete srv;
  return APIC_OK;
}

apic_status apic_sim_open(apic_server* srv, const apic_step_args* a, apic_sim** out) {
  if (!srv || !a || !out) return sfail(APIC_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  if (a->n <= 0 || a->n > (int64_t)INT32_MAX / 4) return sfail(APIC_ERR_INVALID_ARG, "n out of range");
  if (a->n_bodies < 1 || a->n_bodies > 32 || a->n_iter < 0 || !(a->h > 0.0) || !(a->mu >= 0.0))
    return sfail(APIC_ERR_INVALID_ARG, "invalid n_bodies, n_iter, h or mu");
  if (!a->x || !a->body || !a->v || !a->C || !a->m || (!a->nrm && !(a->flags & APIC_MASS_NORMALS)))
    return sfail(APIC_ERR_INVALID_ARG, "a required array pointer is NULL");
  const uint32_t known = APIC_FP64 | APIC_HOST_PTRS | APIC_VARIANT_PIC | APIC_VARIANT_SEP23 | APIC_DETERMINISTIC |
                         APIC_CHECK | APIC_MASS_NORMALS;
  if (a->flags & ~known) return sfail(APIC_ERR_INVALID_ARG, "unknown flag bits");
  const size_t es = (a->flags & APIC_FP64) ? 8 : 4;
  const size_t n = (size_t)a->n;
  const size_t bytes = n * (3 * sizeof(double) + sizeof(int32_t) + es * (3 + 9 + 1 + 3));
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    if (srv->budget && srv->resident + scratch_total(srv) + bytes + n * kScratchPerParticle * (es / 4) > srv->budget)
      return sfail(APIC_ERR_ADMISSION, "the HBM budget cannot hold this simulation now");
    srv->resident += bytes;
  }
  cudaSetDevice(srv->device);
  apic_sim* s = new apic_sim();
  s->srv = srv;
  s->n = a->n;
  s->n_bodies = a->n_bodies;
  s->n_iter = a->n_iter;
  s->flags = a->flags & ~APIC_HOST_PTRS;
  s->h = a->h;
  s->mu = a->mu;
  if (a->mu_pair) s->mu_pair.assign(a->mu_pair, a->mu_pair + a->n_bodies * a->n_bodies);
  s->esize = es;
  s->bytes = bytes;
  const cudaMemcpyKind kind = (a->flags & APIC_HOST_PTRS) ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  cudaError_t e = cudaSuccess;
  auto alloc_copy = [&](void** dst, const void* src, size_t nbytes) {
    if (e != cudaSuccess) return;
    e = cudaMalloc(dst, nbytes);
    if (e == cudaSuccess) e = cudaMemcpy(*dst, src, nbytes, kind);
  };
  alloc_copy(reinterpret_cast<void**>(&s->x), a->x, 3 * n * sizeof(double));
  alloc_copy(reinterpret_cast<void**>(&s->body), a->body, n * sizeof(int32_t));
  alloc_copy(&s->v, a->v, 3 * n * es);
  alloc_copy(&s->C, a->C, 9 * n * es);
  alloc_copy(&s->m, a->m, n * es);
  if (a->nrm) {
    alloc_copy(&s->nrm, a->nrm, 3 * n * es);
  } else if (e == cudaSuccess) {  // APIC_MASS_NORMALS: the steps compute them; keep zeros
    e = cudaMalloc(&s->nrm, 3 * n * es);
    if (e == cudaSuccess) e = cudaMemset(s->nrm, 0, 3 * n * es);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    free_sim_memory(s);
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->resident -= bytes;
    delete s;
    return sfail(e == cudaErrorMemoryAllocation ? APIC_ERR_OUT_OF_MEMORY : APIC_ERR_CUDA, cudaGetErrorString(e));
  }
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->open += 1;
    srv->sims.insert(s);
  }
  *out = s;
  return APIC_OK;
}

apic_status apic_sim_submit(apic_sim* s, double dt_advect, uint64_t* ticket) {
  if (!s || !ticket) return sfail(APIC_ERR_INVALID_ARG, "NULL argument");
  if (!(dt_advect >= 0.0)) return sfail(APIC_ERR_INVALID_ARG, "dt_advect must be >= 0");
  apic_server* srv = s->srv;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    const uint64_t t = srv->next_ticket++;
    Ticket tk;
    tk.sim = s;
    tk.dt = dt_advect;
    tk.t_submit = Clock::now();
    srv->tickets.emplace(t, tk);
    srv->queue.push_back(t);
    s->queued += 1;
    *ticket = t;
  }
  srv->cv_work.notify_one();
  return APIC_OK;
}

apic_status apic_ticket_poll(apic_server* srv, uint64_t ticket, int32_t* done, double* latency_ms) {
  if (!srv || !done) return sfail(APIC_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(srv->mu);
  auto it = srv->tickets.find(ticket);
  if (it == srv->tickets.end()) return sfail(APIC_ERR_INVALID_ARG, "unknown ticket");
  *done = it->second.state == 2;
  if (!*done) return APIC_OK;
  if (latency_ms)
    *latency_ms = std::chrono::duration<double, std::milli>(it->second.t_done - it->second.t_submit).count();
  const apic_status st = it->second.status;
  const std::string why = "the request failed: " + it->second.error;
  srv->tickets.erase(it);  // reported: forgotten
  if (st != APIC_OK) return sfail(st, why.c_str());
  return APIC_OK;
}

apic_status apic_ticket_wait(apic_server* srv, uint64_t ticket, double timeout_s, double* latency_ms) {
  if (!srv) return sfail(APIC_ERR_INVALID_ARG, "NULL argument");
  std::unique_lock<std::mutex> lk(srv->mu);
  auto it = srv->tickets.find(ticket);
  if (it == srv->tickets.end()) return sfail(APIC_ERR_INVALID_ARG, "unknown ticket");
  const auto limit = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                        std::chrono::duration<double>(std::max(0.0, timeout_s)));
  if (!srv->cv_done.wait_until(lk, limit, [&] { return srv->tickets[ticket].state == 2; }))
    return sfail(APIC_ERR_TIMEOUT, "the request did not finish in time");
  auto done = srv->tickets.find(ticket);
  if (latency_ms)
    *latency_ms = std::chrono::duration<double, std::milli>(done->second.t_done - done->second.t_submit).count();
  const apic_status st = done->second.status;
  const std::string why = "the request failed: " + done->second.error;
  srv->tickets.erase(done);  // reported: forgotten
  if (st != APIC_OK) return sfail(st, why.c_str());
  return APIC_OK;
}

apic_status apic_sim_read(apic_sim* s, double* x_out, void* v_out, void* C_out) {
  if (!s) return sfail(APIC_ERR_INVALID_ARG, "NULL argument");
  apic_server* srv = s->srv;
  std::unique_lock<std::mutex> lk(srv->mu);
  wait_idle(srv, lk, s);
  cudaSetDevice(srv->device);
  const size_t n = (size_t)s->n;
  cudaError_t e = cudaSuccess;
  if (x_out) e = cudaMemcpy(x_out, s->x, 3 * n * sizeof(double), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && v_out) e = cudaMemcpy(v_out, s->v, 3 * n * s->esize, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && C_out) e = cudaMemcpy(C_out, s->C, 9 * n * s->esize, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return sfail(APIC_ERR_CUDA, cudaGetErrorString(e));
  return APIC_OK;
}

namespace {

// Checkpoint layout (host byte order): this header, then mu_pair
// (n_bodies^2 doubles, when present), x (3n doubles), body (n int32), and v,
// C, m, normals (3n, 9n, n, 3n values of esize bytes).
struct SimCheckpoint {
  char magic[8];
  uint32_t version, flags;
  int64_t n;
  int32_t n_bodies, n_iter;
  double h, mu;
  int32_t has_mu_pair, esize;
};
constexpr char kCheckpointMagic[8] = {'A', 'P', 'I', 'C', 'S', 'I', 'M', '1'};

size_t checkpoint_bytes(int64_t n, int32_t n_bodies, bool mu_pair, size_t es) {
  return sizeof(SimCheckpoint) + (mu_pair ? sizeof(double) * n_bodies * n_bodies : 0) +
         (size_t)n * (3 * sizeof(double) + sizeof(int32_t) + es * (3 + 9 + 1 + 3));
}

}  // namespace

apic_status apic_sim_export(apic_sim* s, void* host_buf, size_t* bytes) {
  if (!s || !bytes) return sfail(APIC_ERR_INVALID_ARG, "NULL argument");
  const size_t need = checkpoint_bytes(s->n, s->n_bodies, !s->mu_pair.empty(), s->esize);
  if (!host_buf) {
    *bytes = need;
    return APIC_OK;
  }
  if (*bytes < need) return sfail(APIC_ERR_INVALID_ARG, "checkpoint buffer too small (query the size first)");
  apic_server* srv = s->srv;
  std::unique_lock<std::mutex> lk(srv->mu);
  wait_idle(srv, lk, s);
  SimCheckpoint hd{};
  std::memcpy(hd.magic, kCheckpointMagic, 8);
  hd.version = 1;
  hd.flags = s->flags;
  hd.n = s->n;
  hd.n_bodies = s->n_bodies;
  hd.n_iter = s->n_iter;
  hd.h = s->h;
  hd.mu = s->mu;
  hd.has_mu_pair = s->mu_pair.empty() ? 0 : 1;
  hd.esize = (int32_t)s->esize;
  char* o = static_cast<char*>(host_buf);
  std::memcpy(o, &hd, sizeof(hd));
  o += sizeof(hd);
  if (hd.has_mu_pair) {
    std::memcpy(o, s->mu_pair.data(), s->mu_pair.size() * sizeof(double));
    o += s->mu_pair.size() * sizeof(double);
  }
  const size_t n = (size_t)s->n, es = s->esize;
  cudaSetDevice(srv->device);
  const std::pair<const void*, size_t> parts[] = {{s->x, 3 * n * sizeof(double)}, {s->body, n * sizeof(int32_t)},
                                                  {s->v, 3 * n * es}, {s->C, 9 * n * es}, {s->m, n * es},
                                                  {s->nrm, 3 * n * es}};
  for (const auto& pt : parts) {
    const cudaError_t e = cudaMemcpy(o, pt.first, pt.second, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return sfail(APIC_ERR_CUDA, cudaGetErrorString(e));
    o += pt.second;
  }
  *bytes = need;
  return APIC_OK;
}

apic_status apic_sim_import(apic_server* srv, const void* host_buf, size_t bytes, apic_sim** out) {
  if (!srv || !host_buf || !out) return sfail(APIC_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  SimCheckpoint hd{};
  if (bytes < sizeof(hd)) return sfail(APIC_ERR_INVALID_ARG, "not a checkpoint (too short)");
  std::memcpy(&hd, host_buf, sizeof(hd));
  if (std::memcmp(hd.magic, kCheckpointMagic, 8) != 0 || hd.version != 1)
    return sfail(APIC_ERR_INVALID_ARG, "not a checkpoint of this library (magic or version)");
  if (hd.n <= 0 || hd.n > (int64_t)INT32_MAX / 4 || hd.n_bodies < 1 || hd.n_bodies > 32 ||
      (hd.esize != 4 && hd.esize != 8) || (hd.esize == 8) != ((hd.flags & APIC_FP64) != 0))
    return sfail(APIC_ERR_INVALID_ARG, "corrupt checkpoint header");
  if (bytes < checkpoint_bytes(hd.n, hd.n_bodies, hd.has_mu_pair != 0, (size_t)hd.esize))
    return sfail(APIC_ERR_INVALID_ARG, "checkpoint truncated");
  const char* p = static_cast<const char*>(host_buf) + sizeof(hd);
  apic_step_args a{};
  a.n = hd.n;
  a.n_bodies = hd.n_bodies;
  a.n_iter = hd.n_iter;
  a.h = hd.h;
  a.mu = hd.mu;
  a.flags = hd.flags | APIC_HOST_PTRS;
  if (hd.has_mu_pair) {
    a.mu_pair = reinterpret_cast<const double*>(p);
    p += sizeof(double) * hd.n_bodies * hd.n_bodies;
  }
  const size_t n = (size_t)hd.n, es = (size_t)hd.esize;
  a.x = reinterpret_cast<const double*>(p);
  p += 3 * n * sizeof(double);
  a.body = reinterpret_cast<const int32_t*>(p);
  p += n * sizeof(int32_t);
  a.v = const_cast<char*>(p);
  p += 3 * n * es;
  a.C = const_cast<char*>(p);
  p += 9 * n * es;
  a.m = p;
  p += n * es;
  a.nrm = p;
  return apic_sim_open(srv, &a, out);
}

apic_status apic_sim_close(apic_sim* s) {
  if (!s) return APIC_OK;
  apic_server* srv = s->srv;
  {
    std::unique_lock<std::mutex> lk(srv->mu);
    wait_idle(srv, lk, s);
    srv->resident -= s->bytes;
    srv->open -= 1;
    srv->sims.erase(s);
    for (auto it = srv->tickets.begin(); it != srv->tickets.end();)  // its requests are all done
      it = it->second.sim == s ? srv->tickets.erase(it) : std::next(it);
  }
  cudaSetDevice(srv->device);
  free_sim_memory(s);
  delete s;
  return APIC_OK;
}

// ---------------------------------------------------------------------------
// Server groups: one server per device, simulations placed by HBM budget.
// Scenes are independent, so nothing crosses devices on the data path; a
// request goes to the server that holds its simulation.

int32_t apic_place_by_budget(const int64_t* free_bytes, int32_t n_devices, int64_t need) {
  if (!free_bytes || n_devices < 1 || need < 0) return -1;
  int32_t best = -1;
  for (int32_t i = 0; i < n_devices; ++i)
    if (free_bytes[i] >= need && (best < 0 || free_bytes[i] > free_bytes[best])) best = i;
  return best;
}

apic_status apic_sim_server(apic_sim* s, apic_server** out) {
  if (!s || !out) return sfail(APIC_ERR_INVALID_ARG, "NULL argument");
  *out = s->srv;
  return APIC_OK;
}

}  // extern "C"

struct apic_group {
  std::vector<apic_server*> members;
  std::vector<int32_t> devices;
};

namespace {

// Bytes a simulation's admission asks of a server (resident state plus the
// workers' scratch estimate), as apic_sim_open counts them.
int64_t admission_bytes(const apic_step_args* a) {
  const size_t es = (a->flags & APIC_FP64) ? 8 : 4;
  const size_t n = (size_t)a->n;
  const size_t bytes = n * (3 * sizeof(double) + sizeof(int32_t) + es * (3 + 9 + 1 + 3));
  return (int64_t)(bytes + n * kScratchPerParticle * (es / 4));
}

// Bytes a server can still admit (INT64_MAX without a budget).
int64_t free_bytes(apic_server* srv) {
  std::lock_guard<std::mutex> lk(srv->mu);
  if (!srv->budget) return INT64_MAX;
  const size_t used = srv->resident + scratch_total(srv);
  return used >= srv->budget ? 0 : (int64_t)(srv->budget - used);
}

}  // namespace

extern "C" {

apic_status apic_group_create(apic_group** out, const int32_t* devices, int32_t n_devices,
                              size_t hbm_budget_per_device, int32_t n_workers, int32_t max_batch_scenes) {
  if (!out || !devices || n_devices < 1 || n_devices > 64)
    return sfail(APIC_ERR_INVALID_ARG, "need 1..64 devices and an output pointer");
  *out = nullptr;
  apic_group* g = new apic_group();
  for (int32_t i = 0; i < n_devices; ++i) {
    apic_server* srv = nullptr;
    const apic_status st = apic_server_create(&srv, devices[i], hbm_budget_per_device, n_workers, max_batch_scenes);
    if (st != APIC_OK) {
      for (apic_server* m : g->members) apic_server_destroy(m);
      delete g;
      return st;
    }
    g->members.push_back(srv);
    g->devices.push_back(devices[i]);
  }
  *out = g;
  return APIC_OK;
}

apic_status apic_group_destroy(apic_group* g) {
  if (!g) return APIC_OK;
  for (apic_server* m : g->members) apic_server_destroy(m);
  delete g;
  return APIC_OK;
}

apic_status apic_group_server(apic_group* g, int32_t member, apic_server** out) {
  if (!g || !out || member < 0 || member >= (int32_t)g->members.size())
    return sfail(APIC_ERR_INVALID_ARG, "no such group member");
  *out = g->members[(size_t)member];
  return APIC_OK;
}

apic_status apic_group_set_policy(apic_group* g, int32_t variant, int32_t graphs) {
  if (!g) return sfail(APIC_ERR_INVALID_ARG, "group is NULL");
  for (apic_server* m : g->members) {
    const apic_status st = apic_server_set_policy(m, variant, graphs);
    if (st != APIC_OK) return st;
  }
  return APIC_OK;
}

apic_status apic_group_open(apic_group* g, const apic_step_args* a, apic_sim** out, int32_t* member) {
  if (!g || !a || !out) return sfail(APIC_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  const int64_t need = admission_bytes(a);
  const int32_t nm = (int32_t)g->members.size();
  std::vector<int64_t> room((size_t)nm);
  for (int32_t i = 0; i < nm; ++i) room[(size_t)i] = free_bytes(g->members[(size_t)i]);
  // most room first; a member that refuses (others admitted meanwhile) is
  // dropped from the candidates
  for (int32_t tries = 0; tries < nm; ++tries) {
    const int32_t k = apic_place_by_budget(room.data(), nm, need);
    if (k < 0) break;
    const apic_status st = apic_sim_open(g->members[(size_t)k], a, out);
    if (st == APIC_OK) {
      if (member) *member = k;
      return APIC_OK;
    }
    if (st != APIC_ERR_ADMISSION) return st;
    room[(size_t)k] = -1;
  }
  return sfail(APIC_ERR_ADMISSION, "no device of the group has room for this simulation now");
}

apic_status apic_group_get_stats(apic_group* g, apic_server_stats* out, int32_t reset) {
  if (!g || !out) return sfail(APIC_ERR_INVALID_ARG, "NULL argument");
  std::memset(out, 0, sizeof(*out));
  std::vector<double> lat;
  int64_t scenes = 0;
  for (apic_server* m : g->members) {
    std::lock_guard<std::mutex> lk(m->mu);
    out->completed += m->completed;
    out->failed += m->failed;
    out->batches += m->batches;
    out->particle_iters += m->particle_iters;
    out->resident_bytes += (int64_t)m->resident;
    out->open_sims += m->open;
    scenes += m->batch_scenes;
    lat.insert(lat.end(), m->lat_ms.begin(), m->lat_ms.end());
    if (reset) {
      m->lat_ms.clear();
      m->completed = m->failed = m->batches = m->particle_iters = m->batch_scenes = 0;
    }
  }
  out->mean_batch_scenes = out->batches ? (double)scenes / (double)out->batches : 0.0;
  if (!lat.empty()) {
    auto pct = [&](double q) {
      const size_t k = std::min(lat.size() - 1, (size_t)(q * (double)(lat.size() - 1) + 0.5));
      std::nth_element(lat.begin(), lat.begin() + (ptrdiff_t)k, lat.end());
      return lat[k];
    };
    double sum = 0;
    for (double d : lat) sum += d;
    out->latency_mean_ms = sum / (double)lat.size();
    out->latency_p50_ms = pct(0.50);
    out->latency_p99_ms = pct(0.99);
  }
  return APIC_OK;
}

apic_status apic_server_get_stats(apic_server* srv, apic_server_stats* out, int32_t reset) {
  if (!srv || !out) return sfail(APIC_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(srv->mu);
  std::memset(out, 0, sizeof(*out));
  out->completed = srv->completed;
  out->failed = srv->failed;
  out->batches = srv->batches;
  out->particle_iters = srv->particle_iters;
  out->mean_batch_scenes = srv->batches ? (double)srv->batch_scenes / (double)srv->batches : 0.0;
  out->resident_bytes = (int64_t)srv->resident;
  out->open_sims = srv->open;
  if (!srv->lat_ms.empty()) {
    std::vector<double> l = srv->lat_ms;
    auto pct = [&](double q) {
      const size_t k = std::min(l.size() - 1, (size_t)(q * (double)(l.size() - 1) + 0.5));
      std::nth_element(l.begin(), l.begin() + (ptrdiff_t)k, l.end());
      return l[k];
    };
    double sum = 0;
    for (double d : l) sum += d;
    out->latency_mean_ms = sum / (double)l.size();
    out->latency_p50_ms = pct(0.50);
    out->latency_p99_ms = pct(0.99);
  }
  if (reset) {
    srv->lat_ms.clear();
    srv->completed = srv->failed = srv->batches = srv->particle_iters = srv->batch_scenes = 0;
  }
  return APIC_OK;
}

}  // extern "C"
