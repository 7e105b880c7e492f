// C ABI of libapiccontact: contexts, validation, grow-only scratch,
// profiling, and the single-scene and batched contact steps (both run the
// pipeline of pipeline.cuh).
#include <algorithm>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "pipeline.cuh"

using namespace apic;

namespace {

thread_local std::string g_last_error;

// A grow-only device buffer owned by the context.
struct Buf {
  void* ptr = nullptr;
  size_t bytes = 0;
};

}  // namespace

void apic::set_last_error(const char* msg) { g_last_error = msg; }

struct apic_ctx {
  int device = 0;
  int num_sms = 0;
  size_t budget = 0;
  size_t held = 0;
  Buf bufs[kSlotCount];
  DevScalars* ds = nullptr;  // device counters
  DevScalars* hs = nullptr;  // pinned host mirror
  // page-table boxes of the last step, per scene, and host staging
  std::vector<Box> boxes;
  int box_ns = -1;
  bool have_box = false;
  SceneDev* h_scenes = nullptr;  // pinned (a graph's copy node reads it)
  int h_scenes_cap = 0;
  CopyEntry* h_copies = nullptr;  // pinned copy table (the copy kernel reads it)
  int h_copies_cap = 0;
  std::vector<int> h_bbox;
  std::vector<char> h_buf;
  // profiling
  bool prof_on = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  struct SpanRec {
    cudaEvent_t a, b;
    int kind;  // 0 step, 1 prep, 2 transfer pass, 3 mass pass
  };
  std::vector<SpanRec> spans;
  apic_profile prof{};
  // autotuner: per size class (FP32, bit length of the particle count), the
  // best time of the series region seen for each kernel variant
  struct TuneClass {
    float best_ms[kNumVariants];
    int samples[kNumVariants] = {};
    int chosen = -1;
    TuneClass() {
      for (float& b : best_ms) b = 1e30f;
    }
  };
  std::map<int, TuneClass> tune;
  int forced_variant = -1;  // >= 0: fixed by the caller
  int tune_reps = 2;        // timed runs of each variant before choosing
  cudaEvent_t tune_a = nullptr, tune_b = nullptr;
  int pending_class = -1, pending_variant = -1;  // a timed run not yet read back
  int cur_class = -1, cur_variant = 0;
  bool cur_measure = false;
  // CUDA graphs of the grid-sizing sequence and of the series region
  // (memsets, mass pass, N + 1 passes)
  struct GraphSlot {
    std::vector<char> key;  // the region's key at the last call (+ alloc_gen)
    bool captured = false;
    bool failed = false;  // capture failed once: launch directly from then on
    cudaGraphExec_t exec = nullptr;
    int64_t kernels = 0, sorts = 0;  // launches inside the graph
  };
  bool graphs_on = true;
  bool overlap_on = true;  // programmatic dependent launch between the passes
  GraphSlot gsizing, gseries;
  cudaStream_t cap_stream = nullptr;
  // side stream of the host path (v and C cross the host link while the
  // sizing sequence runs) and its two events
  cudaStream_t side = nullptr;
  cudaEvent_t side_ev[3] = {nullptr, nullptr, nullptr};
  uint64_t alloc_gen = 0;  // bumped whenever a scratch buffer moves
  // the caller's device allocator for scratch (apic_set_allocator), or none
  apic_alloc_fn ualloc = nullptr;
  apic_free_fn ufree = nullptr;
  void* uuser = nullptr;
};

namespace {

apic_status grow(apic_ctx* c, Buf& b, size_t bytes) {
  if (bytes <= b.bytes) return APIC_OK;
  size_t want = bytes + bytes / 4 + 256;
  if (c->budget && c->held - b.bytes + want > c->budget) {
    want = bytes;
    if (c->held - b.bytes + want > c->budget)
      return pfail(APIC_ERR_OUT_OF_MEMORY, "scratch of %zu bytes exceeds the context budget (%zu held of %zu)",
                   bytes, c->held, c->budget);
  }
  if (b.ptr) {
    if (c->ufree) {
      // the caller's allocator may hand the block out again at once: every
      // queued kernel that could still use it finishes first (cudaFree
      // implies the same wait)
      const cudaError_t e = cudaDeviceSynchronize();
      if (e != cudaSuccess) return pfail(APIC_ERR_CUDA, "cudaDeviceSynchronize: %s", cudaGetErrorString(e));
      c->ufree(c->uuser, b.ptr, b.bytes, c->device);
    } else {
      const cudaError_t e = cudaFree(b.ptr);
      if (e != cudaSuccess) return pfail(APIC_ERR_CUDA, "cudaFree: %s", cudaGetErrorString(e));
    }
    c->held -= b.bytes;
    b.ptr = nullptr;
    b.bytes = 0;
  }
  c->alloc_gen += 1;
  if (c->ualloc) {
    b.ptr = c->ualloc(c->uuser, want, c->device);
    if (!b.ptr) return pfail(APIC_ERR_OUT_OF_MEMORY, "the caller's allocator returned NULL for %zu bytes", want);
    if (reinterpret_cast<uintptr_t>(b.ptr) % 256 != 0) {
      c->ufree(c->uuser, b.ptr, want, c->device);
      b.ptr = nullptr;
      return pfail(APIC_ERR_INVALID_ARG, "the caller's allocator returned a block not aligned to 256 bytes");
    }
  } else {
    const cudaError_t e = cudaMalloc(&b.ptr, want);
    if (e != cudaSuccess) {
      cudaGetLastError();
      b.ptr = nullptr;
      return pfail(APIC_ERR_OUT_OF_MEMORY, "cudaMalloc(%zu): %s", want, cudaGetErrorString(e));
    }
  }
  b.bytes = want;
  c->held += want;
  return APIC_OK;
}

// (apic_destroy synchronises the device before it frees through the
// caller's allocator)
void free_buf(apic_ctx* c, Buf& b) {
  if (b.ptr) {
    if (c->ufree)
      c->ufree(c->uuser, b.ptr, b.bytes, c->device);
    else
      cudaFree(b.ptr);
  }
  c->held -= b.bytes;
  b = Buf{};
}

cudaEvent_t next_event(apic_ctx* c) {
  if (c->ev_used == c->ev_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    c->ev_pool.push_back(e);
  }
  return c->ev_pool[c->ev_used++];
}

// Fold recorded spans into the profile counters (synchronises on them).
apic_status harvest(apic_ctx* c) {
  for (auto& sp : c->spans) {
    P_CUDA(cudaEventSynchronize(sp.b));
    float ms = 0.f;
    P_CUDA(cudaEventElapsedTime(&ms, sp.a, sp.b));
    if (sp.kind == 0) {
      c->prof.step_ms += ms;
      c->prof.steps += 1;
    } else if (sp.kind == 1) {
      c->prof.prep_ms += ms;
    } else if (sp.kind == 3) {
      c->prof.mass_ms += ms;
    } else {
      c->prof.iter_ms += ms;
      c->prof.iter_launches += 1;
    }
  }
  c->spans.clear();
  c->ev_used = 0;
  return APIC_OK;
}

int tune_class(int64_t n) {
  int b = 0;
  while (b < 62 && (int64_t(1) << b) <= n) ++b;
  return b;  // bit length of n
}

// Read back the last timed run (if it has finished) into its size class.
void collect_tuning(apic_ctx* c) {
  if (c->pending_class < 0) return;
  const cudaError_t q = cudaEventQuery(c->tune_b);
  if (q == cudaSuccess) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->tune_a, c->tune_b) == cudaSuccess) {
      apic_ctx::TuneClass& tc = c->tune[c->pending_class];
      const int v = c->pending_variant;
      tc.best_ms[v] = std::min(tc.best_ms[v], ms);
      tc.samples[v] += 1;
      bool all = true;
      for (int i = 0; i < kNumVariants; ++i) all = all && tc.samples[i] >= c->tune_reps;
      if (all && tc.chosen < 0) {
        int best = 0;
        for (int i = 1; i < kNumVariants; ++i)
          if (tc.best_ms[i] < tc.best_ms[best]) best = i;
        tc.chosen = best;
      }
    }
  }
  cudaGetLastError();  // a run still in flight is dropped, not an error
  c->pending_class = -1;
}

// The pipeline's environment backed by a context: grow-only scratch per
// slot, a page-table box cache across steps, CUDA-event spans.
struct CtxEnv {
  apic_ctx* c;

  template <class U>
  apic_status take(int slot, size_t count, U** out, const char*) {
    P_TRY(grow(c, c->bufs[slot], count * sizeof(U) + 64));
    *out = static_cast<U*>(c->bufs[slot].ptr);
    return APIC_OK;
  }
  DevScalars* ds() { return c->ds; }
  DevScalars* hs() { return c->hs; }
  SceneDev* host_scenes(int ns) {
    if (ns > c->h_scenes_cap) {
      if (c->h_scenes) cudaFreeHost(c->h_scenes);
      c->h_scenes = nullptr;
      c->h_scenes_cap = 0;
      if (cudaMallocHost(&c->h_scenes, ns * sizeof(SceneDev)) != cudaSuccess) {
        cudaGetLastError();
        c->h_scenes = nullptr;
        return nullptr;
      }
      c->h_scenes_cap = ns;
    }
    for (int i = 0; i < ns; ++i) c->h_scenes[i] = SceneDev{};
    return c->h_scenes;
  }
  int* host_bbox(int ns) {
    c->h_bbox.resize(6 * (size_t)ns);
    return c->h_bbox.data();
  }
  Box* box_cache(int ns) {
    if (c->box_ns != ns) {
      c->boxes.assign(ns, Box{});
      c->box_ns = ns;
      c->have_box = false;
    }
    return c->boxes.data();
  }
  bool have_box() const { return c->have_box; }
  void keep_box() { c->have_box = true; }
  void forget_box() { c->have_box = false; }
  void* host_buf(size_t bytes) {
    if (c->h_buf.size() < bytes) c->h_buf.resize(bytes);
    return c->h_buf.data();
  }
  // Pinned, device-visible table of n copy entries (nullptr if unavailable).
  CopyEntry* copy_table(int n) {
    if (n > c->h_copies_cap) {
      if (c->h_copies) cudaFreeHost(c->h_copies);
      c->h_copies = nullptr;
      c->h_copies_cap = 0;
      if (cudaMallocHost(&c->h_copies, (size_t)n * sizeof(CopyEntry)) != cudaSuccess) {
        cudaGetLastError();
        c->h_copies = nullptr;
        return nullptr;
      }
      c->h_copies_cap = n;
    }
    return c->h_copies;
  }
  // Side stream and events for overlapping host-to-device staging (nullptr
  // if they cannot be created: the caller then stages on its own stream).
  cudaStream_t side_stream() {
    if (!c->side) {
      if (cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        c->side = nullptr;
        return nullptr;
      }
      for (cudaEvent_t& e : c->side_ev)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
          cudaGetLastError();
          for (cudaEvent_t& f : c->side_ev)
            if (f) cudaEventDestroy(f), f = nullptr;
          cudaStreamDestroy(c->side);
          c->side = nullptr;
          return nullptr;
        }
    }
    return c->side;
  }
  cudaEvent_t side_event(int k) { return c->side_ev[k]; }
  // The device's address of a page-locked host array, or nullptr (pageable
  // memory, device memory, or no mapping).
  static const void* device_view(const void* p) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
  }
  // Overlap each pass with the tail of the grid before it, except while
  // profiling times the passes one by one.
  bool overlap() const { return c->overlap_on && !c->prof_on; }
  void launched() { c->prof.kernel_launches++; }
  void sorted() { c->prof.sort_launches++; }
  void done(int64_t n, int64_t nodes) {
    c->prof.particles = n;
    c->prof.active_nodes = nodes;
  }

  // Variant 0, untimed (deterministic mode).
  int variant_fixed() {
    collect_tuning(c);
    c->cur_measure = false;
    return 0;
  }
  // Kernel variant for this call: the caller's fixed choice, the size
  // class's tuned choice, or (while the class is being tuned) the variant
  // with the fewest timed runs, whose series region is then timed.
  int variant(size_t tsize, int64_t n) {
    collect_tuning(c);
    c->cur_measure = false;
    if (c->forced_variant >= 0) return c->forced_variant;
    if (tsize != 4) return 0;  // one FP64 variant
    const int k = tune_class(n);
    apic_ctx::TuneClass& tc = c->tune[k];
    if (tc.chosen >= 0) return tc.chosen;
    int v = 0;
    for (int i = 1; i < kNumVariants; ++i)
      if (tc.samples[i] < tc.samples[v]) v = i;
    c->cur_class = k;
    c->cur_variant = v;
    c->cur_measure = c->tune_a != nullptr;
    return v;
  }

  // The sizing sequence, as a graph when `allowed` (device pointers) and the
  // same sizes and buffers come back.
  template <class F>
  apic_status run_sizing(const void* key, size_t kb, bool allowed, cudaStream_t s, F& body) {
    if (!allowed) return body(s);
    return graph_run(c->gsizing, key, kb, s, body);
  }

  // The series region (timed for the autotuner while its class is tuned).
  template <class F>
  apic_status run_series(const void* key, size_t kb, cudaStream_t s, F& body) {
    const bool measure = c->cur_measure;
    if (measure) P_CUDA(cudaEventRecord(c->tune_a, s));
    P_TRY(graph_run(c->gseries, key, kb, s, body));
    if (measure) {
      P_CUDA(cudaEventRecord(c->tune_b, s));
      c->pending_class = c->cur_class;
      c->pending_variant = c->cur_variant;
    }
    return APIC_OK;
  }

  // Run a launch sequence: directly the first time its key is seen (and
  // whenever graphs are off, or profiling needs per-pass events), captured
  // as a CUDA graph the second consecutive time, replayed after that.  The
  // key is the caller's bytes plus the context's allocation generation, so
  // a buffer that moved forces a fresh capture.
  template <class F>
  apic_status graph_run(apic_ctx::GraphSlot& g, const void* key, size_t kb, cudaStream_t s, F& body) {
    if (!c->graphs_on || c->prof_on || g.failed) return body(s);
    std::vector<char> k(static_cast<const char*>(key), static_cast<const char*>(key) + kb);
    const char* gp = reinterpret_cast<const char*>(&c->alloc_gen);
    k.insert(k.end(), gp, gp + sizeof(c->alloc_gen));
    const bool same = g.key == k;
    if (same && g.captured) {
      P_CUDA(cudaGraphLaunch(g.exec, s));
      c->prof.kernel_launches += g.kernels;
      c->prof.sort_launches += g.sorts;
      c->prof.graph_launches += 1;
      return APIC_OK;
    }
    if (!same) {
      g.key = std::move(k);
      g.captured = false;
      return body(s);
    }
    if (!c->cap_stream) P_CUDA(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    const int64_t k0 = c->prof.kernel_launches, s0 = c->prof.sort_launches;
    const uint64_t gen0 = c->alloc_gen;
    P_CUDA(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    const apic_status st = body(c->cap_stream);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(c->cap_stream, &graph);
    g.kernels = c->prof.kernel_launches - k0;
    g.sorts = c->prof.sort_launches - s0;
    c->prof.kernel_launches = k0;
    c->prof.sort_launches = s0;
    if (st != APIC_OK || e != cudaSuccess || c->alloc_gen != gen0) {
      // Nothing ran while capturing.  Whatever went wrong (a buffer that had
      // to grow, a call capture does not allow), run the sequence directly:
      // a real error shows up there and is returned.
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      g.key.clear();
      g.failed = st != APIC_OK || e != cudaSuccess;
      return body(s);
    }
    if (g.exec) {
      cudaGraphExecUpdateResultInfo info;
      if (cudaGraphExecUpdate(g.exec, graph, &info) != cudaSuccess) {
        cudaGetLastError();
        cudaGraphExecDestroy(g.exec);
        g.exec = nullptr;
      }
    }
    if (!g.exec) {
      const cudaError_t ei = cudaGraphInstantiate(&g.exec, graph, 0);
      if (ei != cudaSuccess) {
        cudaGraphDestroy(graph);
        g.exec = nullptr;
        g.key.clear();
        return pfail(APIC_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(ei));
      }
    }
    cudaGraphDestroy(graph);
    g.captured = true;
    P_CUDA(cudaGraphLaunch(g.exec, s));
    c->prof.graph_launches += 1;
    c->prof.kernel_launches += g.kernels;
    c->prof.sort_launches += g.sorts;
    return APIC_OK;
  }

  struct Span {
    apic_ctx* c;
    cudaStream_t s;
    cudaEvent_t a = nullptr;
    int kind;
    Span(CtxEnv& e, cudaStream_t s_, int k) : c(e.c), s(s_), kind(k) {
      if (c->prof_on) {
        a = next_event(c);
        if (a) cudaEventRecord(a, s);
      }
    }
    void stop() {
      if (a) {
        cudaEvent_t b = next_event(c);
        if (b) {
          cudaEventRecord(b, s);
          c->spans.push_back({a, b, kind});
        }
        a = nullptr;
      }
    }
    ~Span() { stop(); }
  };
};

constexpr uint32_t kAllFlags = APIC_FP64 | APIC_HOST_PTRS | APIC_VARIANT_PIC | APIC_VARIANT_SEP23 |
                               APIC_DETERMINISTIC | APIC_CHECK | APIC_MASS_NORMALS | APIC_PARTITIONED;

apic_status run(apic_ctx* c, const apic_step_args* scenes, int ns, void* stream, apic_stats* stats,
                bool normals_only = false, double nthr = kMassNormalThreshold) {
  P_CUDA(cudaSetDevice(c->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CtxEnv env{c};
  const apic_status st = (scenes[0].flags & APIC_FP64)
                             ? run_batch<double>(env, scenes, ns, s, stats, normals_only, nthr)
                             : run_batch<float>(env, scenes, ns, s, stats, normals_only, nthr);
  if (st != APIC_OK) {
    c->spans.clear();  // drop unfinished profile spans
    c->ev_used = 0;
  }
  return st;
}

}  // namespace

apic_status apic::ctx_take(apic_ctx* c, int slot, size_t bytes, void** out) {
  if (slot < 0 || slot >= kSlotCount) return pfail(APIC_ERR_INVALID_ARG, "internal: scratch slot %d", slot);
  P_TRY(grow(c, c->bufs[slot], bytes + 64));
  *out = c->bufs[slot].ptr;
  return APIC_OK;
}

extern "C" {

const char* apic_last_error(void) { return g_last_error.c_str(); }

const char* apic_version(void) { return "libapiccontact 0.2 (sm_103a)"; }

apic_status apic_create(apic_ctx** out, int32_t device, size_t hbm_budget_bytes) {
  if (!out) return pfail(APIC_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  int count = 0;
  P_CUDA(cudaGetDeviceCount(&count));
  if (device < 0 || device >= count) return pfail(APIC_ERR_INVALID_ARG, "device %d not in [0, %d)", device, count);
  P_CUDA(cudaSetDevice(device));
  apic_ctx* c = new apic_ctx();
  c->device = device;
  c->budget = hbm_budget_bytes;
  cudaError_t e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) e = cudaMalloc(&c->ds, sizeof(DevScalars));
  if (e == cudaSuccess) e = cudaMallocHost(&c->hs, sizeof(DevScalars));
  if (e == cudaSuccess) e = cudaEventCreate(&c->tune_a);
  if (e == cudaSuccess) e = cudaEventCreate(&c->tune_b);
  if (e != cudaSuccess) {
    apic_destroy(c);
    return pfail(APIC_ERR_CUDA, "apic_create: %s", cudaGetErrorString(e));
  }
  *out = c;
  return APIC_OK;
}

apic_status apic_destroy(apic_ctx* c) {
  if (!c) return APIC_OK;
  cudaSetDevice(c->device);
  if (c->ufree) cudaDeviceSynchronize();
  for (Buf& b : c->bufs) free_buf(c, b);
  if (c->ds) cudaFree(c->ds);
  if (c->hs) cudaFreeHost(c->hs);
  for (auto e : c->ev_pool) cudaEventDestroy(e);
  if (c->tune_a) cudaEventDestroy(c->tune_a);
  if (c->tune_b) cudaEventDestroy(c->tune_b);
  if (c->gsizing.exec) cudaGraphExecDestroy(c->gsizing.exec);
  if (c->gseries.exec) cudaGraphExecDestroy(c->gseries.exec);
  if (c->h_scenes) cudaFreeHost(c->h_scenes);
  if (c->h_copies) cudaFreeHost(c->h_copies);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->side) cudaStreamDestroy(c->side);
  for (cudaEvent_t e : c->side_ev)
    if (e) cudaEventDestroy(e);
  delete c;
  cudaGetLastError();  // a failed release is not left pending for the caller's next launch
  return APIC_OK;
}

apic_status apic_contact_step(apic_ctx* c, const apic_step_args* a, void* stream, apic_stats* stats) {
  if (!c) return pfail(APIC_ERR_INVALID_ARG, "ctx is NULL");
  P_TRY(validate_scene(a, 0, kAllFlags));
  if (stats) std::memset(stats, 0, sizeof(*stats));
  if (a->n == 0) return APIC_OK;
  return run(c, a, 1, stream, stats);
}

apic_status apic_contact_step_batched(apic_ctx* c, const apic_step_args* scenes, int32_t n_scenes, void* stream,
                                      apic_stats* stats) {
  if (!c) return pfail(APIC_ERR_INVALID_ARG, "ctx is NULL");
  if (n_scenes < 1 || !scenes)
    return pfail(APIC_ERR_INVALID_ARG, "n_scenes = %d (need >= 1 and a scene array)", n_scenes);
  for (int i = 0; i < n_scenes; ++i) {
    P_TRY(validate_scene(&scenes[i], i, kAllFlags));
    if (scenes[i].flags != scenes[0].flags)
      return pfail(APIC_ERR_INVALID_ARG, "scene %d: flags 0x%x differ from scene 0 (0x%x); a batch shares them", i,
                   scenes[i].flags, scenes[0].flags);
    if (scenes[i].n_iter != scenes[0].n_iter)
      return pfail(APIC_ERR_INVALID_ARG, "scene %d: n_iter %d differs from scene 0 (%d); a batch shares it", i,
                   scenes[i].n_iter, scenes[0].n_iter);
  }
  if (scenes[0].flags & APIC_PARTITIONED) {
    // partitions of one scene: one grid spacing, one set of bodies, one friction law
    if (scenes[0].flags & APIC_DETERMINISTIC)
      return pfail(APIC_ERR_INVALID_ARG, "APIC_PARTITIONED does not combine with APIC_DETERMINISTIC");
    const apic_step_args& a0 = scenes[0];
    for (int i = 1; i < n_scenes; ++i) {
      const apic_step_args& a = scenes[i];
      if (a.h != a0.h || a.n_bodies != a0.n_bodies || a.mu != a0.mu || (a.mu_pair == nullptr) != (a0.mu_pair == nullptr))
        return pfail(APIC_ERR_INVALID_ARG,
                     "partition %d: h, n_bodies, mu and the presence of mu_pair must equal partition 0's", i);
      if (a.mu_pair)  // (a host table)
        for (int k = 0; k < a.n_bodies * a.n_bodies; ++k)
          if (a.mu_pair[k] != a0.mu_pair[k])
            return pfail(APIC_ERR_INVALID_ARG, "partition %d: mu_pair differs from partition 0's", i);
    }
  }
  return run(c, scenes, n_scenes, stream, stats);
}

apic_status apic_mass_normals(apic_ctx* c, const apic_step_args* a, double threshold, void* nrm_out, void* stream) {
  if (!c) return pfail(APIC_ERR_INVALID_ARG, "ctx is NULL");
  if (!a) return pfail(APIC_ERR_INVALID_ARG, "args is NULL");
  if (!(threshold >= 0.0) || !std::isfinite(threshold))
    return pfail(APIC_ERR_INVALID_ARG, "threshold = %g must be finite and >= 0", threshold);
  if (a->flags & ~(APIC_FP64 | APIC_DETERMINISTIC))
    return pfail(APIC_ERR_INVALID_ARG, "flag bits 0x%x not accepted here (APIC_FP64, APIC_DETERMINISTIC only)",
                 a->flags & ~(APIC_FP64 | APIC_DETERMINISTIC));
  if (a->n > 0 && (!a->x || !a->body || !a->m || !nrm_out))
    return pfail(APIC_ERR_INVALID_ARG, "x, body, m and nrm_out are required");
  // the step's own checks, on a copy whose velocities are unused stand-ins
  apic_step_args b = *a;
  b.v = b.C = b.v_out = b.C_out = nrm_out;
  b.nrm = nullptr;
  b.mu_pair = nullptr;
  b.flags = a->flags | APIC_MASS_NORMALS;
  P_TRY(validate_scene(&b, 0, kAllFlags));
  if (b.n == 0) return APIC_OK;
  b.v_out = nrm_out;  // where the normals go
  return run(c, &b, 1, stream, nullptr, true, threshold);
}

apic_status apic_set_profiling(apic_ctx* c, int32_t on) {
  if (!c) return pfail(APIC_ERR_INVALID_ARG, "ctx is NULL");
  P_TRY(harvest(c));
  c->prof_on = on != 0;
  c->prof = apic_profile{};
  return APIC_OK;
}

apic_status apic_get_profile(apic_ctx* c, apic_profile* out) {
  if (!c || !out) return pfail(APIC_ERR_INVALID_ARG, "NULL argument");
  P_TRY(harvest(c));
  *out = c->prof;
  return APIC_OK;
}

apic_status apic_node_normals(apic_ctx* c, int64_t n, const double* x, int64_t n_tri, const int32_t* tri,
                              void* nrm_out, uint32_t flags, void* stream) {
  if (!c) return pfail(APIC_ERR_INVALID_ARG, "ctx is NULL");
  if (n < 0 || n_tri < 0) return pfail(APIC_ERR_INVALID_ARG, "n = %lld, n_tri = %lld must be >= 0", (long long)n,
                                       (long long)n_tri);
  if (n > (int64_t)INT32_MAX) return pfail(APIC_ERR_INVALID_ARG, "n = %lld exceeds int32 node ids", (long long)n);
  if (flags & ~(uint32_t)(APIC_FP64 | APIC_HOST_PTRS))
    return pfail(APIC_ERR_INVALID_ARG, "flag bits 0x%x not accepted here", flags & ~(uint32_t)(APIC_FP64 | APIC_HOST_PTRS));
  if (n == 0) {
    if (n_tri > 0) return pfail(APIC_ERR_INVALID_ARG, "triangles given for n = 0 nodes");
    return APIC_OK;
  }
  if (!x || !nrm_out || (n_tri > 0 && !tri)) return pfail(APIC_ERR_INVALID_ARG, "a required array pointer is NULL");
  P_CUDA(cudaSetDevice(c->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CtxEnv env{c};
  const bool host = (flags & APIC_HOST_PTRS) != 0;
  const size_t es = (flags & APIC_FP64) ? sizeof(double) : sizeof(float);
  double* acc;
  P_TRY(env.take(kSlotNrmAcc, 3 * n, &acc, "normal sums"));
  const double* dx = x;
  const int32_t* dtri = tri;
  void* dout = nrm_out;
  if (host) {
    double* sx;
    int32_t* st = nullptr;
    char* so;
    P_TRY(env.take(kSlotNrmX, 3 * n, &sx, "staged x"));
    if (n_tri > 0) P_TRY(env.take(kSlotNrmTri, 3 * n_tri, &st, "staged triangles"));
    P_TRY(env.take(kSlotNrmOut, 3 * n * es, &so, "staged normals"));
    P_CUDA(cudaMemcpyAsync(sx, x, 3 * n * sizeof(double), cudaMemcpyHostToDevice, s));
    if (n_tri > 0) P_CUDA(cudaMemcpyAsync(st, tri, 3 * n_tri * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    dx = sx;
    dtri = st;
    dout = so;
  }
  P_CUDA(cudaMemsetAsync(c->ds, 0, sizeof(DevScalars), s));
  P_CUDA(cudaMemsetAsync(acc, 0, 3 * n * sizeof(double), s));
  P_LAUNCH(env, launch_face_normals(n_tri, dtri, dx, n, acc, &c->ds->err, s));
  if (flags & APIC_FP64)
    P_LAUNCH(env, launch_unit_normals<double>(n, acc, static_cast<double*>(dout), s));
  else
    P_LAUNCH(env, launch_unit_normals<float>(n, acc, static_cast<float*>(dout), s));
  if (host) P_CUDA(cudaMemcpyAsync(nrm_out, dout, 3 * n * es, cudaMemcpyDeviceToHost, s));
  P_CUDA(cudaMemcpyAsync(c->hs, c->ds, sizeof(DevScalars), cudaMemcpyDeviceToHost, s));
  P_CUDA(cudaStreamSynchronize(s));
  if (c->hs->err) return pfail(APIC_ERR_INVALID_ARG, "a triangle index is outside [0, %lld)", (long long)n);
  return APIC_OK;
}

int32_t apic_debug_build(void) {
#ifdef APIC_DEBUG_BOUNDS
  return 1;
#else
  return 0;
#endif
}

apic_status apic_debug_flags(uint32_t* out, int32_t clear) {
  if (!out) return pfail(APIC_ERR_INVALID_ARG, "out is NULL");
  const unsigned a = kernels_debug_flags(clear), b = sort_debug_flags(clear);
  if (a == ~0u || b == ~0u) return pfail(APIC_ERR_CUDA, "reading the bounds-check words failed");
  *out = a | b;
  return APIC_OK;
}

int32_t apic_variant_count(void) { return kNumVariants; }

const char* apic_variant_name(int32_t v) {
  static const char* names[kNumVariants] = {
      "128 threads/CTA, items <= 128, 8 CTAs/SM (64 registers)",
      "128 threads/CTA, items <= 128, 9 CTAs/SM (56 registers)",
      "128 threads/CTA, items <= 128, 7 CTAs/SM (72 registers)",
      "64 threads/CTA, items <= 64, 13 CTAs/SM (72 registers)",
      "64 threads/CTA, items <= 64, 16 CTAs/SM (64 registers, 13 resident by shared memory)",
      "128 threads/CTA, items <= 128, 8 CTAs/SM (64 registers), stashed row weights",
      "128 threads/CTA, items <= 128, 7 CTAs/SM (72 registers), stashed row weights",
      "128 threads/CTA, 2 particles/thread, items <= 256, 8-lane P2G groups, 5 CTAs/SM (96 registers)",
      "128 threads/CTA, items <= 128, 9 CTAs/SM (56 registers), persistent grid",
  };
  return v >= 0 && v < kNumVariants ? names[v] : "";
}

apic_status apic_set_variant(apic_ctx* c, int32_t v) {
  if (!c) return pfail(APIC_ERR_INVALID_ARG, "ctx is NULL");
  if (v < -1 || v >= kNumVariants) return pfail(APIC_ERR_INVALID_ARG, "variant %d not in [-1, %d)", v, kNumVariants);
  c->forced_variant = v;
  return APIC_OK;
}

apic_status apic_get_variant(apic_ctx* c, int64_t n_particles, int32_t* variant, int32_t* decided) {
  if (!c || !variant || !decided) return pfail(APIC_ERR_INVALID_ARG, "NULL argument");
  collect_tuning(c);
  if (c->forced_variant >= 0) {
    *variant = c->forced_variant;
    *decided = 1;
    return APIC_OK;
  }
  auto it = c->tune.find(tune_class(n_particles));
  const bool ok = it != c->tune.end() && it->second.chosen >= 0;
  *variant = ok ? it->second.chosen : 0;
  *decided = ok ? 1 : 0;
  return APIC_OK;
}

apic_status apic_get_tuning(apic_ctx* c, int32_t* classes, int32_t* variants, int32_t cap, int32_t* count) {
  if (!c || !count || cap < 0 || (cap > 0 && (!classes || !variants)))
    return pfail(APIC_ERR_INVALID_ARG, "NULL argument or negative capacity");
  collect_tuning(c);
  int32_t k = 0;
  for (const auto& [cls, tc] : c->tune) {
    if (tc.chosen < 0) continue;
    if (k < cap) {
      classes[k] = cls;
      variants[k] = tc.chosen;
    }
    ++k;
  }
  *count = k;
  return APIC_OK;
}

apic_status apic_set_tuning(apic_ctx* c, const int32_t* classes, const int32_t* variants, int32_t count) {
  if (!c || count < 0 || (count > 0 && (!classes || !variants)))
    return pfail(APIC_ERR_INVALID_ARG, "NULL argument or negative count");
  for (int32_t i = 0; i < count; ++i) {
    if (classes[i] < 0 || classes[i] > 62)
      return pfail(APIC_ERR_INVALID_ARG, "entry %d: size class %d outside [0, 62]", i, classes[i]);
    if (variants[i] < 0 || variants[i] >= kNumVariants)
      return pfail(APIC_ERR_INVALID_ARG, "entry %d: variant %d outside [0, %d)", i, variants[i], kNumVariants);
  }
  collect_tuning(c);
  for (int32_t i = 0; i < count; ++i) c->tune[classes[i]].chosen = variants[i];
  return APIC_OK;
}

apic_status apic_autotune(apic_ctx* c, const apic_step_args* scenes, int32_t n_scenes, void* stream,
                          int32_t* variant) {
  if (!c) return pfail(APIC_ERR_INVALID_ARG, "ctx is NULL");
  if (c->forced_variant >= 0)
    return pfail(APIC_ERR_INVALID_ARG, "the variant is fixed (apic_set_variant); set -1 to tune");
  int64_t n = 0;
  for (int i = 0; scenes && i < n_scenes; ++i) n += scenes[i].n;
  const int rounds = kNumVariants * c->tune_reps + 1;
  int32_t v = 0, decided = 0;
  for (int r = 0; r < rounds; ++r) {
    P_TRY(apic_get_variant(c, n, &v, &decided));
    if (decided) break;
    P_TRY(apic_contact_step_batched(c, scenes, n_scenes, stream, nullptr));
    P_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  }
  P_TRY(apic_get_variant(c, n, &v, &decided));
  if (!decided) return pfail(APIC_ERR_CUDA, "autotuning did not finish (timings unavailable)");
  if (variant) *variant = v;
  return APIC_OK;
}

apic_status apic_set_graphs(apic_ctx* c, int32_t on) {
  if (!c) return pfail(APIC_ERR_INVALID_ARG, "ctx is NULL");
  c->graphs_on = on != 0;
  for (apic_ctx::GraphSlot* g : {&c->gsizing, &c->gseries}) {
    g->key.clear();
    g->captured = false;
    g->failed = false;
  }
  return APIC_OK;
}

apic_status apic_set_allocator(apic_ctx* c, apic_alloc_fn alloc, apic_free_fn free_fn, void* user) {
  if (!c) return pfail(APIC_ERR_INVALID_ARG, "ctx is NULL");
  if ((alloc == nullptr) != (free_fn == nullptr))
    return pfail(APIC_ERR_INVALID_ARG, "give both allocator functions, or neither");
  if (c->held != 0)
    return pfail(APIC_ERR_INVALID_ARG, "the context already holds %zu bytes of scratch: set the allocator first",
                 c->held);
  c->ualloc = alloc;
  c->ufree = free_fn;
  c->uuser = user;
  return APIC_OK;
}

apic_status apic_set_overlap(apic_ctx* c, int32_t on) {
  if (!c) return pfail(APIC_ERR_INVALID_ARG, "ctx is NULL");
  c->overlap_on = on != 0;
  for (apic_ctx::GraphSlot* g : {&c->gsizing, &c->gseries}) {
    g->key.clear();
    g->captured = false;
    g->failed = false;
  }
  return APIC_OK;
}

apic_status apic_scratch_bytes(apic_ctx* c, size_t* out) {
  if (!c || !out) return pfail(APIC_ERR_INVALID_ARG, "NULL argument");
  *out = c->held;
  return APIC_OK;
}

}  // extern "C"
