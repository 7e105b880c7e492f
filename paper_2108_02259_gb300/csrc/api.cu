// C ABI of libapiccontact: contexts, validation, grow-only scratch,
// profiling, and the single-scene and batched contact steps (both run the
// pipeline of pipeline.cuh).
#include <cstring>
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
  std::vector<SceneDev> h_scenes;
  std::vector<int> h_bbox;
  std::vector<char> h_buf;
  // profiling
  bool prof_on = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  struct SpanRec {
    cudaEvent_t a, b;
    int kind;  // 0 step, 1 prep, 2 transfer pass
  };
  std::vector<SpanRec> spans;
  apic_profile prof{};
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
    cudaError_t e = cudaFree(b.ptr);
    if (e != cudaSuccess) return pfail(APIC_ERR_CUDA, "cudaFree: %s", cudaGetErrorString(e));
    c->held -= b.bytes;
    b.ptr = nullptr;
    b.bytes = 0;
  }
  cudaError_t e = cudaMalloc(&b.ptr, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    b.ptr = nullptr;
    return pfail(APIC_ERR_OUT_OF_MEMORY, "cudaMalloc(%zu): %s", want, cudaGetErrorString(e));
  }
  b.bytes = want;
  c->held += want;
  return APIC_OK;
}

void free_buf(apic_ctx* c, Buf& b) {
  if (b.ptr) cudaFree(b.ptr);
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
    } else {
      c->prof.iter_ms += ms;
      c->prof.iter_launches += 1;
    }
  }
  c->spans.clear();
  c->ev_used = 0;
  return APIC_OK;
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
    c->h_scenes.assign(ns, SceneDev{});
    return c->h_scenes.data();
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
  void launched() { c->prof.kernel_launches++; }
  void sorted() { c->prof.sort_launches++; }
  void done(int64_t n, int64_t nodes) {
    c->prof.particles = n;
    c->prof.active_nodes = nodes;
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

constexpr uint32_t kAllFlags = APIC_FP64 | APIC_HOST_PTRS | APIC_VARIANT_PIC | APIC_VARIANT_SEP23;

apic_status run(apic_ctx* c, const apic_step_args* scenes, int ns, void* stream, apic_stats* stats) {
  P_CUDA(cudaSetDevice(c->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CtxEnv env{c};
  const apic_status st = (scenes[0].flags & APIC_FP64) ? run_batch<double>(env, scenes, ns, s, stats)
                                                      : run_batch<float>(env, scenes, ns, s, stats);
  if (st != APIC_OK) {
    c->spans.clear();  // drop unfinished profile spans
    c->ev_used = 0;
  }
  return st;
}

}  // namespace

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
  for (Buf& b : c->bufs) free_buf(c, b);
  if (c->ds) cudaFree(c->ds);
  if (c->hs) cudaFreeHost(c->hs);
  for (auto e : c->ev_pool) cudaEventDestroy(e);
  delete c;
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
  return run(c, scenes, n_scenes, stream, stats);
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

apic_status apic_scratch_bytes(apic_ctx* c, size_t* out) {
  if (!c || !out) return pfail(APIC_ERR_INVALID_ARG, "NULL argument");
  *out = c->held;
  return APIC_OK;
}

}  // extern "C"
