// apic_contact_step_static: the contact step for callers that cannot
// allocate device memory.
//
// Some hosts cannot call cudaMalloc while they run a contact step: an
// application whose own pool already reserved (nearly) all of the GPU's
// memory and hands out nothing else, or a real-time loop in which the
// device-wide synchronisation that cudaMalloc and cudaFree imply is not
// acceptable.  This entry point serves them: it takes the same inputs and
// outputs as apic_contact_step but carves every scratch buffer (sort keys,
// sorted particle planes, page table, grid nodes, sort and scan temporaries,
// the small device-side counters) out of one statically sized device array,
// kStaticScratchBytes long, that the library defines at file scope.  It
// calls no cudaMalloc, cudaFree or allocating library routine.
//
// The array exists once per GPU that loads the library and stays allocated
// until the process exits.  Every call uses the same array and leaves the
// last call's data in it; each call clears what must start at zero.  Two
// calls whose GPU work overlaps (two streams, two host threads) race on the
// array and corrupt each other's results: serialise them.
//
// In host code the array's name is only a host-side stand-in, so every call
// looks up the array's device address on the current device with
// cudaGetSymbolAddress (a host-side table lookup once the module is loaded).
// The address is not cached: a device reset, or a primary context torn down
// and created again, reloads the module at another address, and a cached
// pointer would then be stale.  The first call on a device loads the module
// there; make that first call before any stream capture begins.
#include "pipeline.cuh"

using namespace apic;

namespace {

constexpr size_t kStaticScratchBytes = size_t(32) << 20;  // 32 MiB

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of the static array on the current device, looked up on
// every call (never cached, so that it stays valid across device resets).
apic_status scratch_base(void** out) {
  int dev = 0;
  P_CUDA(cudaGetDevice(&dev));
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
  if (e != cudaSuccess || p == nullptr)
    return pfail(APIC_ERR_CUDA, "cudaGetSymbolAddress(static scratch) on device %d: %s", dev,
                 cudaGetErrorString(e));
  *out = p;
  return APIC_OK;
}

// The pipeline's environment for this entry point: a bump allocator over the
// static array (refusing what does not fit), host staging on the stack, no
// box reuse between calls, no profiling.
struct StaticEnv {
  char* base = nullptr;
  size_t used = 0;
  DevScalars* d = nullptr;
  DevScalars h{};
  SceneDev scene{};
  int bbox[6] = {};
  Box box{};
  alignas(16) char hbuf[32 * 32 * sizeof(double) + 16 * sizeof(double)];

  template <class U>
  apic_status take(int, size_t count, U** out, const char* what) {
    const size_t off = (used + 255) & ~size_t(255);
    const size_t bytes = count * sizeof(U);
    if (off + bytes > kStaticScratchBytes)
      return pfail(APIC_ERR_INVALID_ARG,
                   "scene too large for the static scratch: %s needs %zu bytes at offset %zu of %zu "
                   "(apic_contact_step handles larger scenes)",
                   what, bytes, off, kStaticScratchBytes);
    *out = reinterpret_cast<U*>(base + off);
    used = off + bytes;
    return APIC_OK;
  }
  DevScalars* ds() { return d; }
  DevScalars* hs() { return &h; }
  SceneDev* host_scenes(int ns) { return ns == 1 ? &scene : nullptr; }
  int* host_bbox(int) { return bbox; }
  Box* box_cache(int) { return &box; }
  bool have_box() const { return false; }
  void keep_box() {}
  void forget_box() {}
  void* host_buf(size_t bytes) { return bytes <= sizeof(hbuf) ? hbuf : nullptr; }
  void launched() {}
  void sorted() {}
  void done(int64_t, int64_t) {}
  // device pointers only: no host staging
  CopyEntry* copy_table(int) { return nullptr; }
  cudaStream_t side_stream() { return nullptr; }
  cudaEvent_t side_event(int) { return nullptr; }
  static const void* device_view(const void*) { return nullptr; }
  // default kernel variant, launched directly (no graph, no tuning state)
  int variant(size_t, int64_t) { return 0; }
  int variant_fixed() { return 0; }
  template <class F>
  apic_status run_series(const void*, size_t, cudaStream_t s, F& body) {
    return body(s);
  }
  template <class F>
  apic_status run_sizing(const void*, size_t, bool, cudaStream_t s, F& body) {
    return body(s);
  }
  bool overlap() const { return true; }
  struct Span {
    Span(StaticEnv&, cudaStream_t, int) {}
    void stop() {}
  };
};

}  // namespace

extern "C" {

apic_status apic_contact_step_static(const apic_step_args* a, void* stream, apic_stats* stats) {
  P_TRY(validate_scene(a, 0, APIC_FP64 | APIC_VARIANT_PIC | APIC_VARIANT_SEP23 | APIC_DETERMINISTIC | APIC_CHECK |
                                   APIC_MASS_NORMALS));
  if (stats) std::memset(stats, 0, sizeof(*stats));
  if (a->n == 0) return APIC_OK;
  StaticEnv env;
  void* base = nullptr;
  P_TRY(scratch_base(&base));
  env.base = static_cast<char*>(base);
  P_TRY(env.take(kSlotDS, 1, &env.d, "counters"));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return (a->flags & APIC_FP64) ? run_batch<double>(env, a, 1, s, stats) : run_batch<float>(env, a, 1, s, stats);
}

}  // extern "C"
