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
// In host code the array's name is only a host-side stand-in, so the device
// address is looked up with cudaGetSymbolAddress once per device, on the
// first call made with that device current; make that first call before
// any stream capture begins.
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/apiccontact.h"
#include "apic_internal.h"

using namespace apic;

namespace {

constexpr size_t kStaticScratchBytes = size_t(32) << 20;  // 32 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_setup_mu;
void* g_scratch_ptr[kMaxDevices] = {};

apic_status sfail(apic_status code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  set_last_error(buf);  // reported by apic_last_error()
  return code;
}

#define S_CUDA(expr)                                                                          \
  do {                                                                                        \
    cudaError_t e_ = (expr);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return sfail(APIC_ERR_CUDA, "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, \
                   __LINE__);                                                                 \
  } while (0)

#define S_TRY(expr)               \
  do {                            \
    apic_status s_ = (expr);      \
    if (s_ != APIC_OK) return s_; \
  } while (0)

// Device address of the static array on the current device (set up once).
apic_status scratch_base(void** out) {
  int dev = 0;
  S_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return sfail(APIC_ERR_INVALID_ARG, "device %d beyond %d", dev, kMaxDevices);
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || p == nullptr)
      return sfail(APIC_ERR_CUDA, "cudaGetSymbolAddress(static scratch) on device %d: %s", dev,
                   cudaGetErrorString(e));
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return APIC_OK;
}

// Bump allocator over the static array; fails (no allocation) when full.
struct Carve {
  char* base;
  size_t used = 0;
  template <class U>
  apic_status take(size_t count, U** out, const char* what) {
    const size_t off = (used + 255) & ~size_t(255);
    const size_t bytes = count * sizeof(U);
    if (off + bytes > kStaticScratchBytes)
      return sfail(APIC_ERR_INVALID_ARG,
                   "scene too large for the static scratch: %s needs %zu bytes at offset %zu of %zu "
                   "(apic_contact_step handles larger scenes)",
                   what, bytes, off, kStaticScratchBytes);
    *out = reinterpret_cast<U*>(base + off);
    used = off + bytes;
    return APIC_OK;
  }
};

int bits_needed(uint64_t v) {
  int b = 0;
  while (b < 64 && (v >> b) != 0) ++b;
  return b;
}

template <class K>
apic_status sort_static(Carve& cv, int64_t n, const int4* cellb, Box box, int n_bodies, int end_bit,
                        int** perm, const void** keys_sorted, int* err, cudaStream_t s) {
  K *ka, *kb;
  int *va, *vb;
  S_TRY(cv.take(n, &ka, "sort keys"));
  S_TRY(cv.take(n, &kb, "sorted keys"));
  S_TRY(cv.take(n, &va, "sort values"));
  S_TRY(cv.take(n, &vb, "permutation"));
  S_CUDA(launch_keys<K>(n, cellb, box, n_bodies, ka, va, err, s));
  size_t tmp = 0;
  S_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, tmp, ka, kb, va, vb, (int)n, 0, end_bit, s));
  char* t;
  S_TRY(cv.take(tmp, &t, "sort temporaries"));
  S_CUDA(cub::DeviceRadixSort::SortPairs(t, tmp, ka, kb, va, vb, (int)n, 0, end_bit, s));
  *perm = vb;
  *keys_sorted = kb;
  return APIC_OK;
}

apic_status scan_static(Carve& cv, const int* in, int* out, int64_t n, cudaStream_t s) {
  size_t tmp = 0;
  S_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, tmp, in, out, n, s));
  char* t;
  S_TRY(cv.take(tmp, &t, "scan temporaries"));
  S_CUDA(cub::DeviceScan::ExclusiveSum(t, tmp, in, out, n, s));
  return APIC_OK;
}

template <class T>
apic_status static_impl(const apic_step_args* a, cudaStream_t s, apic_stats* stats) {
  const int64_t n = a->n;
  void* base = nullptr;
  S_TRY(scratch_base(&base));
  Carve cv{static_cast<char*>(base)};
  const double* x = a->x;
  const int32_t* body = a->body;
  const T* v = static_cast<const T*>(a->v);
  const T* C = static_cast<const T*>(a->C);
  const T* m = static_cast<const T*>(a->m);
  const T* nrm = static_cast<const T*>(a->nrm);

  DevScalars* ds;
  int4* cellb;
  S_TRY(cv.take(1, &ds, "counters"));
  S_TRY(cv.take(n, &cellb, "cells"));
  DevScalars hs{};
  hs.bbox[0] = hs.bbox[1] = hs.bbox[2] = INT32_MAX;
  hs.bbox[3] = hs.bbox[4] = hs.bbox[5] = INT32_MIN;
  S_CUDA(cudaMemcpyAsync(ds, &hs, sizeof(DevScalars), cudaMemcpyHostToDevice, s));
  const double inv_h = 1.0 / a->h;
  S_CUDA(launch_cells<T>(n, x, body, m, inv_h, a->n_bodies, cellb, ds, s));
  if (stats) S_CUDA(launch_momentum<T>(n, x, v, C, m, a->h, &ds->mom[0], s));
  S_CUDA(cudaMemcpyAsync(&hs, ds, sizeof(DevScalars), cudaMemcpyDeviceToHost, s));
  S_CUDA(cudaStreamSynchronize(s));
  if (hs.err) return sfail(APIC_ERR_INVALID_ARG, "invalid particle data (error bits 0x%x)", hs.err);

  Box box;
  box.ox = hs.bbox[0] - 1;
  box.oy = hs.bbox[1] - 1;
  box.oz = hs.bbox[2] - 1;
  box.nx = hs.bbox[3] - hs.bbox[0] + 3;
  box.ny = hs.bbox[4] - hs.bbox[1] + 3;
  box.nz = hs.bbox[5] - hs.bbox[2] + 3;
  const int64_t NB = (int64_t)box.nx * box.ny * box.nz;
  if (NB > (int64_t)(kStaticScratchBytes / 16))
    return sfail(APIC_ERR_INVALID_ARG, "scene spans %lld grid blocks: too large for the static scratch",
                 (long long)NB);
  const int end_bit = bits_needed((uint64_t)NB * (uint64_t)a->n_bodies - 1) + 6;
  const bool k64 = end_bit > 32;
  int* perm = nullptr;
  const void* keys = nullptr;
  if (k64)
    S_TRY(sort_static<uint64_t>(cv, n, cellb, box, a->n_bodies, end_bit, &perm, &keys, &ds->err, s));
  else
    S_TRY(sort_static<uint32_t>(cv, n, cellb, box, a->n_bodies, end_bit, &perm, &keys, &ds->err, s));

  V4<T> *pt, *pn, *V, *D;
  S_TRY(cv.take(n, &pt, "particle offsets"));
  S_TRY(cv.take(n, &pn, "particle normals"));
  S_TRY(cv.take(3 * n, &V, "sorted V"));
  S_TRY(cv.take(3 * n, &D, "Delta"));
  S_CUDA(launch_gather<T>(n, perm, cellb, x, v, C, m, nrm, a->h, inv_h, pt, pn, V, s));

  int *heads, *offs, *item_start;
  int2* item_info;
  S_TRY(cv.take(n, &heads, "item heads"));
  S_TRY(cv.take(n, &offs, "item offsets"));
  S_TRY(cv.take(n, &item_start, "item starts"));
  S_TRY(cv.take(n, &item_info, "item info"));
  if (k64)
    S_CUDA(launch_heads<uint64_t>(n, static_cast<const uint64_t*>(keys), heads, s));
  else
    S_CUDA(launch_heads<uint32_t>(n, static_cast<const uint32_t*>(keys), heads, s));
  S_TRY(scan_static(cv, heads, offs, n, s));
  S_CUDA(launch_compact(n, heads, offs, item_start, nullptr, &ds->n_items, s));
  if (k64)
    S_CUDA(launch_item_info<uint64_t>(item_start, &ds->n_items, static_cast<const uint64_t*>(keys), a->n_bodies,
                                      item_info, (int)n, s));
  else
    S_CUDA(launch_item_info<uint32_t>(item_start, &ds->n_items, static_cast<const uint32_t*>(keys), a->n_bodies,
                                      item_info, (int)n, s));

  int *bflags, *boffs, *blist, *page;
  S_TRY(cv.take(NB, &bflags, "block flags"));
  S_TRY(cv.take(NB, &boffs, "block offsets"));
  S_TRY(cv.take(NB, &blist, "block list"));
  S_TRY(cv.take(NB, &page, "page table"));
  S_CUDA(cudaMemsetAsync(bflags, 0, NB * sizeof(int), s));
  S_CUDA(launch_mark(n, cellb, box, bflags, &ds->err, s));
  S_TRY(scan_static(cv, bflags, boffs, NB, s));
  S_CUDA(launch_compact(NB, bflags, boffs, blist, page, &ds->n_blocks, s));
  S_CUDA(cudaMemcpyAsync(&hs.n_items, &ds->n_items, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
  S_CUDA(cudaStreamSynchronize(s));
  const int n_items = hs.n_items, n_blocks = hs.n_blocks;
  const int64_t n_nodes = (int64_t)n_blocks * kNodesPerBlock;

  T* gm;
  uint32_t* gmask;
  V4<T>*gp, *gv;
  V4<double>* gp64 = nullptr;
  T* gmb = nullptr;
  T* mu_pair_d = nullptr;
  T* mup = nullptr;
  S_TRY(cv.take(n_nodes, &gm, "grid mass"));
  S_TRY(cv.take(n_nodes, &gmask, "grid body mask"));
  S_TRY(cv.take(n_nodes, &gp, "grid momentum"));
  S_TRY(cv.take(n_nodes, &gv, "grid velocity"));
  S_CUDA(cudaMemsetAsync(gm, 0, n_nodes * sizeof(T), s));
  S_CUDA(cudaMemsetAsync(gmask, 0, n_nodes * sizeof(uint32_t), s));
  S_CUDA(cudaMemsetAsync(gp, 0, n_nodes * sizeof(V4<T>), s));
  if (sizeof(T) == 4) {
    S_TRY(cv.take(n_nodes, &gp64, "FP64 node momentum"));
    S_CUDA(cudaMemsetAsync(gp64, 0, n_nodes * sizeof(V4<double>), s));
  }
  T mu_host[32 * 32];
  if (a->mu_pair) {
    const int nb = a->n_bodies;
    S_TRY(cv.take((size_t)nb * n_nodes, &gmb, "per-body grid mass"));
    S_CUDA(cudaMemsetAsync(gmb, 0, (size_t)nb * n_nodes * sizeof(T), s));
    S_TRY(cv.take((size_t)nb * nb, &mu_pair_d, "friction table"));
    S_TRY(cv.take(n, &mup, "particle friction"));
    for (int i = 0; i < nb * nb; ++i) mu_host[i] = (T)a->mu_pair[i];
    S_CUDA(cudaMemcpyAsync(mu_pair_d, mu_host, (size_t)nb * nb * sizeof(T), cudaMemcpyHostToDevice, s));
  }

  IterParams<T> p{};
  p.n_items = n_items;
  p.n_particles = (int)n;
  p.n_bodies = a->n_bodies;
  p.box = box;
  p.item_start = item_start;
  p.item_info = item_info;
  p.page = page;
  p.pt = pt;
  p.pn = pn;
  p.mu = (T)a->mu;
  p.mu_pair = mu_pair_d;
  p.gmb = gmb;
  p.mup_out = mup;
  p.n_nodes = n_nodes;
  p.V = V;
  p.D = D;
  p.gv = gv;
  p.gp = gp;
  p.gm = gm;
  p.gmask = gmask;
  p.gp64 = gp64;
  p.perm = perm;
  p.v_out = a->v_out;
  p.C_out = a->C_out;
  p.inv_h = (T)inv_h;
  p.pic = (a->flags & APIC_VARIANT_PIC) ? 1 : 0;
  p.sep23 = (a->flags & APIC_VARIANT_SEP23) ? 1 : 0;
  S_CUDA(launch_items<T>(p, kModeMass, kChunk, s));
  if (a->mu_pair) {
    S_CUDA(launch_items<T>(p, kModeMu, kChunk, s));
    p.mup = mup;
  }
  S_CUDA(launch_items<T>(p, kModeP2GV, kChunk, s));
  S_CUDA(launch_normalize<T>(n_nodes, gm, gmask, gp, gp64, gv, 0, s));
  const int N = a->n_iter;
  for (int pass = 0; pass <= N; ++pass) {
    const int mode = N == 0 ? kModeOnly : pass == 0 ? kModeFirst : pass == N ? kModeLast : kModeMid;
    S_CUDA(launch_items<T>(p, mode, kChunk, s));
    if (pass < N) S_CUDA(launch_normalize<T>(n_nodes, gm, gmask, gp, gp64, gv, 0, s));
  }
  if (stats) {
    S_CUDA(launch_momentum<T>(n, x, static_cast<const T*>(a->v_out), static_cast<const T*>(a->C_out), m, a->h,
                              &ds->mom[6], s));
    S_CUDA(launch_count_multibody(n_nodes, gmask, &ds->multibody, s));
    S_CUDA(cudaMemcpyAsync(&hs, ds, sizeof(DevScalars), cudaMemcpyDeviceToHost, s));
    S_CUDA(cudaStreamSynchronize(s));
    for (int k = 0; k < 3; ++k) {
      stats->P_in[k] = hs.mom[k];
      stats->L_in[k] = hs.mom[3 + k];
      stats->P_out[k] = hs.mom[6 + k];
      stats->L_out[k] = hs.mom[9 + k];
    }
    stats->multibody_nodes = (int64_t)hs.multibody;
    stats->active_blocks = n_blocks;
    stats->work_items = n_items;
  }
  return APIC_OK;
}

}  // namespace

extern "C" {

apic_status apic_contact_step_static(const apic_step_args* a, void* stream, apic_stats* stats) {
  if (!a) return sfail(APIC_ERR_INVALID_ARG, "args is NULL");
  if (a->n < 0 || a->n > (int64_t)INT32_MAX / 4) return sfail(APIC_ERR_INVALID_ARG, "n = %lld out of range", (long long)a->n);
  if (a->n_bodies < 1 || a->n_bodies > 32) return sfail(APIC_ERR_INVALID_ARG, "n_bodies = %d outside [1, 32]", a->n_bodies);
  if (a->n_iter < 0) return sfail(APIC_ERR_INVALID_ARG, "n_iter = %d < 0", a->n_iter);
  if (!(a->h > 0.0) || !std::isfinite(a->h)) return sfail(APIC_ERR_INVALID_ARG, "h = %g must be finite and > 0", a->h);
  if (!(a->mu >= 0.0) || !std::isfinite(a->mu)) return sfail(APIC_ERR_INVALID_ARG, "mu = %g must be finite and >= 0", a->mu);
  if (a->flags & APIC_HOST_PTRS)
    return sfail(APIC_ERR_INVALID_ARG, "apic_contact_step_static takes device pointers only (no APIC_HOST_PTRS)");
  const uint32_t known = APIC_FP64 | APIC_VARIANT_PIC | APIC_VARIANT_SEP23;
  if (a->flags & ~known) return sfail(APIC_ERR_INVALID_ARG, "unknown flag bits 0x%x", a->flags & ~known);
  if (a->n > 0 && (!a->body || !a->x || !a->v || !a->C || !a->m || !a->nrm || !a->v_out || !a->C_out))
    return sfail(APIC_ERR_INVALID_ARG, "a required array pointer is NULL");
  if (a->mu_pair)
    for (int i = 0; i < a->n_bodies * a->n_bodies; ++i)
      if (!(a->mu_pair[i] >= 0.0) || !std::isfinite(a->mu_pair[i]))
        return sfail(APIC_ERR_INVALID_ARG, "mu_pair[%d] = %g must be finite and >= 0", i, a->mu_pair[i]);
  if (stats) std::memset(stats, 0, sizeof(*stats));
  if (a->n == 0) return APIC_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return (a->flags & APIC_FP64) ? static_impl<double>(a, s, stats) : static_impl<float>(a, s, stats);
}

}  // extern "C"
