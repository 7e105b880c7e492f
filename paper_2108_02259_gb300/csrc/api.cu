// C ABI of libapiccontact: context, validation, scratch management and the
// per-step orchestration of the kernels in kernels.cu.
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/apiccontact.h"
#include "apic_internal.h"

using namespace apic;

namespace {

thread_local std::string g_last_error;

apic_status fail(apic_status code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

#define CUDA_TRY(expr)                                                                       \
  do {                                                                                       \
    cudaError_t e_ = (expr);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return fail(e_ == cudaErrorMemoryAllocation ? APIC_ERR_OUT_OF_MEMORY : APIC_ERR_CUDA, \
                  "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, __LINE__);     \
  } while (0)

// Launch of one of this library's kernels (counted for the profile).
#define KLAUNCH(c, expr)    \
  do {                      \
    (c)->prof.kernel_launches++; \
    CUDA_TRY(expr);         \
  } while (0)

#define APIC_TRY(expr)              \
  do {                              \
    apic_status s_ = (expr);        \
    if (s_ != APIC_OK) return s_;   \
  } while (0)

// A grow-only device buffer owned by the context.
struct Buf {
  void* ptr = nullptr;
  size_t bytes = 0;
};

constexpr int kMaxBodies = 32;
constexpr int64_t kMaxPageEntries = int64_t(1) << 28;  // dense page table limit (1 GiB)
constexpr int kBoxSlack = 2;  // blocks of room for motion when a page-table box is reused

}  // namespace

void apic::set_last_error(const char* msg) { g_last_error = msg; }

struct apic_ctx {
  int device = 0;
  int num_sms = 0;
  size_t budget = 0;
  size_t held = 0;
  // scratch
  Buf cellb, keys_a, keys_b, vals_a, perm, pt, pn, V, D, mup, heads, offs, item_start, item_info;
  Buf bflags, boffs, blist, page, gm, gmask, gp, gp64, gv, gmb, mu_pair, cub_tmp;
  Buf h_x, h_body, h_v, h_C, h_m, h_nrm, h_vo, h_Co;  // staging for APIC_HOST_PTRS
  Box box{};                      // page-table box of the last step
  bool have_box = false;
  DevScalars* ds = nullptr;       // device
  DevScalars* hs = nullptr;       // pinned host mirror
  // profiling
  bool prof_on = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  struct Span {
    cudaEvent_t a, b;
    int kind;  // 0 step, 1 prep, 2 iteration kernel
  };
  std::vector<Span> spans;
  apic_profile prof{};
};

namespace {

apic_status grow(apic_ctx* c, Buf& b, size_t bytes) {
  if (bytes <= b.bytes) return APIC_OK;
  size_t want = bytes + bytes / 4 + 256;
  if (c->budget && c->held - b.bytes + want > c->budget) {
    want = bytes;
    if (c->held - b.bytes + want > c->budget)
      return fail(APIC_ERR_OUT_OF_MEMORY, "scratch of %zu bytes exceeds the context budget (%zu held of %zu)",
                  bytes, c->held, c->budget);
  }
  if (b.ptr) {
    cudaError_t e = cudaFree(b.ptr);
    if (e != cudaSuccess) return fail(APIC_ERR_CUDA, "cudaFree: %s", cudaGetErrorString(e));
    c->held -= b.bytes;
    b.ptr = nullptr;
    b.bytes = 0;
  }
  cudaError_t e = cudaMalloc(&b.ptr, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    b.ptr = nullptr;
    return fail(APIC_ERR_OUT_OF_MEMORY, "cudaMalloc(%zu): %s", want, cudaGetErrorString(e));
  }
  b.bytes = want;
  c->held += want;
  return APIC_OK;
}

template <class U>
apic_status get(apic_ctx* c, Buf& b, size_t count, U** out) {
  APIC_TRY(grow(c, b, count * sizeof(U) + 64));
  *out = static_cast<U*>(b.ptr);
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

struct Timer {
  apic_ctx* c;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  int kind;
  Timer(apic_ctx* c_, cudaStream_t s_, int k) : c(c_), s(s_), kind(k) {
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
  ~Timer() { stop(); }
};

// Fold recorded spans into the profile counters (synchronises on them).
apic_status harvest(apic_ctx* c) {
  for (auto& sp : c->spans) {
    CUDA_TRY(cudaEventSynchronize(sp.b));
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, sp.a, sp.b));
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

int bits_for(uint64_t v) {  // bits needed to represent 0..v
  int b = 0;
  while (b < 64 && (v >> b) != 0) ++b;
  return b;
}

template <class K>
apic_status sort_pairs(apic_ctx* c, const K* kin, K* kout, const int* vin, int* vout, int n, int end_bit,
                       cudaStream_t s) {
  size_t tmp = 0;
  CUDA_TRY(cub::DeviceRadixSort::SortPairs(nullptr, tmp, kin, kout, vin, vout, n, 0, end_bit, s));
  void* t = nullptr;
  APIC_TRY(get(c, c->cub_tmp, tmp, reinterpret_cast<char**>(&t)));
  CUDA_TRY(cub::DeviceRadixSort::SortPairs(t, tmp, kin, kout, vin, vout, n, 0, end_bit, s));
  c->prof.sort_launches++;
  return APIC_OK;
}

apic_status exclusive_sum(apic_ctx* c, const int* in, int* out, int64_t n, cudaStream_t s) {
  size_t tmp = 0;
  CUDA_TRY(cub::DeviceScan::ExclusiveSum(nullptr, tmp, in, out, n, s));
  void* t = nullptr;
  APIC_TRY(get(c, c->cub_tmp, tmp, reinterpret_cast<char**>(&t)));
  CUDA_TRY(cub::DeviceScan::ExclusiveSum(t, tmp, in, out, n, s));
  c->prof.sort_launches++;
  return APIC_OK;
}

apic_status validate(const apic_step_args* a) {
  if (!a) return fail(APIC_ERR_INVALID_ARG, "args is NULL");
  if (a->n < 0) return fail(APIC_ERR_INVALID_ARG, "n = %lld < 0", (long long)a->n);
  if (a->n > (int64_t)INT32_MAX / 4)
    return fail(APIC_ERR_INVALID_ARG, "n = %lld exceeds the per-call limit %d", (long long)a->n, INT32_MAX / 4);
  if (a->n_bodies < 1 || a->n_bodies > kMaxBodies)
    return fail(APIC_ERR_INVALID_ARG, "n_bodies = %d outside [1, %d]", a->n_bodies, kMaxBodies);
  if (a->n_iter < 0) return fail(APIC_ERR_INVALID_ARG, "n_iter = %d < 0", a->n_iter);
  if (!(a->h > 0.0) || !std::isfinite(a->h)) return fail(APIC_ERR_INVALID_ARG, "h = %g must be finite and > 0", a->h);
  if (!(a->mu >= 0.0) || !std::isfinite(a->mu)) return fail(APIC_ERR_INVALID_ARG, "mu = %g must be finite and >= 0", a->mu);
  const uint32_t known = APIC_FP64 | APIC_HOST_PTRS | APIC_VARIANT_PIC | APIC_VARIANT_SEP23;
  if (a->flags & ~known) return fail(APIC_ERR_INVALID_ARG, "unknown flag bits 0x%x", a->flags & ~known);
  if (a->n > 0 && (!a->body || !a->x || !a->v || !a->C || !a->m || !a->nrm || !a->v_out || !a->C_out))
    return fail(APIC_ERR_INVALID_ARG, "a required array pointer is NULL");
  if (a->mu_pair) {
    const int nb = a->n_bodies;
    for (int i = 0; i < nb * nb; ++i)
      if (!(a->mu_pair[i] >= 0.0) || !std::isfinite(a->mu_pair[i]))
        return fail(APIC_ERR_INVALID_ARG, "mu_pair[%d] = %g must be finite and >= 0", i, a->mu_pair[i]);
    for (int i = 0; i < nb; ++i)
      for (int j = 0; j < nb; ++j)
        if (a->mu_pair[i * nb + j] != a->mu_pair[j * nb + i])
          return fail(APIC_ERR_INVALID_ARG, "mu_pair is not symmetric at (%d, %d)", i, j);
  }
  return APIC_OK;
}

template <class K>
apic_status keys_sort(apic_ctx* c, int64_t n, const int4* cellb, Box box, int n_bodies, int end_bit,
                      int** perm_out, const void** keys_out, cudaStream_t s) {
  // particles outside the (possibly reused) box raise kErrBox
  K *ka, *kb;
  int *va, *vb;
  APIC_TRY(get(c, c->keys_a, n, &ka));
  APIC_TRY(get(c, c->keys_b, n, &kb));
  APIC_TRY(get(c, c->vals_a, n, &va));
  APIC_TRY(get(c, c->perm, n, &vb));
  KLAUNCH(c, launch_keys<K>(n, cellb, box, n_bodies, ka, va, &c->ds->err, s));
  APIC_TRY(sort_pairs<K>(c, ka, kb, va, vb, (int)n, end_bit, s));
  *perm_out = vb;
  *keys_out = kb;
  return APIC_OK;
}

template <class T>
apic_status step_impl(apic_ctx* c, const apic_step_args* a, cudaStream_t s, apic_stats* stats) {
  const int64_t n = a->n;
  const bool host = (a->flags & APIC_HOST_PTRS) != 0;
  Timer t_step(c, s, 0);
  Timer t_prep(c, s, 1);

  // Inputs on the device (staged through scratch for host pointers).
  const double* x = a->x;
  const int32_t* body = a->body;
  const T* v = static_cast<const T*>(a->v);
  const T* C = static_cast<const T*>(a->C);
  const T* m = static_cast<const T*>(a->m);
  const T* nrm = static_cast<const T*>(a->nrm);
  T* vo = static_cast<T*>(a->v_out);
  T* Co = static_cast<T*>(a->C_out);
  if (host) {
    double* dx;
    int32_t* db;
    T *dv, *dC, *dm, *dn, *dvo, *dCo;
    APIC_TRY(get(c, c->h_x, 3 * n, &dx));
    APIC_TRY(get(c, c->h_body, n, &db));
    APIC_TRY(get(c, c->h_v, 3 * n, &dv));
    APIC_TRY(get(c, c->h_C, 9 * n, &dC));
    APIC_TRY(get(c, c->h_m, n, &dm));
    APIC_TRY(get(c, c->h_nrm, 3 * n, &dn));
    APIC_TRY(get(c, c->h_vo, 3 * n, &dvo));
    APIC_TRY(get(c, c->h_Co, 9 * n, &dCo));
    CUDA_TRY(cudaMemcpyAsync(dx, x, 3 * n * sizeof(double), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(db, body, n * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(dv, v, 3 * n * sizeof(T), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(dC, C, 9 * n * sizeof(T), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(dm, m, n * sizeof(T), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(dn, nrm, 3 * n * sizeof(T), cudaMemcpyHostToDevice, s));
    x = dx; body = db; v = dv; C = dC; m = dm; nrm = dn; vo = dvo; Co = dCo;
  }

  // Steps 1-5 size the sparse grid.  The page-table box of the previous step
  // (kept with a margin) is reused when every particle still fits in it;
  // otherwise the kernels flag kErrBox and the steps are redone with a box
  // fitted to this step's particles.  Nothing is written to the outputs
  // before the grid is sized, so redoing is safe.
  int4* cellb;
  APIC_TRY(get(c, c->cellb, n, &cellb));
  const double inv_h = 1.0 / a->h;
  Box box{};
  int64_t NB = 0;
  int* perm = nullptr;
  const void* keys = nullptr;
  bool k64 = false;
  V4<T> *pt, *pn, *V, *D;
  int *heads, *offs, *item_start;
  int2* item_info;
  int* page = nullptr;
  for (int attempt = 0;; ++attempt) {
    // 1. cells, validation, bounding box of particle blocks; momentum of V.
    DevScalars init{};
    init.bbox[0] = init.bbox[1] = init.bbox[2] = INT32_MAX;
    init.bbox[3] = init.bbox[4] = init.bbox[5] = INT32_MIN;
    *c->hs = init;
    CUDA_TRY(cudaMemcpyAsync(c->ds, c->hs, sizeof(DevScalars), cudaMemcpyHostToDevice, s));
    KLAUNCH(c, launch_cells<T>(n, x, body, m, inv_h, a->n_bodies, cellb, c->ds, s));
    if (stats) KLAUNCH(c, launch_momentum<T>(n, x, v, C, m, a->h, &c->ds->mom[0], s));
    const bool fresh = !c->have_box || attempt > 0;
    if (fresh) {
      CUDA_TRY(cudaMemcpyAsync(c->hs, c->ds, sizeof(DevScalars), cudaMemcpyDeviceToHost, s));
      CUDA_TRY(cudaStreamSynchronize(s));
      if (c->hs->err) break;  // reported below
      // 2. page-table box: one block of stencil margin plus kBoxSlack blocks of
      //    room for motion in later steps.
      const int g = 1 + kBoxSlack;
      c->box.ox = c->hs->bbox[0] - g;
      c->box.oy = c->hs->bbox[1] - g;
      c->box.oz = c->hs->bbox[2] - g;
      c->box.nx = c->hs->bbox[3] - c->hs->bbox[0] + 1 + 2 * g;
      c->box.ny = c->hs->bbox[4] - c->hs->bbox[1] + 1 + 2 * g;
      c->box.nz = c->hs->bbox[5] - c->hs->bbox[2] + 1 + 2 * g;
      c->have_box = true;
    }
    box = c->box;
    NB = (int64_t)box.nx * box.ny * box.nz;
    if (NB > kMaxPageEntries) {
      c->have_box = false;
      return fail(APIC_ERR_INVALID_ARG,
                  "the particles span %lld grid blocks of 4^3 nodes; the dense page table is limited to %lld",
                  (long long)NB, (long long)kMaxPageEntries);
    }
    const int end_bit = bits_for((uint64_t)NB * (uint64_t)a->n_bodies - 1) + 6;
    k64 = end_bit > 32;
    if (k64)
      APIC_TRY(keys_sort<uint64_t>(c, n, cellb, box, a->n_bodies, end_bit, &perm, &keys, s));
    else
      APIC_TRY(keys_sort<uint32_t>(c, n, cellb, box, a->n_bodies, end_bit, &perm, &keys, s));

    // 3. sorted SoA.
    APIC_TRY(get(c, c->pt, n, &pt));
    APIC_TRY(get(c, c->pn, n, &pn));
    APIC_TRY(get(c, c->V, 3 * n, &V));
    APIC_TRY(get(c, c->D, 3 * n, &D));
    KLAUNCH(c, launch_gather<T>(n, perm, cellb, x, v, C, m, nrm, a->h, inv_h, pt, pn, V, s));

    // 4. work items: runs of equal (grid block, body), at most kChunk long.
    APIC_TRY(get(c, c->heads, n, &heads));
    APIC_TRY(get(c, c->offs, n, &offs));
    APIC_TRY(get(c, c->item_start, n, &item_start));
    APIC_TRY(get(c, c->item_info, n, &item_info));
    if (k64)
      KLAUNCH(c, launch_heads<uint64_t>(n, static_cast<const uint64_t*>(keys), heads, s));
    else
      KLAUNCH(c, launch_heads<uint32_t>(n, static_cast<const uint32_t*>(keys), heads, s));
    APIC_TRY(exclusive_sum(c, heads, offs, n, s));
    KLAUNCH(c, launch_compact(n, heads, offs, item_start, nullptr, &c->ds->n_items, s));
    if (k64)
      KLAUNCH(c, launch_item_info<uint64_t>(item_start, &c->ds->n_items, static_cast<const uint64_t*>(keys),
                                          a->n_bodies, item_info, (int)n, s));
    else
      KLAUNCH(c, launch_item_info<uint32_t>(item_start, &c->ds->n_items, static_cast<const uint32_t*>(keys),
                                          a->n_bodies, item_info, (int)n, s));

    // 5. active grid blocks: every block some stencil reaches; page table.
    int *bflags, *boffs, *blist;
    APIC_TRY(get(c, c->bflags, NB, &bflags));
    APIC_TRY(get(c, c->boffs, NB, &boffs));
    APIC_TRY(get(c, c->blist, NB, &blist));
    APIC_TRY(get(c, c->page, NB, &page));
    CUDA_TRY(cudaMemsetAsync(bflags, 0, NB * sizeof(int), s));
    if (k64)
      KLAUNCH(c, launch_mark_items<uint64_t>(item_start, item_info, &c->ds->n_items,
                                           static_cast<const uint64_t*>(keys), n, (int)n, box, bflags, s));
    else
      KLAUNCH(c, launch_mark_items<uint32_t>(item_start, item_info, &c->ds->n_items,
                                           static_cast<const uint32_t*>(keys), n, (int)n, box, bflags, s));
    APIC_TRY(exclusive_sum(c, bflags, boffs, NB, s));
    KLAUNCH(c, launch_compact(NB, bflags, boffs, blist, page, &c->ds->n_blocks, s));
    CUDA_TRY(cudaMemcpyAsync(c->hs, c->ds, sizeof(DevScalars), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if ((c->hs->err & kErrBox) && !(c->hs->err & ~kErrBox) && attempt == 0) {
      c->have_box = false;  // a particle left the reused box: size a fresh one
      continue;
    }
    break;
  }
  if (c->hs->err) {
    const int e = c->hs->err;
    c->have_box = false;
    return fail(APIC_ERR_INVALID_ARG, "invalid particle data:%s%s%s%s", (e & kErrBody) ? " body id out of range" : "",
                (e & kErrMass) ? " mass not finite and > 0" : "",
                (e & kErrPos) ? " position not finite or |x/h| >= 2^29" : "",
                (e & kErrBox) ? " (internal: page-table box)" : "");
  }
  const int n_items = c->hs->n_items;
  const int n_blocks = c->hs->n_blocks;
  const int64_t n_nodes = (int64_t)n_blocks * kNodesPerBlock;

  // 6. node arrays.
  T* gm;
  uint32_t* gmask;
  V4<T>* gp;
  V4<T>* gv;
  V4<double>* gp64 = nullptr;
  T* gmb = nullptr;
  APIC_TRY(get(c, c->gm, n_nodes, &gm));
  APIC_TRY(get(c, c->gmask, n_nodes, &gmask));
  APIC_TRY(get(c, c->gp, n_nodes, &gp));
  APIC_TRY(get(c, c->gv, n_nodes, &gv));
  CUDA_TRY(cudaMemsetAsync(gm, 0, n_nodes * sizeof(T), s));
  CUDA_TRY(cudaMemsetAsync(gmask, 0, n_nodes * sizeof(uint32_t), s));
  CUDA_TRY(cudaMemsetAsync(gp, 0, n_nodes * sizeof(V4<T>), s));
  if (sizeof(T) == 4) {
    APIC_TRY(get(c, c->gp64, n_nodes, &gp64));
    CUDA_TRY(cudaMemsetAsync(gp64, 0, n_nodes * sizeof(V4<double>), s));
  }
  T* mu_pair_d = nullptr;
  T* mup = nullptr;
  if (a->mu_pair) {
    const int nb = a->n_bodies;
    APIC_TRY(get(c, c->gmb, (size_t)nb * n_nodes, &gmb));
    CUDA_TRY(cudaMemsetAsync(gmb, 0, (size_t)nb * n_nodes * sizeof(T), s));
    APIC_TRY(get(c, c->mu_pair, (size_t)nb * nb, &mu_pair_d));
    APIC_TRY(get(c, c->mup, n, &mup));
    std::vector<T> tmp((size_t)nb * nb);
    for (int i = 0; i < nb * nb; ++i) tmp[i] = (T)a->mu_pair[i];
    CUDA_TRY(cudaMemcpyAsync(mu_pair_d, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice, s));
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
  p.mup = nullptr;
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
  p.v_out = vo;
  p.C_out = Co;
  p.inv_h = (T)inv_h;
  p.pic = (a->flags & APIC_VARIANT_PIC) ? 1 : 0;
  p.sep23 = (a->flags & APIC_VARIANT_SEP23) ? 1 : 0;
  const int threads = 128;

  // 7. mass, optional friction blend, P2G(V), then the N+1 transfer passes.
  KLAUNCH(c, launch_items<T>(p, kModeMassV, threads, s));
  if (a->mu_pair) {
    KLAUNCH(c, launch_items<T>(p, kModeMu, threads, s));
    p.mup = mup;
  }
  KLAUNCH(c, launch_normalize<T>(n_nodes, gm, gmask, gp, gp64, gv, 1, s));
  t_prep.stop();
  const int N = a->n_iter;
  for (int pass = 0; pass <= N; ++pass) {
    const int mode = N == 0 ? kModeOnly : pass == 0 ? kModeFirst : pass == N ? kModeLast : kModeMid;
    {
      Timer t_it(c, s, 2);
      KLAUNCH(c, launch_items<T>(p, mode, threads, s));
    }
    if (pass < N) KLAUNCH(c, launch_normalize<T>(n_nodes, gm, gmask, gp, gp64, gv, 0, s));
  }
  t_step.stop();

  if (stats) {
    KLAUNCH(c, launch_momentum<T>(n, x, vo, Co, m, a->h, &c->ds->mom[6], s));
    KLAUNCH(c, launch_count_multibody(n_nodes, gmask, &c->ds->multibody, s));
  }
  if (host) {
    CUDA_TRY(cudaMemcpyAsync(a->v_out, vo, 3 * n * sizeof(T), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(a->C_out, Co, 9 * n * sizeof(T), cudaMemcpyDeviceToHost, s));
  }
  if (stats) {
    CUDA_TRY(cudaMemcpyAsync(c->hs, c->ds, sizeof(DevScalars), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    for (int k = 0; k < 3; ++k) {
      stats->P_in[k] = c->hs->mom[k];
      stats->L_in[k] = c->hs->mom[3 + k];
      stats->P_out[k] = c->hs->mom[6 + k];
      stats->L_out[k] = c->hs->mom[9 + k];
    }
    stats->multibody_nodes = (int64_t)c->hs->multibody;
    stats->active_blocks = n_blocks;
    stats->work_items = n_items;
  }
  if (host) CUDA_TRY(cudaStreamSynchronize(s));
  c->prof.particles = n;
  c->prof.active_nodes = n_nodes;
  return APIC_OK;
}

}  // namespace

extern "C" {

const char* apic_last_error(void) { return g_last_error.c_str(); }

const char* apic_version(void) { return "libapiccontact 0.1 (sm_103a)"; }

apic_status apic_create(apic_ctx** out, int32_t device, size_t hbm_budget_bytes) {
  if (!out) return fail(APIC_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  int count = 0;
  CUDA_TRY(cudaGetDeviceCount(&count));
  if (device < 0 || device >= count) return fail(APIC_ERR_INVALID_ARG, "device %d not in [0, %d)", device, count);
  CUDA_TRY(cudaSetDevice(device));
  apic_ctx* c = new apic_ctx();
  c->device = device;
  c->budget = hbm_budget_bytes;
  cudaError_t e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) e = cudaMalloc(&c->ds, sizeof(DevScalars));
  if (e == cudaSuccess) e = cudaMallocHost(&c->hs, sizeof(DevScalars));
  if (e != cudaSuccess) {
    apic_destroy(c);
    return fail(APIC_ERR_CUDA, "apic_create: %s", cudaGetErrorString(e));
  }
  *out = c;
  return APIC_OK;
}

apic_status apic_destroy(apic_ctx* c) {
  if (!c) return APIC_OK;
  cudaSetDevice(c->device);
  Buf* all[] = {&c->cellb, &c->keys_a, &c->keys_b, &c->vals_a, &c->perm, &c->pt, &c->pn, &c->V, &c->D,
                &c->mup, &c->heads, &c->offs, &c->item_start, &c->item_info, &c->bflags, &c->boffs,
                &c->blist, &c->page, &c->gm, &c->gmask, &c->gp, &c->gp64, &c->gv, &c->gmb, &c->mu_pair,
                &c->cub_tmp, &c->h_x, &c->h_body, &c->h_v, &c->h_C, &c->h_m, &c->h_nrm, &c->h_vo, &c->h_Co};
  for (Buf* b : all) free_buf(c, *b);
  if (c->ds) cudaFree(c->ds);
  if (c->hs) cudaFreeHost(c->hs);
  for (auto e : c->ev_pool) cudaEventDestroy(e);
  delete c;
  return APIC_OK;
}

apic_status apic_contact_step(apic_ctx* c, const apic_step_args* a, void* stream, apic_stats* stats) {
  if (!c) return fail(APIC_ERR_INVALID_ARG, "ctx is NULL");
  APIC_TRY(validate(a));
  if (stats) std::memset(stats, 0, sizeof(*stats));
  if (a->n == 0) return APIC_OK;
  CUDA_TRY(cudaSetDevice(c->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  apic_status st = (a->flags & APIC_FP64) ? step_impl<double>(c, a, s, stats) : step_impl<float>(c, a, s, stats);
  if (st != APIC_OK) {
    // leave the stream usable: drop unfinished profile spans
    c->spans.clear();
    c->ev_used = 0;
  }
  return st;
}

apic_status apic_set_profiling(apic_ctx* c, int32_t on) {
  if (!c) return fail(APIC_ERR_INVALID_ARG, "ctx is NULL");
  APIC_TRY(harvest(c));
  c->prof_on = on != 0;
  c->prof = apic_profile{};
  return APIC_OK;
}

apic_status apic_get_profile(apic_ctx* c, apic_profile* out) {
  if (!c || !out) return fail(APIC_ERR_INVALID_ARG, "NULL argument");
  APIC_TRY(harvest(c));
  *out = c->prof;
  return APIC_OK;
}

apic_status apic_scratch_bytes(apic_ctx* c, size_t* out) {
  if (!c || !out) return fail(APIC_ERR_INVALID_ARG, "NULL argument");
  *out = c->held;
  return APIC_OK;
}

}  // extern "C"
