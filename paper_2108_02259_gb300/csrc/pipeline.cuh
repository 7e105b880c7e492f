// The per-step pipeline of libapiccontact, shared by the context-backed
// entry points (api.cu) and the no-allocation entry point (static_step.cu).
//
// A call steps a batch of independent scenes (one scene is a batch of one):
//   1. cells + validation + per-scene bounding boxes      (k_cells)
//   2. per-scene page-table boxes laid end to end          (host, or reused)
//   3. keys and one radix sort over all scenes              (k_keys, sort.cu)
//   4. sorted SoA planes                                    (k_gather)
//   5. work items of <= chunk particles of one (block, body) (k_run_items,
//      scan, k_item_write)
//   6. active blocks and the page table                     (k_mark_items, scan, k_compact)
//   7. mass, body mask and P2G(V); optional friction blend; normalise
//   8. N + 1 fused transfer passes (Sec. 2.3 series, Sec. 2.4 projection)
// Everything runs on the caller's stream; the host synchronises while the
// sparse grid is sized (after 2 when no box can be reused, and after 6).
//
// The environment `Env` supplies device scratch by slot, a host mirror of
// the device counters, an optional per-scene box cache and profiling hooks.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <utility>
#include <vector>

#include "../../include/apiccontact.h"
#include "apic_internal.h"

namespace apic {

enum Slot : int {
  kSlotCells = 0, kSlotKeysA, kSlotKeysB, kSlotVals, kSlotPerm, kSlotPt, kSlotPn, kSlotV, kSlotD, kSlotMup,
  kSlotItemStart, kSlotItemInfo, kSlotBFlags, kSlotBOffs, kSlotBList, kSlotPage,
  kSlotGm, kSlotGmask, kSlotGp, kSlotGp64, kSlotGv, kSlotGmb, kSlotMuTable, kSlotSortTmp, kSlotScenes,
  kSlotSBbox, kSlotSMom, kSlotSCount, kSlotHX, kSlotHBody, kSlotHV, kSlotHC, kSlotHM, kSlotHN, kSlotHVo,
  kSlotHCo, kSlotDS, kSlotNrmAcc, kSlotNrmX, kSlotNrmTri, kSlotNrmOut, kSlotAugF, kSlotAugAm, kSlotAugVbar,
  kSlotAugVhat, kSlotAugChat, kSlotAugNrm, kSlotAugOut, kSlotRunCnt, kSlotRunOffs, kSlotRunEnd, kSlotFxMax,
  kSlotFxErr, kSlotGmbFx, kSlotTicket, kSlotHaloRep, kSlotPtc, kSlotCount
};

constexpr int kMaxBodies = 32;
constexpr int64_t kMaxPageEntries = int64_t(1) << 28;  // dense page table limit (1 GiB)
constexpr int kBoxSlack = 2;  // blocks of room for motion when a page-table box is reused

apic_status pfail(apic_status code, const char* fmt, ...);

// Grow-only scratch of a context, by slot (defined with the context).
apic_status ctx_take(apic_ctx* c, int slot, size_t bytes, void** out);

#define P_CUDA(expr)                                                                              \
  do {                                                                                            \
    cudaError_t e_ = (expr);                                                                      \
    if (e_ != cudaSuccess)                                                                        \
      return ::apic::pfail(e_ == cudaErrorMemoryAllocation ? APIC_ERR_OUT_OF_MEMORY : APIC_ERR_CUDA, \
                           "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, __LINE__);  \
  } while (0)

#define P_TRY(expr)               \
  do {                            \
    apic_status s_ = (expr);      \
    if (s_ != APIC_OK) return s_; \
  } while (0)

#define P_LAUNCH(env, expr) \
  do {                      \
    (env).launched();       \
    P_CUDA(expr);           \
  } while (0)

inline apic_status pfail(apic_status code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  set_last_error(buf);
  return code;
}

inline int bits_for(uint64_t v) {  // bits needed to represent 0..v
  int b = 0;
  while (b < 64 && (v >> b) != 0) ++b;
  return b;
}

// Checks shared by every entry point, for one scene.
inline apic_status validate_scene(const apic_step_args* a, int idx, uint32_t allowed_flags) {
  if (!a) return pfail(APIC_ERR_INVALID_ARG, "scene %d: args is NULL", idx);
  if (a->n < 0) return pfail(APIC_ERR_INVALID_ARG, "scene %d: n = %lld < 0", idx, (long long)a->n);
  if (a->n > (int64_t)INT32_MAX / 4)
    return pfail(APIC_ERR_INVALID_ARG, "scene %d: n = %lld exceeds the per-call limit %d", idx, (long long)a->n,
                 INT32_MAX / 4);
  if (a->n_bodies < 1 || a->n_bodies > kMaxBodies)
    return pfail(APIC_ERR_INVALID_ARG, "scene %d: n_bodies = %d outside [1, %d]", idx, a->n_bodies, kMaxBodies);
  if (a->n_iter < 0) return pfail(APIC_ERR_INVALID_ARG, "scene %d: n_iter = %d < 0", idx, a->n_iter);
  if (!(a->h > 0.0) || !std::isfinite(a->h))
    return pfail(APIC_ERR_INVALID_ARG, "scene %d: h = %g must be finite and > 0", idx, a->h);
  if (!(a->mu >= 0.0) || !std::isfinite(a->mu))
    return pfail(APIC_ERR_INVALID_ARG, "scene %d: mu = %g must be finite and >= 0", idx, a->mu);
  if (a->flags & ~allowed_flags)
    return pfail(APIC_ERR_INVALID_ARG, "scene %d: flag bits 0x%x not accepted here", idx, a->flags & ~allowed_flags);
  if (a->n > 0 && (!a->body || !a->x || !a->v || !a->C || !a->m || !a->v_out || !a->C_out ||
                   (!a->nrm && !(a->flags & APIC_MASS_NORMALS))))
    return pfail(APIC_ERR_INVALID_ARG, "scene %d: a required array pointer is NULL", idx);
  if (a->mu_pair) {
    const int nb = a->n_bodies;
    for (int i = 0; i < nb * nb; ++i)
      if (!(a->mu_pair[i] >= 0.0) || !std::isfinite(a->mu_pair[i]))
        return pfail(APIC_ERR_INVALID_ARG, "scene %d: mu_pair[%d] = %g must be finite and >= 0", idx, i,
                     a->mu_pair[i]);
    for (int i = 0; i < nb; ++i)
      for (int j = 0; j < nb; ++j)
        if (a->mu_pair[i * nb + j] != a->mu_pair[j * nb + i])
          return pfail(APIC_ERR_INVALID_ARG, "scene %d: mu_pair is not symmetric at (%d, %d)", idx, i, j);
  }
  return APIC_OK;
}

// Scratch of steps 3-6 for n particles and NB page-table entries.  Every
// buffer and every temporary size is fixed here, before any of those steps
// is enqueued, so that the enqueue sequence itself allocates nothing and
// assigns nothing (it may be captured once and replayed as a graph).
struct SizingBufs {
  int end_bit = 0;
  bool k64 = false;
  void *ka = nullptr, *kb = nullptr;  // key buffers (uint32_t or uint64_t); sorted keys end in kb
  int *va = nullptr, *perm = nullptr; // value buffers; the sorted permutation ends in perm
  int* tmp = nullptr;                  // sort and scan temporaries
  int *run_cnt = nullptr, *run_offs = nullptr, *run_end = nullptr;  // per run head: items, their offset, end
  int* item_start = nullptr;
  int4* item_info = nullptr;
  int *bflags = nullptr, *boffs = nullptr, *blist = nullptr, *page = nullptr;
};

template <class K, class Env>
apic_status plan_keys(Env& env, int64_t n, SizingBufs& b, int64_t* tmp_ints) {
  K *ka, *kb;
  P_TRY(env.take(kSlotKeysA, n, &ka, "sort keys"));
  P_TRY(env.take(kSlotKeysB, n, &kb, "sorted keys"));
  P_TRY(env.take(kSlotVals, n, &b.va, "sort values"));
  P_TRY(env.take(kSlotPerm, n, &b.perm, "permutation"));
  *tmp_ints = radix_temp_ints<K>(n, b.end_bit);
  b.ka = ka;
  b.kb = kb;
  return APIC_OK;
}

template <class Env>
apic_status plan_sizing(Env& env, int64_t n, int64_t NB, int max_bodies, SizingBufs& b) {
  b.end_bit = bits_for((uint64_t)NB * (uint64_t)max_bodies - 1) + 6;
  b.k64 = b.end_bit > 32;
  int64_t t_sort = 0;
  if (b.k64)
    P_TRY(plan_keys<uint64_t>(env, n, b, &t_sort));
  else
    P_TRY(plan_keys<uint32_t>(env, n, b, &t_sort));
  P_TRY(env.take(kSlotRunCnt, n, &b.run_cnt, "items per run"));
  P_TRY(env.take(kSlotRunOffs, n, &b.run_offs, "item offsets"));
  P_TRY(env.take(kSlotRunEnd, n, &b.run_end, "run ends"));
  P_TRY(env.take(kSlotItemStart, n, &b.item_start, "item starts"));
  P_TRY(env.take(kSlotItemInfo, n, &b.item_info, "item info"));
  P_TRY(env.take(kSlotBFlags, NB, &b.bflags, "block flags"));
  P_TRY(env.take(kSlotBOffs, NB, &b.boffs, "block offsets"));
  P_TRY(env.take(kSlotBList, NB, &b.blist, "block list"));
  P_TRY(env.take(kSlotPage, NB, &b.page, "page table"));
  const int64_t t = std::max(t_sort, std::max(scan_temp_ints(n), scan_temp_ints(NB)));
  P_TRY(env.take(kSlotSortTmp, (size_t)t, &b.tmp, "sort and scan temporaries"));
  return APIC_OK;
}

// Keys of every particle, then the radix sort; the sorted keys land in kb
// and the permutation in perm (the keys start in the buffer that makes the
// last pass end there).
// The buffer the keys start in (so that the last pass ends in kb).
inline void* first_keys(const SizingBufs& b) { return radix_passes(b.end_bit) % 2 == 1 ? b.ka : b.kb; }

// keys_ready: the cell kernel has already written the keys (reused boxes).
template <class K, class Env>
apic_status sort_keys(Env& env, int64_t n, const SceneDev* sc, int ns, const int4* cellb, int max_bodies,
                      int* err, const SizingBufs& b, bool keys_ready, cudaStream_t s) {
  const bool odd = radix_passes(b.end_bit) % 2 == 1;
  K* k0 = static_cast<K*>(first_keys(b));
  K* k1 = static_cast<K*>(odd ? b.kb : b.ka);
  int* v0 = odd ? b.va : b.perm;
  int* v1 = odd ? b.perm : b.va;
  if (!keys_ready) P_LAUNCH(env, launch_keys<K>(n, sc, ns, cellb, max_bodies, k0, v0, err, s));
  P_CUDA(launch_radix_sort<K>(k0, v0, k1, v1, n, b.end_bit, true, b.tmp, err, s));
  env.sorted();
  return APIC_OK;
}

template <class Env>
apic_status exclusive_sum(Env& env, const SizingBufs& b, const int* in, int* out, int64_t n, cudaStream_t s) {
  P_CUDA(launch_exclusive_scan(in, out, n, b.tmp, s));
  env.sorted();
  return APIC_OK;
}

// Steps `ns` scenes in one batch.  All scenes share the precision and
// variant flags of scene 0 and its n_iter (checked by the caller).
//
// With APIC_MASS_NORMALS the normals come from each body's grid mass
// (threshold nthr) after the mass pass instead of from the scenes' nrm.
// normals_only: stop after those normals and write them to each scene's
// v_out (caller order, [n*3]) instead of stepping (device pointers, no
// statistics).
template <class T, class Env>
apic_status run_batch(Env& env, const apic_step_args* scenes, int ns, cudaStream_t s, apic_stats* stats,
                      bool normals_only = false, double nthr = kMassNormalThreshold) {
  const uint32_t flags = scenes[0].flags;
  const bool host = (flags & APIC_HOST_PTRS) != 0;
  const bool det = (flags & APIC_DETERMINISTIC) != 0;
  const bool mnrm = normals_only || (flags & APIC_MASS_NORMALS) != 0;
  const int check = (flags & APIC_CHECK) ? 1 : 0;
  // partitions of one scene: their grids are summed where they share blocks
  const bool parts = (flags & APIC_PARTITIONED) != 0 && ns > 1;
  const int N = scenes[0].n_iter;
  if (normals_only && (host || stats)) return pfail(APIC_ERR_INVALID_ARG, "normals: device pointers, no statistics");
  if (det && sizeof(T) != 4)
    return pfail(APIC_ERR_INVALID_ARG, "APIC_DETERMINISTIC applies to the FP32 path (not with APIC_FP64)");
  typename Env::Span span_step(env, s, 0);
  typename Env::Span span_prep(env, s, 1);

  // Scene table: particle offsets, caller pointers (staged for host arrays).
  SceneDev* hsc = env.host_scenes(ns);
  if (!hsc) return pfail(APIC_ERR_OUT_OF_MEMORY, "no host staging for a table of %d scenes", ns);
  int64_t n = 0;
  int max_bodies = 1, n_mu = 0;
  bool any_mu = false;
  for (int i = 0; i < ns; ++i) {
    const apic_step_args& a = scenes[i];
    SceneDev d{};
    d.x = a.x;
    d.body = a.body;
    d.v = a.v;
    d.C = a.C;
    d.m = a.m;
    d.nrm = mnrm ? nullptr : a.nrm;  // computed on the device instead
    d.nthr = (float)nthr;
    d.v_out = a.v_out;
    d.C_out = a.C_out;
    d.part_off = n;
    d.n = (int)a.n;
    d.n_bodies = a.n_bodies;
    d.mu_off = -1;
    if (a.mu_pair) {
      d.mu_off = n_mu;
      n_mu += a.n_bodies * a.n_bodies;
      any_mu = true;
    }
    d.h = a.h;
    d.inv_h = 1.0 / a.h;
    d.mu = a.mu;
    hsc[i] = d;
    n += a.n;
    if (a.n_bodies > max_bodies) max_bodies = a.n_bodies;
  }
  if (stats) std::memset(stats, 0, sizeof(apic_stats) * ns);
  if (n == 0) return APIC_OK;
  if (n > (int64_t)INT32_MAX / 4)
    return pfail(APIC_ERR_INVALID_ARG, "the batch holds %lld particles, beyond the per-call limit %d", (long long)n,
                 INT32_MAX / 4);

  bool split_v = false;  // V planes gathered after the sizing sequence (see below)
  bool split_n = false;  // ... and the normals after the mass pass
  // CTAs of the copy that runs beside the sizing sequence (with four 16-byte
  // loads in flight per thread, 64 CTAs keep the host link full)
  constexpr int kSideCopyCtas = 64;
  if (host) {
    double* dx;
    int32_t* db;
    T *dv, *dC, *dm, *dn, *dvo, *dCo;
    P_TRY(env.take(kSlotHX, 3 * n, &dx, "staged x"));
    P_TRY(env.take(kSlotHBody, n, &db, "staged body"));
    P_TRY(env.take(kSlotHV, 3 * n, &dv, "staged v"));
    P_TRY(env.take(kSlotHC, 9 * n, &dC, "staged C"));
    P_TRY(env.take(kSlotHM, n, &dm, "staged m"));
    P_TRY(env.take(kSlotHN, 3 * n, &dn, "staged normals"));
    P_TRY(env.take(kSlotHVo, 3 * n, &dvo, "staged v_out"));
    P_TRY(env.take(kSlotHCo, 9 * n, &dCo, "staged C_out"));
    // Page-locked caller arrays are staged by table-driven copy kernels (the
    // host link is the limit either way, but per-copy overheads add up over
    // many scenes); otherwise, or when a table is not available, one copy
    // per array.  With a side stream, normals, v and C (60 of the 92 bytes
    // per FP32 particle) cross the link while the sizing sequence runs: only
    // the passes need them (split_v): v and C first (the mass pass needs
    // them), then the normals, which cross while the mass pass runs (only the
    // transfer passes read them: split_n).  Table layout: [0, 3 ns) x, body,
    // m (all six arrays in [0, 6 ns) without the side stream); [3 ns, 5 ns)
    // v, C; [5 ns, 6 ns) nrm; [6 ns, 8 ns) the results on the way back,
    // written while the side copies may still be reading their own entries.
    CopyEntry* tab = env.copy_table(8 * ns);
    bool direct = tab != nullptr;
    // (APIC_CHECK reads v, C and the normals in the cell kernel: no split)
    cudaStream_t side = direct && !check ? env.side_stream() : nullptr;
    int na = 0, nb = 0, nn = 0;
    long long max_a = 0, max_b = 0, max_n = 0;
    for (int i = 0; i < ns && direct; ++i) {
      const apic_step_args& a = scenes[i];
      const int64_t o = hsc[i].part_off, m = a.n;
      if (m == 0) continue;
      const std::pair<const void*, std::pair<void*, long long>> parts[6] = {
          {a.x, {dx + 3 * o, 3 * m * (long long)sizeof(double)}}, {a.body, {db + o, m * (long long)sizeof(int32_t)}},
          {a.m, {dm + o, m * (long long)sizeof(T)}},               {a.nrm, {dn + 3 * o, 3 * m * (long long)sizeof(T)}},
          {a.v, {dv + 3 * o, 3 * m * (long long)sizeof(T)}},      {a.C, {dC + 9 * o, 9 * m * (long long)sizeof(T)}}};
      for (int k = 0; k < 6; ++k) {
        if (k == 3 && mnrm) continue;  // no normals to stage
        const void* src = env.device_view(parts[k].first);
        if (!src) {
          direct = false;
          break;
        }
        const CopyEntry e{src, parts[k].second.first, parts[k].second.second};
        if (k < 3 || !side) {
          tab[na++] = e;
          max_a = std::max(max_a, e.bytes);
        } else if (k == 3) {
          tab[5 * ns + nn++] = e;
          max_n = std::max(max_n, e.bytes);
        } else {
          tab[3 * ns + nb++] = e;
          max_b = std::max(max_b, e.bytes);
        }
      }
    }
    split_v = direct && side != nullptr && nb > 0;
    split_n = split_v && nn > 0;
    if (direct) P_LAUNCH(env, launch_copy_table(tab, na, max_a, s));
    if (split_v) {
      // after the first copy (which the sizing sequence waits for, so the
      // two do not share the link) and everything queued before it
      P_CUDA(cudaEventRecord(env.side_event(0), s));
      P_CUDA(cudaStreamWaitEvent(side, env.side_event(0), 0));
      P_LAUNCH(env, launch_copy_table(tab + 3 * ns, nb, max_b, side, kSideCopyCtas));
      P_CUDA(cudaEventRecord(env.side_event(1), side));
      if (split_n) {
        P_LAUNCH(env, launch_copy_table(tab + 5 * ns, nn, max_n, side, kSideCopyCtas));
        P_CUDA(cudaEventRecord(env.side_event(2), side));
      }
    }
    for (int i = 0; i < ns; ++i) {
      const apic_step_args& a = scenes[i];
      const int64_t o = hsc[i].part_off, m = a.n;
      if (m == 0) continue;
      if (!direct) {
        P_CUDA(cudaMemcpyAsync(dx + 3 * o, a.x, 3 * m * sizeof(double), cudaMemcpyHostToDevice, s));
        P_CUDA(cudaMemcpyAsync(db + o, a.body, m * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        P_CUDA(cudaMemcpyAsync(dv + 3 * o, a.v, 3 * m * sizeof(T), cudaMemcpyHostToDevice, s));
        P_CUDA(cudaMemcpyAsync(dC + 9 * o, a.C, 9 * m * sizeof(T), cudaMemcpyHostToDevice, s));
        P_CUDA(cudaMemcpyAsync(dm + o, a.m, m * sizeof(T), cudaMemcpyHostToDevice, s));
        if (!mnrm) P_CUDA(cudaMemcpyAsync(dn + 3 * o, a.nrm, 3 * m * sizeof(T), cudaMemcpyHostToDevice, s));
      }
      hsc[i].x = dx + 3 * o;
      hsc[i].body = db + o;
      hsc[i].v = dv + 3 * o;
      hsc[i].C = dC + 9 * o;
      hsc[i].m = dm + o;
      hsc[i].nrm = mnrm ? nullptr : dn + 3 * o;
      hsc[i].v_out = dvo + 3 * o;
      hsc[i].C_out = dCo + 9 * o;
    }
  }

  // Kernel variant of this call (the autotuner's choice, or a variant it is
  // timing): its CTA size is also the largest work item the sizing makes.
  // (deterministic mode: variant 0, whose item split fixes the order of
  // every floating-point sum)
  const int variant = det ? env.variant_fixed() : env.variant(sizeof(T), n);
  const int chunk = kVariantChunk[sizeof(T) == 4 ? variant : 0];

  DevScalars* ds = env.ds();
  DevScalars* hs = env.hs();
  SceneDev* sc;
  int* sbbox;
  int4* cellb;
  P_TRY(env.take(kSlotScenes, ns, &sc, "scene table"));
  P_TRY(env.take(kSlotSBbox, 6 * ns, &sbbox, "scene boxes"));
  P_TRY(env.take(kSlotCells, n, &cellb, "cells"));
  V4<T>* ptc = nullptr;  // FP32 path: offsets and masses for the gather
  if (sizeof(T) == 4) P_TRY(env.take(kSlotPtc, n, &ptc, "cell offsets"));
  int* hbbox = env.host_bbox(ns);
  Box* boxes = env.box_cache(ns);  // persistent per-scene boxes (or scratch)

  int64_t NB = 0;
  V4<T> *pt, *pn, *V, *D;
  // 3-6 as one launch sequence (cells first when the box is reused): keys,
  // one radix sort over all scenes, sorted SoA, work items, active blocks
  // and the page table, then the device counters back to the host.  Only
  // enqueues work: every buffer comes from plan_sizing.
  SizingBufs sb;
  auto sizing = [&](cudaStream_t q, bool with_cells) -> apic_status {
    if (with_cells) {
      P_CUDA(cudaMemcpyAsync(ds, hs, sizeof(DevScalars), cudaMemcpyHostToDevice, q));
      P_CUDA(cudaMemcpyAsync(sc, hsc, ns * sizeof(SceneDev), cudaMemcpyHostToDevice, q));
      // the boxes are reused: the cell kernel writes the sort keys too
      P_LAUNCH(env, launch_cells<T>(n, sc, ns, cellb, ptc, sbbox, &ds->err, check, first_keys(sb), sb.k64 ? 8 : 4,
                                    max_bodies, q));
    }
    // 3. keys and one radix sort over all scenes.
    if (sb.k64)
      P_TRY((sort_keys<uint64_t>(env, n, sc, ns, cellb, max_bodies, &ds->err, sb, with_cells, q)));
    else
      P_TRY((sort_keys<uint32_t>(env, n, sc, ns, cellb, max_bodies, &ds->err, sb, with_cells, q)));
    // 4. sorted SoA (normals and V planes later when they are still in
    //    transit).
    P_LAUNCH(env, launch_gather<T>(n, sc, ns, sb.perm, ptc, sb.kb, sb.k64 ? 8 : 4, pt, pn,
                                   (split_v || normals_only) ? nullptr : V, q));
    // 5. work items: runs of equal (grid block, body), each split into
    //    equal items of at most `chunk` particles (the variant's CTA size).
    if (sb.k64) {
      const uint64_t* kb = static_cast<const uint64_t*>(sb.kb);
      P_LAUNCH(env, launch_run_items<uint64_t>(n, kb, chunk, sb.run_cnt, sb.run_end, q));
      P_TRY(exclusive_sum(env, sb, sb.run_cnt, sb.run_offs, n, q));
      P_LAUNCH(env, launch_item_write<uint64_t>(n, kb, sb.run_cnt, sb.run_offs, sb.run_end, max_bodies, sc, ns,
                                                sb.item_start, sb.item_info, &ds->n_items, q));
    } else {
      const uint32_t* kb = static_cast<const uint32_t*>(sb.kb);
      P_LAUNCH(env, launch_run_items<uint32_t>(n, kb, chunk, sb.run_cnt, sb.run_end, q));
      P_TRY(exclusive_sum(env, sb, sb.run_cnt, sb.run_offs, n, q));
      P_LAUNCH(env, launch_item_write<uint32_t>(n, kb, sb.run_cnt, sb.run_offs, sb.run_end, max_bodies, sc, ns,
                                                sb.item_start, sb.item_info, &ds->n_items, q));
    }
    // 6. active grid blocks: every block some stencil reaches; page table.
    P_CUDA(cudaMemsetAsync(sb.bflags, 0, NB * sizeof(int), q));
    if (sb.k64)
      P_LAUNCH(env, launch_mark_items<uint64_t>(sb.item_start, sb.item_info, &ds->n_items,
                                                static_cast<const uint64_t*>(sb.kb), n, (int)n, sc, sb.bflags, q));
    else
      P_LAUNCH(env, launch_mark_items<uint32_t>(sb.item_start, sb.item_info, &ds->n_items,
                                                static_cast<const uint32_t*>(sb.kb), n, (int)n, sc, sb.bflags, q));
    P_TRY(exclusive_sum(env, sb, sb.bflags, sb.boffs, NB, q));
    P_LAUNCH(env, launch_compact(NB, sb.bflags, sb.boffs, sb.blist, sb.page, &ds->n_blocks, q));
    P_CUDA(cudaMemcpyAsync(hs, ds, sizeof(DevScalars), cudaMemcpyDeviceToHost, q));
    return APIC_OK;
  };
  P_TRY(env.take(kSlotPt, n, &pt, "particle offsets"));
  P_TRY(env.take(kSlotPn, n, &pn, "particle normals"));
  P_TRY(env.take(kSlotV, 3 * n, &V, "sorted V"));
  P_TRY(env.take(kSlotD, 3 * n, &D, "Delta"));

  for (int attempt = 0;; ++attempt) {
    // 1. cells, validation, bounding boxes of particle blocks.
    const bool fresh = !env.have_box() || attempt > 0;
    *hs = DevScalars{};
    if (!fresh) {
      // boxes reused from the previous step: the whole sequence depends only
      // on the sizes below (and the buffers), so it may run as a graph
      NB = 0;
      for (int i = 0; i < ns; ++i) {
        hsc[i].box = boxes[i];
        hsc[i].page_off = NB;
        NB += (int64_t)hsc[i].box.nx * hsc[i].box.ny * hsc[i].box.nz;
      }
      struct SizingKey {
        int64_t n, NB;
        int ns, max_bodies, tsize, host, chunk, split_v, check, pad;
      } key;
      std::memset(&key, 0, sizeof(key));
      key.check = check;
      key.chunk = chunk;
      key.split_v = split_v ? 1 : 0;
      key.n = n;
      key.NB = NB;
      key.ns = ns;
      key.max_bodies = max_bodies;
      key.tsize = (int)sizeof(T);
      key.host = host ? 1 : 0;
      P_TRY(plan_sizing(env, n, NB, max_bodies, sb));
      auto body = [&](cudaStream_t q) -> apic_status { return sizing(q, true); };
      P_TRY(env.run_sizing(&key, sizeof(key), true, s, body));
    } else {
      for (int i = 0; i < ns; ++i) {
        int* b = hbbox + 6 * i;
        b[0] = b[1] = b[2] = INT32_MAX;
        b[3] = b[4] = b[5] = INT32_MIN;
      }
      P_CUDA(cudaMemcpyAsync(sbbox, hbbox, 6 * ns * sizeof(int), cudaMemcpyHostToDevice, s));
      P_CUDA(cudaMemcpyAsync(ds, hs, sizeof(DevScalars), cudaMemcpyHostToDevice, s));
      P_CUDA(cudaMemcpyAsync(sc, hsc, ns * sizeof(SceneDev), cudaMemcpyHostToDevice, s));
      P_LAUNCH(env, launch_cells<T>(n, sc, ns, cellb, ptc, sbbox, &ds->err, check, nullptr, 0, max_bodies, s));
      // 2. page-table boxes: one block of stencil margin plus kBoxSlack
      //    blocks of room for motion in later steps; laid end to end.
      P_CUDA(cudaMemcpyAsync(hbbox, sbbox, 6 * ns * sizeof(int), cudaMemcpyDeviceToHost, s));
      P_CUDA(cudaMemcpyAsync(hs, ds, sizeof(DevScalars), cudaMemcpyDeviceToHost, s));
      P_CUDA(cudaStreamSynchronize(s));
      if (hs->err) break;  // reported below
      const int g = 1 + kBoxSlack;
      NB = 0;
      for (int i = 0; i < ns; ++i) {
        const int* b = hbbox + 6 * i;
        Box bx{};
        if (hsc[i].n > 0) {
          bx.ox = b[0] - g;
          bx.oy = b[1] - g;
          bx.oz = b[2] - g;
          bx.nx = b[3] - b[0] + 1 + 2 * g;
          bx.ny = b[4] - b[1] + 1 + 2 * g;
          bx.nz = b[5] - b[2] + 1 + 2 * g;
        }
        hsc[i].box = bx;
        boxes[i] = bx;
        hsc[i].page_off = NB;
        NB += (int64_t)bx.nx * bx.ny * bx.nz;
        if (NB > kMaxPageEntries) {
          env.forget_box();
          return pfail(APIC_ERR_INVALID_ARG,
                       "the scenes span more than %lld grid blocks of 4^3 nodes (dense page-table limit)",
                       (long long)kMaxPageEntries);
        }
      }
      env.keep_box();
      P_CUDA(cudaMemcpyAsync(sc, hsc, ns * sizeof(SceneDev), cudaMemcpyHostToDevice, s));
      P_TRY(plan_sizing(env, n, NB, max_bodies, sb));
      P_TRY(sizing(s, false));
    }
    span_prep.stop();
    P_CUDA(cudaStreamSynchronize(s));
    if ((hs->err & kErrBox) && !(hs->err & ~kErrBox) && attempt == 0) {
      env.forget_box();  // a particle left a reused box: size fresh ones
      continue;
    }
    break;
  }
  const int* perm = sb.perm;
  const int* item_start = sb.item_start;
  const int4* item_info = sb.item_info;
  const int* page = sb.page;
  const int* blist = sb.blist;
  if (hs->err & kErrSort) {
    env.forget_box();
    return pfail(APIC_ERR_TIMEOUT, "the radix sort's bounded device-side wait gave up (no result was written)");
  }
  if (hs->err) {
    const int e = hs->err;
    env.forget_box();
    return pfail(APIC_ERR_INVALID_ARG, "invalid particle data:%s%s%s%s%s%s", (e & kErrBody) ? " body id out of range" : "",
                 (e & kErrMass) ? " mass not finite and > 0" : "",
                 (e & kErrPos) ? " position not finite or |x/h| >= 2^29" : "",
                 (e & kErrFinite) ? " v, C or normal not finite" : "",
                 (e & kErrNormal) ? " normal neither 0 nor of unit length" : "",
                 (e & kErrBox) ? " (internal: page-table box)" : "");
  }
  const int n_items = hs->n_items;
  const int n_blocks = hs->n_blocks;
  const int64_t n_nodes = (int64_t)n_blocks * kNodesPerBlock;

  // 7. node arrays; mass, body mask and P2G(V); friction blend; normalise.
  T* gm;
  uint32_t* gmask;
  V4<T>*gp, *gv;
  V4<double>* gp64 = nullptr;
  T* gmb = nullptr;
  T* mu_table = nullptr;
  T* mup = nullptr;
  P_TRY(env.take(kSlotGm, n_nodes, &gm, "grid mass"));
  P_TRY(env.take(kSlotGmask, n_nodes, &gmask, "grid body mask"));
  P_TRY(env.take(kSlotGp, n_nodes, &gp, "grid momentum"));
  P_TRY(env.take(kSlotGv, n_nodes, &gv, "grid velocity"));
  unsigned* ticket = nullptr;
  P_TRY(env.take(kSlotTicket, 1, &ticket, "item tickets"));
  int* halo_rep = nullptr;
  if (parts) P_TRY(env.take(kSlotHaloRep, std::max(n_blocks, 1), &halo_rep, "shared-block map"));
  if (sizeof(T) == 4) P_TRY(env.take(kSlotGp64, n_nodes, &gp64, "FP64 node momentum"));
  unsigned* fx_max = nullptr;
  int* fx_err = nullptr;
  long long* gmb_fx = nullptr;
  const int fx_stride = N + 2;
  if (det) {
    P_TRY(env.take(kSlotFxMax, (size_t)ns * fx_stride, &fx_max, "fixed-point bounds"));
    P_TRY(env.take(kSlotFxErr, (size_t)2 * (ns + 1), &fx_err, "fixed-point range flags"));
    if (any_mu || mnrm)
      P_TRY(env.take(kSlotGmbFx, (size_t)max_bodies * n_nodes, &gmb_fx, "per-body grid mass (fixed)"));
  }
  if (mnrm && !det) P_TRY(env.take(kSlotGmb, (size_t)max_bodies * n_nodes, &gmb, "per-body grid mass"));
  if (any_mu) {
    if (!det && !gmb) P_TRY(env.take(kSlotGmb, (size_t)max_bodies * n_nodes, &gmb, "per-body grid mass"));
    P_TRY(env.take(kSlotMuTable, (size_t)n_mu, &mu_table, "friction tables"));
    P_TRY(env.take(kSlotMup, n, &mup, "particle friction"));
    T* hmu = static_cast<T*>(env.host_buf((size_t)n_mu * sizeof(T)));
    if (!hmu) return pfail(APIC_ERR_INVALID_ARG, "friction tables too large for this entry point");
    for (int i = 0; i < ns; ++i)
      if (scenes[i].mu_pair)
        for (int k = 0; k < scenes[i].n_bodies * scenes[i].n_bodies; ++k)
          hmu[hsc[i].mu_off + k] = (T)scenes[i].mu_pair[k];
    P_CUDA(cudaMemcpyAsync(mu_table, hmu, (size_t)n_mu * sizeof(T), cudaMemcpyHostToDevice, s));
  }

  // The launch sequence from here to the end of the series depends only on
  // these values, so an environment may capture it once as a CUDA graph and
  // replay it while they stay the same.
  struct PassKey {
    IterParams<T> p;
    T* mup;
    int n_iter, any_mu, variant, split_v, split_n, mnrm, normals_only, parts;
  };
  PassKey key;
  std::memset(&key, 0, sizeof(key));  // padding bytes take part in the comparison
  IterParams<T>& p = key.p;
  p.n_items = n_items;
  p.n_particles = (int)n;
  p.max_bodies = max_bodies;
  p.n_scenes = ns;
  p.sc = sc;
  p.item_start = item_start;
  p.item_info = item_info;
  p.page = page;
  p.pt = pt;
  p.pn = pn;
  p.mup = nullptr;
  p.mu_table = mu_table;
  p.gmb = gmb;
  p.mup_out = mup;
  p.n_nodes = n_nodes;
  p.n_pages = NB;
  p.V = V;
  p.D = D;
  p.gv = gv;
  p.gp = gp;
  p.gm = gm;
  p.gmask = gmask;
  p.gp64 = gp64;
  p.perm = perm;
  p.pn_out = pn;
  p.normals_out = normals_only ? 1 : 0;
  p.pic = (flags & APIC_VARIANT_PIC) ? 1 : 0;
  p.sep23 = (flags & APIC_VARIANT_SEP23) ? 1 : 0;
  p.fx_max = fx_max;
  p.fx_err = fx_err;
  p.gmb_fx = gmb_fx;
  p.fx_stride = fx_stride;
  p.fold_mu = 0;
  p.ticket = ticket;
  key.mup = mup;
  key.n_iter = N;
  key.any_mu = any_mu ? 1 : 0;
  key.variant = variant;
  key.split_v = split_v ? 1 : 0;
  key.split_n = split_n ? 1 : 0;
  key.mnrm = mnrm ? 1 : 0;
  key.normals_only = normals_only ? 1 : 0;
  key.parts = parts ? 1 : 0;

  auto series = [&](cudaStream_t q) -> apic_status {
    IterParams<T> pp = key.p;
    const int var = key.variant;
    if (split_v) P_LAUNCH(env, launch_gather_v<T>(n, sc, ns, perm, pn, V, split_n ? 1 : 3, q));
    // every launch after the mass pass follows a k_items or k_normalize launch
    const bool ov = env.overlap();
    typename Env::Span span_mass(env, q, 3);
    P_CUDA(cudaMemsetAsync(gm, 0, n_nodes * sizeof(T), q));
    P_CUDA(cudaMemsetAsync(gmask, 0, n_nodes * sizeof(uint32_t), q));
    P_CUDA(cudaMemsetAsync(ticket, 0, sizeof(unsigned), q));
    if (parts) P_LAUNCH(env, launch_halo_map(n_blocks, blist, sc, ns, page, halo_rep, q));
    // the ghost sum over grid blocks that several partitions share, after a
    // particle-to-grid transfer and before the normalisation
    auto halo = [&](bool mass) -> cudaError_t {
      return launch_halo_sum<T>(n_blocks, halo_rep, gp, gp64, gm, gmask, gmb, max_bodies, n_nodes, mass, q);
    };
    P_CUDA(cudaMemsetAsync(gp, 0, n_nodes * sizeof(V4<T>), q));
    if (gp64) P_CUDA(cudaMemsetAsync(gp64, 0, n_nodes * sizeof(V4<double>), q));
    if (gmb) P_CUDA(cudaMemsetAsync(gmb, 0, (size_t)max_bodies * n_nodes * sizeof(T), q));
    // deterministic mode: the fixed-point sums live in gp64's storage as
    // int64 (x, y, z, mass); bounds and this attempt's range flags start at 0
    long long* gfx = reinterpret_cast<long long*>(gp64);
    if (det) {
      if (gmb_fx) P_CUDA(cudaMemsetAsync(gmb_fx, 0, (size_t)max_bodies * n_nodes * sizeof(long long), q));
      P_CUDA(cudaMemsetAsync(fx_max, 0, (size_t)ns * fx_stride * sizeof(unsigned), q));
      P_CUDA(cudaMemsetAsync(fx_err + pp.fx_attempt * (ns + 1), 0, (ns + 1) * sizeof(int), q));
      P_LAUNCH(env, launch_fx_prep(n, sc, ns, perm, reinterpret_cast<const V4<float>*>(pt),
                                   reinterpret_cast<const V4<float>*>(V), fx_max, fx_stride,
                                   fx_err + pp.fx_attempt * (ns + 1), q));
    }
    auto normalize = [&](int slot, int all64) -> cudaError_t {
      if (det)
        return launch_normalize_fx(n_nodes, blist, sc, ns, reinterpret_cast<float*>(gm), gfx,
                                   reinterpret_cast<V4<float>*>(gv), fx_max, fx_err, fx_stride, slot,
                                   pp.fx_attempt, all64, ov, q);
      return launch_normalize<T>(n_nodes, gm, gmask, gp, gp64, gv, all64, ov, q);
    };
    if (normals_only) P_CUDA(cudaMemsetAsync(V, 0, 3 * n * sizeof(V4<T>), q));  // (the mass pass reads V)
    P_LAUNCH(env, launch_items<T>(pp, kModeMassV, var, false, q));
    if (parts) P_LAUNCH(env, halo(true));
    // the per-pair friction blend: a pass of its own, or (FP32 default path
    // with transfer passes) computed by the first pass from the node masks it
    // fetches with its tile and written for the passes after it
    const bool fold_mu = any_mu && sizeof(T) == 4 && !det && N > 0;
    if (any_mu && !fold_mu) {
      P_LAUNCH(env, launch_items<T>(pp, kModeMu, var, ov, q));
      pp.mup = mup;
    }
    if (mnrm) {
      // normals into the sorted pn plane (or the callers' arrays).  The
      // passes read pn before their dependent-launch wait, so this grid and
      // the normalisation after it launch without overlap: every later grid
      // starts after the normals are complete.
      P_LAUNCH(env, launch_items<T>(pp, kModeNormals, var, false, q));
      if (normals_only) return APIC_OK;
    }
    if (mnrm) {
      if (det)
        P_LAUNCH(env, launch_normalize_fx(n_nodes, blist, sc, ns, reinterpret_cast<float*>(gm), gfx,
                                          reinterpret_cast<V4<float>*>(gv), fx_max, fx_err, fx_stride, 1,
                                          pp.fx_attempt, 1, false, q));
      else
        P_LAUNCH(env, launch_normalize<T>(n_nodes, gm, gmask, gp, gp64, gv, 1, false, q));
    } else {
      P_LAUNCH(env, normalize(1, 1));
    }
    span_mass.stop();

    // Staged normals that crossed the link during the mass pass: wait for
    // their copy (in a captured graph, as an external event) and gather them;
    // the first transfer pass then launches without overlap, since it reads
    // the normals before its dependent-launch wait.
    if (split_n) {
      cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
      P_CUDA(cudaStreamIsCapturing(q, &cs));
      P_CUDA(cudaStreamWaitEvent(q, env.side_event(2),
                                 cs == cudaStreamCaptureStatusActive ? cudaEventWaitExternal : cudaEventWaitDefault));
      P_LAUNCH(env, launch_gather_v<T>(n, sc, ns, perm, pn, V, 2, q));
    }

    // 8. the N + 1 transfer passes.
    for (int pass = 0; pass <= N; ++pass) {
      const int mode = N == 0 ? kModeOnly : pass == 0 ? kModeFirst : pass == N ? kModeLast : kModeMid;
      pp.fx_slot = 1 + pass;  // bound of the W this pass scatters, measured by the pass before
      pp.fold_mu = fold_mu && pass == 0 ? 1 : 0;
      if (fold_mu && pass == 1) pp.mup = mup;  // written by the first pass
      {
        typename Env::Span span_pass(env, q, 2);
        P_LAUNCH(env, launch_items<T>(pp, mode, var, ov && !(pass == 0 && split_n), q));
      }
      if (pass < N && parts) P_LAUNCH(env, halo(false));
      if (pass < N) P_LAUNCH(env, normalize(1 + pass, 0));
    }
    return APIC_OK;
  };
  if (split_v) P_CUDA(cudaStreamWaitEvent(s, env.side_event(1), 0));  // v and C staged
  P_TRY(env.run_series(&key, sizeof(key), s, series));
  if (det) {
    // A pass whose terms outgrew the headroom of its fixed-point scale left
    // every scene's outputs untouched: repeat the series once with a wider
    // headroom for the scenes concerned (the sorted inputs are unchanged; the
    // others compute the same bits again).
    std::vector<int> bad(ns);
    for (int attempt = 0;; ++attempt) {
      P_CUDA(cudaMemcpyAsync(bad.data(), fx_err + attempt * (ns + 1), ns * sizeof(int), cudaMemcpyDeviceToHost,
                             s));
      P_CUDA(cudaStreamSynchronize(s));
      int first_bad = -1;
      for (int i = 0; i < ns && first_bad < 0; ++i)
        if (bad[i]) first_bad = i;
      if (first_bad < 0) break;
      if (attempt == 1)
        return pfail(APIC_ERR_INVALID_ARG,
                     "scene %d: deterministic mode: node sums outgrew their fixed-point range "
                     "(non-finite inputs, or terms growing by more than 2^%d within one pass)",
                     first_bad, kFxRetryHeadLog2);
      key.p.fx_attempt = 1;
      P_TRY(env.run_series(&key, sizeof(key), s, series));
    }
  }
  span_step.stop();

  if (stats) {
    double* smom;
    unsigned long long* scount;
    // per scene: (P, L, E) of the inputs, then of the outputs
    P_TRY(env.take(kSlotSMom, 14 * ns, &smom, "scene momenta"));
    P_TRY(env.take(kSlotSCount, 3 * ns, &scount, "scene counts"));
    P_CUDA(cudaMemsetAsync(smom, 0, 14 * ns * sizeof(double), s));
    P_CUDA(cudaMemsetAsync(scount, 0, 3 * ns * sizeof(unsigned long long), s));
    for (int i = 0; i < ns; ++i) {
      const SceneDev& d = hsc[i];
      if (d.n == 0) continue;
      const double* x = d.x;
      const T* m = static_cast<const T*>(d.m);
      P_LAUNCH(env, launch_momentum<T>(d.n, x, static_cast<const T*>(d.v), static_cast<const T*>(d.C), m, d.h,
                                       smom + 14 * i, s));
      P_LAUNCH(env, launch_momentum<T>(d.n, x, static_cast<const T*>(d.v_out), static_cast<const T*>(d.C_out),
                                       m, d.h, smom + 14 * i + 7, s));
    }
    P_LAUNCH(env, launch_scene_counts(n_blocks, blist, gmask, n_items, item_info, sc, ns, scount, s));
    double* hm = static_cast<double*>(env.host_buf(14 * ns * sizeof(double) + 3 * ns * sizeof(unsigned long long)));
    if (!hm) return pfail(APIC_ERR_INVALID_ARG, "too many scenes for statistics on this entry point");
    unsigned long long* hc = reinterpret_cast<unsigned long long*>(hm + 14 * ns);
    P_CUDA(cudaMemcpyAsync(hm, smom, 14 * ns * sizeof(double), cudaMemcpyDeviceToHost, s));
    P_CUDA(cudaMemcpyAsync(hc, scount, 3 * ns * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    P_CUDA(cudaStreamSynchronize(s));
    for (int i = 0; i < ns; ++i) {
      for (int k = 0; k < 3; ++k) {
        stats[i].P_in[k] = hm[14 * i + k];
        stats[i].L_in[k] = hm[14 * i + 3 + k];
        stats[i].P_out[k] = hm[14 * i + 7 + k];
        stats[i].L_out[k] = hm[14 * i + 10 + k];
      }
      stats[i].E_in = hm[14 * i + 6];
      stats[i].E_out = hm[14 * i + 13];
      stats[i].multibody_nodes = (int64_t)hc[3 * i];
      stats[i].active_blocks = (int64_t)hc[3 * i + 1];
      stats[i].work_items = (int64_t)hc[3 * i + 2];
    }
  }
  if (host) {
    // results back: one table-driven kernel into page-locked outputs (the
    // table's last 2 ns entries; the input copies used the first ones and
    // finished before the mid-step synchronisation), else one copy each
    CopyEntry* tab = env.copy_table(8 * ns);
    bool direct = tab != nullptr;
    int nt = 0;
    long long max_bytes = 0;
    CopyEntry* out = direct ? tab + 6 * ns : nullptr;
    for (int i = 0; i < ns && direct; ++i) {
      const apic_step_args& a = scenes[i];
      if (a.n == 0) continue;
      void* dvo = const_cast<void*>(env.device_view(a.v_out));
      void* dCo = const_cast<void*>(env.device_view(a.C_out));
      if (!dvo || !dCo) {
        direct = false;
        break;
      }
      out[nt++] = CopyEntry{hsc[i].v_out, dvo, 3 * a.n * (long long)sizeof(T)};
      out[nt++] = CopyEntry{hsc[i].C_out, dCo, 9 * a.n * (long long)sizeof(T)};
      max_bytes = std::max(max_bytes, 9 * a.n * (long long)sizeof(T));
    }
    if (direct) {
      P_LAUNCH(env, launch_copy_table(out, nt, max_bytes, s));
    } else {
      for (int i = 0; i < ns; ++i) {
        const apic_step_args& a = scenes[i];
        if (a.n == 0) continue;
        P_CUDA(cudaMemcpyAsync(a.v_out, hsc[i].v_out, 3 * a.n * sizeof(T), cudaMemcpyDeviceToHost, s));
        P_CUDA(cudaMemcpyAsync(a.C_out, hsc[i].C_out, 9 * a.n * sizeof(T), cudaMemcpyDeviceToHost, s));
      }
    }
    P_CUDA(cudaStreamSynchronize(s));
  }
  env.done(n, n_nodes);
  return APIC_OK;
}

}  // namespace apic
