// Internal types and launchers of libapiccontact (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace apic {

// 4-wide vector with natural alignment (16 B for float, 32 B for double).
template <class T>
struct alignas(4 * sizeof(T)) V4 {
  T x, y, z, w;
};

// The background grid is stored in blocks of 4x4x4 nodes.  A work item is
// the run of sorted particles whose cell lies in one grid block and that
// belong to one body.  Its particles touch nodes [4B-1, 4B+5] per dimension:
// a 7x7x7 node tile spanning the 3x3x3 blocks around B.
constexpr int kBlk = 4;
constexpr int kTile = 7;
constexpr int kTile3 = kTile * kTile * kTile;
constexpr int kNodesPerBlock = kBlk * kBlk * kBlk;
// A work item holds at most kChunk particles; each kernel variant has its
// own largest item (kVariantChunk).
#ifndef APIC_CHUNK
#define APIC_CHUNK 256
#endif
constexpr int kChunk = APIC_CHUNK;

// Error bits raised by the validation pass.
constexpr int kErrBody = 1;
constexpr int kErrMass = 2;
constexpr int kErrPos = 4;
constexpr int kErrBox = 8;  // a particle lies outside a page-table box reused from an earlier step
constexpr int kErrFinite = 16;  // v, C or a normal not finite (checked with APIC_CHECK)
constexpr int kErrNormal = 32;  // a normal neither 0 nor of unit length (checked with APIC_CHECK)
constexpr int kErrSort = 64;    // a bounded wait of the radix sort gave up (internal)

// Bounds checks of the kernels' own indexing (a debug build: compiled with
// -DAPIC_DEBUG_BOUNDS; build.build(debug=True) makes libapiccontact_debug.so).
// A failed check records its bit in the translation unit's debug word and
// the access is skipped (no trap, no fault); apic_debug_flags reads and
// clears the words.  In the normal build every check is `true`.
constexpr unsigned kDbgTileNode = 1;  // a tile node outside the node arrays
constexpr unsigned kDbgPage = 2;      // a page-table index outside the table
constexpr unsigned kDbgSlot = 4;      // an item size or a particle's cell bits out of range
constexpr unsigned kDbgPerm = 8;      // a permutation entry outside its scene
constexpr unsigned kDbgSortPos = 16;  // a sort output position outside the keys
#ifdef APIC_DEBUG_BOUNDS
#define APIC_DBG_CHECK(cond, bit) ((cond) ? true : (::apic::dbg_record(bit), false))
#else
#define APIC_DBG_CHECK(cond, bit) true
#endif
// Debug words of the kernel and sort translation units (0 in the normal
// build); clear: reset them.
unsigned kernels_debug_flags(int clear);
unsigned sort_debug_flags(int clear);

// Device-side scalars the host reads back while sizing the grid.
struct DevScalars {
  int err;       // kErr* bits
  int n_items;   // work items
  int n_blocks;  // active grid blocks
  int n_runs;    // runs of equal (grid block, body)
};

// Dense page table over a box of grid blocks (block coordinates relative to
// the box origin).  The box has a one-block margin around every particle
// block so that a particle's stencil never leaves it.
struct Box {
  int ox, oy, oz;  // origin block coordinates
  int nx, ny, nz;  // extent in blocks
};

// One scene of a batch as the kernels see it.  Scenes are independent: each
// has its own grid spacing, friction and page-table box; their boxes are
// laid end to end in one page table and their particles end to end in one
// index space.
struct SceneDev {
  const double* x;
  const int32_t* body;
  const void* v;
  const void* C;
  const void* m;
  const void* nrm;
  void* v_out;
  void* C_out;
  long long part_off;  // first particle of the scene in the batch
  long long page_off;  // first page-table entry of the scene's box
  int n;
  int n_bodies;
  int mu_off;          // offset of the scene's body-pair friction table, or -1
  float nthr;          // normals from the grid mass: surface where |grad rho| h > nthr rho
  Box box;
  int pad2[2];
  double h, inv_h, mu;
};

// Iteration-kernel modes (one transfer pair each; Sec. 2.3).  The numbers
// appear in profiles; 0 and 1 are not used.
enum Mode : int {
  kModeFirst = 2,  // G2P -> Delta_0 = H V - V -> W_1 -> P2G(W_1)
  kModeMid = 3,    // G2P -> Delta_m = Delta_{m-1} + H W_m - W_m -> W_{m+1} -> P2G
  kModeLast = 4,   // G2P -> Delta_N -> V_hat = V + Delta_N in caller order
  kModeOnly = 5,   // N = 0: G2P -> V_hat = H V in caller order
  kModeMu = 6,     // per-particle friction blend from a body-pair table
  kModeMassV = 7,  // m_i, body mask and P2G of V in one pass (momentum to FP64)
  kModeNormals = 8,  // normals from each body's grid mass (needs the per-body node masses)
};

// Normals from a body's grid mass: a particle is on the surface where the
// gradient of its body's interpolated grid mass, times h, exceeds this
// fraction of the interpolated mass (about the outermost layer of a
// lattice at node spacing h/2).
constexpr double kMassNormalThreshold = 0.5;

// Everything the per-item kernel needs, by value.
template <class T>
struct IterParams {
  int n_items;
  int n_particles;
  int max_bodies;          // key multiplier: bodies of the largest scene
  int n_scenes;
  const SceneDev* sc;      // [n_scenes]
  const int* item_start;   // [n_items] first sorted particle of each item
  const int4* item_info;   // [n_items] (global page index of the block, body, scene, 0)
  const int* page;         // page table: compact block id or -1
  const V4<T>* pt;         // [n] (t_x, t_y, t_z, m) sorted
  const V4<T>* pn;         // [n] (n_x, n_y, n_z, local cell bits) sorted
  const T* mup;            // [n] per-particle mu or nullptr (then the scene's mu)
  const T* mu_table;       // concatenated body-pair friction tables (kModeMu)
  T* gmb;                  // [max_bodies * nodes] per-body node mass, or nullptr
  T* mup_out;              // [n] written by kModeMu
  int64_t n_nodes;
  int64_t n_pages;         // page-table entries (bounds checks of the debug build)
  const V4<T>* V;          // [3n] sorted V = (v, h C) as 3 planes of n
  V4<T>* D;                // [3n] Delta planes
  const V4<T>* gv;         // grid velocity (normalised), [nodes]
  V4<T>* gp;               // grid momentum accumulators, [nodes]
  T* gm;                   // grid mass, [nodes]
  uint32_t* gmask;         // body bits, [nodes]
  V4<double>* gp64;        // FP64 momentum at multi-body nodes (FP32 path), [nodes]
  const int* perm;         // sorted -> batch particle index
  V4<T>* pn_out;           // kModeNormals: sorted normals written here (the pn plane) ...
  int normals_out;         // ... or, when set, into each scene's v_out in caller order
  int pic;                 // PIC transfers
  int sep23;               // Sec. 2.3 rule
  // Fixed-point node sums (deterministic mode): per scene, fx_max[scene *
  // fx_stride + k] holds the float bits of a bound on the particle terms a
  // pass scatters (k = 0: masses, 1: V, 2 + j: W of pass j); fx_err[attempt
  // * (n_scenes + 1) + scene] is set when a term exceeded the bound its scale
  // allowed, and fx_err[attempt * (n_scenes + 1) + n_scenes] when that
  // happened in any scene; gmb_fx replaces gmb.  The pass's own slot is
  // fx_slot.
  unsigned* fx_max;
  int* fx_err;
  long long* gmb_fx;
  int fx_stride;
  int fx_slot;
  int fx_attempt;
  // FP32 default path: the first transfer pass computes each particle's
  // per-pair friction blend itself (from the node masks it fetches with its
  // tile) and writes it to mup_out for the later passes, instead of a
  // separate blend pass before it.
  int fold_mu;
  // Persistent grids: a counter of item tickets, 0 between launches (the
  // launch draws exactly n_items tickets and atomicInc wraps it back to 0).
  unsigned* ticket;
};

// Deterministic mode: fixed-point headroom (log2) of a pass's scale over the
// bound measured in the pass before, first try and retry.
constexpr int kFxHeadLog2 = 12;
constexpr int kFxRetryHeadLog2 = 24;

// Cells, validation, per-scene bounding boxes of particle blocks (sbbox[6 s]).
template <class T>
// check: also validate v, C and the normals (APIC_CHECK).
// ptc (FP32 path, else NULL): each particle's offset in its cell and mass,
// (t_x, t_y, t_z, m) in caller order, for the gather.  keys (NULL, or with
// every scene's page-table box already in sc): the sort keys of k_keys
// (key_bytes 4 or 8) instead of the cells, so that k_keys is not needed.
cudaError_t launch_cells(int64_t n, const SceneDev* sc, int ns, int4* cellb, V4<T>* ptc, int* sbbox, int* err,
                         int check, void* keys, int key_bytes, int max_bodies, cudaStream_t s);
template <class K>
cudaError_t launch_keys(int64_t n, const SceneDev* sc, int ns, const int4* cellb, int max_bodies, K* keys,
                        int* vals, int* err, cudaStream_t s);
// V == nullptr: pt and pn's cell bits only (launch_gather_v fills the
// normals and V later).
template <class T>
// With ptc, pt comes from it and the cell-in-block bits from the sorted keys
// (key_bytes 4 or 8); without (FP64 path), both are recomputed from x.
cudaError_t launch_gather(int64_t n, const SceneDev* sc, int ns, const int* perm, const V4<T>* ptc, const void* skeys,
                          int key_bytes, V4<T>* pt, V4<T>* pn, V4<T>* V, cudaStream_t s);
// what: 1 the V planes, 2 the normals, 3 both.
template <class T>
cudaError_t launch_gather_v(int64_t n, const SceneDev* sc, int ns, const int* perm, V4<T>* pn, V4<T>* V,
                            int what, cudaStream_t s);
// Work items from the sorted keys: at each run head (a new (grid block,
// body)) the run's end and its item count ceil(len / chunk) (16 <= chunk <=
// kChunk), 0 elsewhere; then, with the exclusive sum of the counts, every
// item's start (equal split of its run) and (global page index, body, scene,
// 0), and the item count.
template <class K>
cudaError_t launch_run_items(int64_t n, const K* keys, int chunk, int* cnt, int* rend, cudaStream_t s);
template <class K>
cudaError_t launch_item_write(int64_t n, const K* keys, const int* cnt, const int* off, const int* rend,
                              int max_bodies, const SceneDev* sc, int ns, int* item_start, int4* item_info,
                              int* n_items, cudaStream_t s);
cudaError_t launch_compact(int64_t n, const int* flags, const int* offs, int* list, int* page,
                           int* count, cudaStream_t s);
template <class K>
cudaError_t launch_mark_items(const int* item_start, const int4* item_info, const int* n_items, const K* keys,
                              int64_t n, int max_items, const SceneDev* sc, int* flags, cudaStream_t s);
// Variants of the fused transfer kernel: CTA size, particles per thread in
// phase 1 (= stencil rows per lane in phase 2, "RPL"), the largest work item
// (CTA size x RPL), resident CTAs per SM it is compiled for (its register
// cap), and how P2G lanes get their row weights m N_y N_z (recomputed per
// lane from t, or read from factors stashed per particle in phase 1: fewer
// instructions, one more stash row), and whether the grid is persistent
// (as many CTAs as fit on the device at once, each walking items with a grid
// stride) or one CTA per item.  Variant 0 is the default; the FP32 path
// exists in all of them, the FP64 path in variant 0 only (which it always
// uses).
constexpr int kNumVariants = 9;
constexpr int kVariantThreads[kNumVariants] = {128, 128, 128, 64, 64, 128, 128, 128, 128};
constexpr int kVariantRPL[kNumVariants] = {1, 1, 1, 1, 1, 1, 1, 2, 1};
constexpr int kVariantChunk[kNumVariants] = {128, 128, 128, 64, 64, 128, 128, 256, 128};
constexpr int kVariantMinBlocks[kNumVariants] = {8, 9, 7, 13, 16, 8, 7, 5, 9};
constexpr bool kVariantRowTab[kNumVariants] = {false, false, false, false, false, true, true, false, false};
constexpr bool kVariantPersist[kNumVariants] = {false, false, false, false, false, false, false, false, true};
// overlap: launch with programmatic stream serialization, so that the grid's
// prologue (item metadata, particle loads, page lookups) runs while the grid
// before it finishes.  Only for a launch that directly follows another
// k_items or k_normalize launch in the same stream.
template <class T>
cudaError_t launch_items(const IterParams<T>& p, int mode, int variant, bool overlap, cudaStream_t s);
// Partitions of one scene (APIC_PARTITIONED): rep[cb] = the compact id of
// block cb's copy in the lowest-numbered partition where the same grid
// block is active, or -1 (cb is that copy, or no other partition has it).
cudaError_t launch_halo_map(int n_blocks, const int* blist, const SceneDev* sc, int ns, const int* page, int* rep,
                            cudaStream_t s);
// The ghost sum over those copies, in two launches: every copy's node sums
// (momentum, its FP64 accumulators, and with `mass` the mass, body mask and
// per-body masses) added into its representative, then the totals copied
// back to every copy.
template <class T>
cudaError_t launch_halo_sum(int n_blocks, const int* rep, V4<T>* gp, V4<double>* gp64, T* gm, uint32_t* gmask,
                            T* gmb, int max_bodies, int64_t n_nodes, bool mass, cudaStream_t s);
// all64: take every node's momentum from the FP64 accumulators (after kModeMassV).
template <class T>
cudaError_t launch_normalize(int64_t n_nodes, const T* gm, const uint32_t* gmask, V4<T>* gp,
                             V4<double>* gp64, V4<T>* gv, int all64, bool overlap, cudaStream_t s);
// Deterministic mode (FP32 path).  fx_prep: per scene, bounds of the mass and
// V terms of the mass pass (fx_max slots 0 and 1, zeroed by the caller);
// err_row[scene] is set where a bound is not finite.
cudaError_t launch_fx_prep(int64_t n, const SceneDev* sc, int ns, const int* perm, const V4<float>* pt,
                           const V4<float>* V, unsigned* fx_max, int fx_stride, int* err_row, cudaStream_t s);
// v_i from the fixed-point sums of the pass that used scale slot `slot`
// (all64: after the mass pass, which also gives m_i); clears the sums.
cudaError_t launch_normalize_fx(int64_t n_nodes, const int* blist, const SceneDev* sc, int ns, float* gm,
                                long long* gfx, V4<float>* gv, const unsigned* fx_max, const int* fx_err,
                                int fx_stride, int slot, int attempt, int all64, bool overlap, cudaStream_t s);
// FP64 totals of one scene: out7 = (P, L, E).
template <class T>
cudaError_t launch_momentum(int64_t n, const double* x, const T* v, const T* C, const T* m, double h,
                            double* out7, cudaStream_t s);
// Per-scene counts: out[3 s] = (multi-body nodes, active blocks, work items).
cudaError_t launch_scene_counts(int n_blocks, const int* blist, const uint32_t* gmask, int n_items,
                                const int4* item_info, const SceneDev* sc, int ns, unsigned long long* out,
                                cudaStream_t s);

// x += dt v for n particles (x double, v in T).
template <class T>
cudaError_t launch_advect(int64_t n, double* x, const T* v, double dt, cudaStream_t s);

// Sec. 2.3 node normals: FP64 area-weighted face-normal sums (acc[3 n],
// zeroed by the caller; err |= kErrBody for a bad index), then unit normals.
cudaError_t launch_face_normals(int64_t n_tri, const int32_t* tri, const double* x, int64_t n, double* acc,
                                int* err, cudaStream_t s);
template <class T>
cudaError_t launch_unit_normals(int64_t n, const double* acc, T* out, cudaStream_t s);

// Augury dynamics kernels (see kernels.cu): kick + drift, FP64 spring
// forces (err |= kErrBody for a bad index), prediction, finish, energies.
template <class T>
cudaError_t launch_aug_kick_drift(int64_t n, double* x, T* v, T* C, const T* av, const T* aC, const uint8_t* fixed,
                                  T half_dt, double dt, cudaStream_t s);
cudaError_t launch_aug_springs(int64_t n_springs, const int32_t* springs, const double* rest, const double* k,
                               const double* x, int64_t n, double* f, int* err, cudaStream_t s);
template <class T>
cudaError_t launch_aug_predict(int64_t n, const double* f, const T* m, const double* g, const T* v, T* am, T* vbar,
                               T c_bar, cudaStream_t s);
template <class T>
cudaError_t launch_aug_finish(int64_t n, const T* am, const T* vbar, const T* vhat, const T* Chat,
                              const uint8_t* fixed, T inv_tau, T half_dt, T* v, T* C, T* av, T* aC,
                              cudaStream_t s);
template <class T>
cudaError_t launch_aug_energy(int64_t n, const double* x, const T* v, const T* m, const double* g, int64_t n_springs,
                              const int32_t* springs, const double* rest, const double* k, double* out,
                              cudaStream_t s);

// Stable LSD radix sort of (key, value) pairs over the low end_bit bits of
// the keys (sort.cu): radix_passes(end_bit) passes of at most 9 bits, each
// from (keys, vals) to (keys_alt, vals_alt) and back, so the result is in
// (keys_alt, vals_alt) when the pass count is odd and in (keys, vals) when it
// is even.  vals_iota: the input values are the indices 0..n-1 (not read).
// temp holds radix_temp_ints<K>(n, end_bit) ints.  A bounded device-side
// wait that gives up sets kErrSort in *err (the sorted output is then not
// valid).
int radix_passes(int end_bit);
template <class K>
int64_t radix_temp_ints(int64_t n, int end_bit);
template <class K>
cudaError_t launch_radix_sort(K* keys, int* vals, K* keys_alt, int* vals_alt, int64_t n, int end_bit,
                              bool vals_iota, int* temp, int* err, cudaStream_t s);
// Exclusive sum of n ints (in == out allowed); temp holds scan_temp_ints(n)
// ints.
int64_t scan_temp_ints(int64_t n);
cudaError_t launch_exclusive_scan(const int* in, int* out, int64_t n, int* temp, cudaStream_t s);

// One copy of `bytes` bytes between device-visible addresses (device memory
// or page-locked host memory seen through its device pointer).
struct CopyEntry {
  const void* src;
  void* dst;
  long long bytes;
  long long chunk0;  // with a CTA budget: the entry's first chunk (set by launch_copy_table)
};
// All copies of a table (itself device-visible) in one launch.
// max_ctas > 0: at most that many CTAs, each taking an equal share of the
// entries' bytes, for a copy that runs beside compute kernels (CTAs that
// wait on the host link hold SM slots the compute kernels need).  The table
// is then host memory: its chunk0 fields are filled here.
cudaError_t launch_copy_table(CopyEntry* table, int n_entries, long long max_bytes, cudaStream_t s,
                              int max_ctas = 0);

// Set the calling thread's message returned by apic_last_error().
void set_last_error(const char* msg);

}  // namespace apic
