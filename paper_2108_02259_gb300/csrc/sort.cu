// Radix sort and exclusive scan of libapiccontact (sm_103a).
//
// The per-step sort orders particles by their key (grid block of the
// scene's page-table box, body, cell in block), so that every work item is
// a run of particles of one body in one grid block, cell by cell.  It is a
// stable least-significant-digit radix sort over the key's significant bits
// (end_bit), in passes of at most 9-bit digits:
//
//   k_radix_counts  one read of all keys: for every pass, how many keys have
//                   each digit value (the digit's first output position is
//                   the sum over smaller digits);
//   k_onesweep      one launch per pass.  Tiles take their index in launch
//                   order from a counter.  A tile ranks its keys among the
//                   keys of equal digit, warp by warp in index order (so the
//                   sort is stable), publishes its digit counts, and finds
//                   how many keys of each digit the tiles before it hold by
//                   looking back through their published counts ("decoupled
//                   look-back": a tile that has its own full prefix publishes
//                   it, so a look-back stops at the first such tile).  It
//                   then stages the tile in sorted order in shared memory and
//                   writes it out, runs of equal digits contiguous.
//
// A tile waits only for tiles that took their index before it (so they are
// running or done).  Each wait is bounded: a tile that gives up sets
// kErrSort in the call's error word, writes nothing, and still publishes a
// prefix so that no later tile waits on it; the host then fails the call.
//
// Values are the particles' original indices, so the sorted permutation is
// unique for given keys (ties keep index order).  The first pass takes its
// values as the index itself instead of reading them.
//
// The exclusive scan (run counts, block flags) is a reduce-then-scan in
// three launches: tile sums, one CTA scanning the tile sums, then every tile
// scanned from its offset.
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "apic_internal.h"

namespace apic {

#ifdef APIC_DEBUG_BOUNDS
__device__ unsigned g_dbg_sort;  // bounds-check bits of this translation unit
namespace {
__device__ __forceinline__ void dbg_record(unsigned bit) { atomicOr(&g_dbg_sort, bit); }
}  // namespace
#endif

unsigned sort_debug_flags(int clear) {
#ifdef APIC_DEBUG_BOUNDS
  unsigned v = 0;
  if (cudaMemcpyFromSymbol(&v, g_dbg_sort, sizeof(v)) != cudaSuccess) return ~0u;
  if (clear) {
    const unsigned z = 0;
    if (cudaMemcpyToSymbol(g_dbg_sort, &z, sizeof(z)) != cudaSuccess) return ~0u;
  }
  return v;
#else
  (void)clear;
  return 0;
#endif
}

namespace {

constexpr int kSortThreads = 512;  // one thread per digit value in a pass
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kRadixMaxBits = 9;
constexpr int kRadixBins = 1 << kRadixMaxBits;
constexpr int kBinsPerThread = kRadixBins / kSortThreads;
static_assert(kRadixBins % kSortThreads == 0, "each thread owns whole digits");
constexpr int kCountThreads = 256;  // CTA size of the count kernel

// Keys per thread and per tile: 32-bit keys 6 per thread (3072 a tile) or,
// from kBigSort keys on, 10 (5120 a tile: fewer tiles to look back over;
// measured on 4 M keys, 4.189 -> 4.161 ms a step, while at 200 k keys the
// smaller tiles keep more CTAs busy); 64-bit keys 4 (2048).  The tile is
// staged in dynamic shared memory.
constexpr int64_t kBigSort = int64_t(1) << 20;
template <class K, int ITEMS>
struct SortTile {
  static constexpr int kItems = ITEMS;
  static constexpr int kTile = kSortThreads * kItems;
  static constexpr int kWarpTile = 32 * kItems;
};
template <class K>
int sort_items(int64_t n) {
  return sizeof(K) == 4 ? (n >= kBigSort ? 10 : 6) : 4;
}

// Look-back status words: two flag bits over a 30-bit count (a scene holds
// at most 2^29 particles).
constexpr unsigned kStatAggregate = 1u << 30;  // this tile's own count
constexpr unsigned kStatPrefix = 2u << 30;     // count of this and every earlier tile
constexpr unsigned kStatValue = (1u << 30) - 1u;
constexpr int kLookbackSpins = 1 << 22;  // per status word, then the tile gives up

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// A status word carries its flag and its count together, and no other
// memory is read on the strength of it, so relaxed device-scope accesses are
// enough (no fences).
__device__ __forceinline__ void st_status(unsigned* p, unsigned v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_status(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Lanes of the warp whose digit equals this lane's, among the valid lanes
// (0 for an invalid lane).  Every lane of the warp must call it.
__device__ __forceinline__ unsigned digit_peers(unsigned d, bool valid) {
  const unsigned v = __ballot_sync(0xffffffffu, valid);
  const unsigned m = __match_any_sync(0xffffffffu, valid ? d : 0xffffffffu);
  return valid ? (m & v) : 0u;
}

template <class K>
__device__ __forceinline__ unsigned digit_of(K k, int shift, unsigned mask) {
  return (unsigned)(k >> shift) & mask;
}

// Digit counts of every pass: counts[p * kRadixBins + d].  Pass p covers
// bits [p per, p per + bits_p) with bits_p = min(per, end_bit - p per).
// Each thread reads kCountRun consecutive keys at a time and keeps, per
// pass, the current digit and its run length, adding a run to the CTA's
// shared histogram when the digit changes (the keys arrive in the caller's
// order, which is spatially coherent, so runs are long in the high digits).
constexpr int kMaxPasses = 8;  // 64-bit keys at 9 bits a pass
constexpr int kCountRun = 16;
template <class K>
__global__ void __launch_bounds__(kCountThreads) k_radix_counts(const K* __restrict__ keys, int64_t n, int end_bit,
                                                                 int per, int passes, int* __restrict__ counts) {
  __shared__ int cnt[kMaxPasses][kRadixBins];
  for (int i = threadIdx.x; i < passes * kRadixBins; i += kCountThreads) (&cnt[0][0])[i] = 0;
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * kCountThreads * kCountRun;
  for (int64_t c0 = ((int64_t)blockIdx.x * kCountThreads + threadIdx.x) * kCountRun; c0 < n; c0 += stride) {
    const int64_t c1 = c0 + kCountRun < n ? c0 + kCountRun : n;
    unsigned prev[kMaxPasses];
    int run[kMaxPasses];
#pragma unroll
    for (int p = 0; p < kMaxPasses; ++p) {
      prev[p] = 0u;
      run[p] = 0;
    }
    for (int64_t i = c0; i < c1; ++i) {
      const K k = keys[i];
#pragma unroll
      for (int p = 0; p < kMaxPasses; ++p) {
        if (p >= passes) break;
        const int shift = p * per;
        const int bits = end_bit - shift < per ? end_bit - shift : per;
        const unsigned d = digit_of(k, shift, (1u << bits) - 1u);
        if (run[p] > 0 && d != prev[p]) {
          atomicAdd(&cnt[p][prev[p]], run[p]);
          run[p] = 0;
        }
        prev[p] = d;
        ++run[p];
      }
    }
#pragma unroll
    for (int p = 0; p < kMaxPasses; ++p)
      if (p < passes && run[p] > 0) atomicAdd(&cnt[p][prev[p]], run[p]);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < passes * kRadixBins; i += kCountThreads)
    if ((&cnt[0][0])[i]) atomicAdd(&counts[i], (&cnt[0][0])[i]);
}

// Exclusive scan of one value per thread over a CTA of WARPS warps; also
// returns the total.  warp_tot holds WARPS + 1 ints.
template <int WARPS>
__device__ __forceinline__ int cta_exclusive_scan(int x, int* warp_tot, int* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_tot[w] = incl;
  __syncthreads();
  if (w == 0) {
    int t = lane < WARPS ? warp_tot[lane] : 0;
    int ti = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, ti, o);
      if (lane >= o) ti += y;
    }
    if (lane < WARPS) warp_tot[lane] = ti - t;  // exclusive warp offsets
    if (lane == WARPS - 1) warp_tot[WARPS] = ti;
  }
  __syncthreads();
  const int r = warp_tot[w] + incl - x;
  if (total) *total = warp_tot[WARPS];
  return r;
}

// One pass: keys (kin, vin) -> (kout, vout) by the digit [shift, shift +
// bits).  counts: this pass's digit counts over all keys; status: n_tiles *
// kRadixBins words and tile_ctr, zero on entry; vin == nullptr: the values
// are the indices.
template <class K, int ITEMS>
__global__ void __launch_bounds__(kSortThreads, 2)
    k_onesweep(const K* __restrict__ kin, const int* __restrict__ vin, K* __restrict__ kout, int* __restrict__ vout,
               int64_t n, int shift, int bits, const int* __restrict__ counts, unsigned* status, int* tile_ctr,
               int* err) {
  using TT = SortTile<K, ITEMS>;
  __shared__ uint16_t wcnt[kSortWarps][kRadixBins];  // per warp: keys of each digit so far, then warp offsets
  __shared__ int tstart[kRadixBins];            // the tile's count of each digit, then its first tile position
  __shared__ int gbase[kRadixBins];             // earlier tiles' keys of each digit, then its first output position
  __shared__ int scan_a[kSortWarps + 1], scan_b[kSortWarps + 1];
  __shared__ int s_tile, s_bad;
  // the staged tile in dynamic shared memory: keys, then values
  extern __shared__ __align__(16) unsigned char s_tile_dyn[];
  K* skey = reinterpret_cast<K*>(s_tile_dyn);
  int* sval = reinterpret_cast<int*>(s_tile_dyn + sizeof(K) * TT::kTile);
  const unsigned mask = (1u << bits) - 1u;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    s_tile = atomicAdd(tile_ctr, 1);  // tiles in the order their CTAs start
    s_bad = 0;
  }
  for (int i = threadIdx.x; i < kSortWarps * kRadixBins; i += kSortThreads) (&wcnt[0][0])[i] = 0;
  __syncthreads();
  const int tile = s_tile;
  const int64_t base = (int64_t)tile * TT::kTile;
  const int tile_n = (int)(n - base < TT::kTile ? n - base : TT::kTile);

  // Phase A: warp w ranks the keys [w kWarpTile, (w + 1) kWarpTile) of the
  // tile, 32 at a time in index order.
  K key[TT::kItems];
  int rank[TT::kItems];
#pragma unroll
  for (int r = 0; r < TT::kItems; ++r) {
    const int t = w * TT::kWarpTile + r * 32 + lane;
    key[r] = t < tile_n ? kin[base + t] : K(0);
  }
#pragma unroll
  for (int r = 0; r < TT::kItems; ++r) {
    const int t = w * TT::kWarpTile + r * 32 + lane;
    const bool valid = t < tile_n;
    const unsigned d = digit_of(key[r], shift, mask);
    const unsigned peers = digit_peers(d, valid);
    const int prior = valid ? (int)wcnt[w][d] : 0;
    rank[r] = prior + __popc(peers & lanemask_lt());
    __syncwarp();
    if (valid && lane == __ffs(peers) - 1) wcnt[w][d] = (uint16_t)(prior + __popc(peers));
    __syncwarp();
  }
  __syncthreads();

  // Phase B: for each digit (thread t owns t, t + kSortThreads, ...), the
  // warps' exclusive offsets and the tile's count; publish the count, look
  // back for the earlier tiles' total, publish this tile's prefix.
  int dtot[kBinsPerThread];
#pragma unroll
  for (int j = 0; j < kBinsPerThread; ++j) {
    const int d = threadIdx.x + j * kSortThreads;
    int run = 0;
#pragma unroll
    for (int q = 0; q < kSortWarps; ++q) {
      const int c = wcnt[q][d];
      wcnt[q][d] = (uint16_t)run;
      run += c;
    }
    dtot[j] = run;
    tstart[d] = run;
    if (d <= (int)mask)
      st_status(status + (int64_t)tile * kRadixBins + d, (tile == 0 ? kStatPrefix : kStatAggregate) | (unsigned)run);
  }
  // Look-back over a window of kWindow earlier tiles at a time, for all of
  // the thread's digits together: the status words of the window load at
  // once, then each digit folds them from the nearest tile back to the first
  // one that carries a full prefix (waiting, bounded, on any that has not
  // published yet).
  constexpr int kWindow = 16;
  {
    unsigned excl[kBinsPerThread];
    bool live[kBinsPerThread];
    bool ok = true;
#pragma unroll
    for (int j = 0; j < kBinsPerThread; ++j) {
      excl[j] = 0u;
      live[j] = tile > 0 && (int)(threadIdx.x + j * kSortThreads) <= (int)mask;
    }
    for (int t0 = tile - 1; t0 >= 0 && ok; t0 -= kWindow) {
      bool any = false;
#pragma unroll
      for (int j = 0; j < kBinsPerThread; ++j) any |= live[j];
      if (!any) break;
      unsigned v[kBinsPerThread][kWindow];
#pragma unroll
      for (int j = 0; j < kBinsPerThread; ++j)
#pragma unroll
        for (int q = 0; q < kWindow; ++q)
          v[j][q] = live[j] && t0 - q >= 0
                        ? ld_status(status + (int64_t)(t0 - q) * kRadixBins + threadIdx.x + j * kSortThreads)
                        : kStatPrefix;
#pragma unroll
      for (int j = 0; j < kBinsPerThread; ++j) {
#pragma unroll
        for (int q = 0; q < kWindow; ++q) {
          if (!live[j] || !ok) continue;
          int spins = 0;
          while ((v[j][q] & ~kStatValue) == 0u) {
            if (++spins > kLookbackSpins) {
              ok = false;  // give up: the tile writes nothing and the call fails
              break;
            }
            __nanosleep(32);
            v[j][q] = ld_status(status + (int64_t)(t0 - q) * kRadixBins + threadIdx.x + j * kSortThreads);
          }
          if (!ok) break;
          excl[j] += v[j][q] & kStatValue;
          if (v[j][q] & kStatPrefix) live[j] = false;
        }
      }
    }
    if (!ok) s_bad = 1;
#pragma unroll
    for (int j = 0; j < kBinsPerThread; ++j) {
      const int d = threadIdx.x + j * kSortThreads;
      // published even after giving up, so that no later tile waits here
      if (tile > 0 && d <= (int)mask)
        st_status(status + (int64_t)tile * kRadixBins + d, kStatPrefix | ((excl[j] + (unsigned)dtot[j]) & kStatValue));
      gbase[d] = (int)excl[j];
    }
  }
  __syncthreads();

  // Each digit's first output position (keys of smaller digits in the whole
  // input, then earlier tiles' keys of this digit) and first tile position
  // (exclusive scans over the digits; thread t owns kBinsPerThread
  // consecutive digits here).
  {
    int c[kBinsPerThread], tc[kBinsPerThread], cs = 0, ts = 0;
#pragma unroll
    for (int j = 0; j < kBinsPerThread; ++j) {
      const int d = threadIdx.x * kBinsPerThread + j;
      c[j] = d <= (int)mask ? counts[d] : 0;
      tc[j] = tstart[d];
      cs += c[j];
      ts += tc[j];
    }
    int g = cta_exclusive_scan<kSortWarps>(cs, scan_a, nullptr);
    int h = cta_exclusive_scan<kSortWarps>(ts, scan_b, nullptr);
#pragma unroll
    for (int j = 0; j < kBinsPerThread; ++j) {
      const int d = threadIdx.x * kBinsPerThread + j;
      gbase[d] += g;
      tstart[d] = h;
      g += c[j];
      h += tc[j];
    }
  }
  __syncthreads();
  if (s_bad) {
    if (threadIdx.x == 0) atomicOr(err, kErrSort);
    return;  // nothing written: the host fails the call
  }

  // Phase C: stage the tile in sorted order (values read here, so that they
  // hold no registers across the look-back).
#pragma unroll
  for (int r = 0; r < TT::kItems; ++r) {
    const int t = w * TT::kWarpTile + r * 32 + lane;
    if (t < tile_n) {
      const unsigned d = digit_of(key[r], shift, mask);
      const int pos = tstart[d] + wcnt[w][d] + rank[r];
      if (APIC_DBG_CHECK(pos >= 0 && pos < tile_n, kDbgSortPos)) {
        skey[pos] = key[r];
        sval[pos] = vin ? vin[base + t] : (int)(base + t);
      }
    }
  }
  __syncthreads();
  // Phase D: write out; consecutive threads write consecutive positions of a
  // digit's run.
  for (int i = threadIdx.x; i < tile_n; i += kSortThreads) {
    const K k = skey[i];
    const unsigned d = digit_of(k, shift, mask);
    const int64_t o = (int64_t)gbase[d] + (i - tstart[d]);
    if (APIC_DBG_CHECK(o >= 0 && o < n, kDbgSortPos)) {
      kout[o] = k;
      vout[o] = sval[i];
    }
  }
}

// ---- exclusive scan of int32 ----
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__global__ void __launch_bounds__(kScanThreads) k_scan_tile_sums(const int* __restrict__ in, int64_t n,
                                                                 int* __restrict__ sums) {
  __shared__ int red[kScanThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  int s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const int64_t idx = base + (int64_t)i * kScanThreads + threadIdx.x;
    if (idx < n) s += in[idx];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
#pragma unroll
    for (int q = 0; q < kScanThreads / 32; ++q) t += red[q];
    sums[blockIdx.x] = t;
  }
}

// One CTA: exclusive scan of the tile sums in place, in chunks of the CTA.
__global__ void __launch_bounds__(kScanThreads) k_scan_top(int* sums, int n_tiles) {
  __shared__ int warp_tot[kSortWarps + 1];
  int carry = 0;
  for (int c = 0; c < n_tiles; c += kScanThreads) {
    const int i = c + threadIdx.x;
    const int x = i < n_tiles ? sums[i] : 0;
    int total;
    const int e = cta_exclusive_scan<kScanThreads / 32>(x, warp_tot, &total);
    if (i < n_tiles) sums[i] = carry + e;
    carry += total;
    __syncthreads();
  }
}

// Each tile from its offset: out[i] = sums[tile] + exclusive sum within the
// tile.  Items are read before any is written (in == out allowed).
__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const int* in, int64_t n, const int* __restrict__ sums,
                                                             int* out) {
  __shared__ int warp_tot[kSortWarps + 1];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int x[kScanItems];
  int s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const int64_t idx = base + i;
    x[i] = idx < n ? in[idx] : 0;
    s += x[i];
  }
  int run = sums[blockIdx.x] + cta_exclusive_scan<kScanThreads / 32>(s, warp_tot, nullptr);
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const int64_t idx = base + i;
    if (idx < n) out[idx] = run;
    run += x[i];
  }
}

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace

// ------------------------------------------------------------ launchers --

int64_t scan_temp_ints(int64_t n) { return cdiv(n > 0 ? n : 1, kScanTile); }

cudaError_t launch_exclusive_scan(const int* in, int* out, int64_t n, int* temp, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int64_t tiles = cdiv(n, kScanTile);
  if (tiles > INT32_MAX) return cudaErrorInvalidValue;
  k_scan_tile_sums<<<(unsigned)tiles, kScanThreads, 0, s>>>(in, n, temp);
  k_scan_top<<<1, kScanThreads, 0, s>>>(temp, (int)tiles);
  k_scan_apply<<<(unsigned)tiles, kScanThreads, 0, s>>>(in, n, temp, out);
  return cudaGetLastError();
}

int radix_passes(int end_bit) { return end_bit <= 0 ? 0 : (end_bit + kRadixMaxBits - 1) / kRadixMaxBits; }

// temp layout (ints): digit counts [passes][kRadixBins], tile counters
// [32], look-back status [passes][tiles][kRadixBins]; all zeroed per sort.
template <class K>
int64_t radix_temp_ints(int64_t n, int end_bit) {
  const int64_t tiles = cdiv(n > 0 ? n : 1, (int64_t)kSortThreads * sort_items<K>(n));
  const int passes = radix_passes(end_bit) > 0 ? radix_passes(end_bit) : 1;
  return (int64_t)passes * kRadixBins + 32 + (int64_t)passes * tiles * kRadixBins;
}

// One pass of k_onesweep with ITEMS keys a thread.  Its shared memory (static
// plus the staged tile) can exceed 48 KB, which each device allows once per
// instantiation (the flag is per device ordinal; beyond kAttrDevices the
// attribute is set on every launch).
constexpr int kAttrDevices = 64;
template <class K, int ITEMS>
cudaError_t launch_onesweep(int64_t tiles, const K* kin, const int* vin, K* kout, int* vout, int64_t n, int shift,
                            int bits, const int* counts, unsigned* status, int* tile_ctr, int* err, cudaStream_t s) {
  static std::atomic<bool> attr_set[kAttrDevices];
  const size_t dyn = (size_t)SortTile<K, ITEMS>::kTile * (sizeof(K) + sizeof(int));
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const bool known = dev >= 0 && dev < kAttrDevices;
  if (!known || !attr_set[dev].load()) {
    e = cudaFuncSetAttribute(k_onesweep<K, ITEMS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
    if (known) attr_set[dev].store(true);
  }
  k_onesweep<K, ITEMS><<<(unsigned)tiles, kSortThreads, dyn, s>>>(kin, vin, kout, vout, n, shift, bits, counts, status,
                                                                   tile_ctr, err);
  return cudaGetLastError();
}

template <class K>
cudaError_t launch_radix_sort(K* keys, int* vals, K* keys_alt, int* vals_alt, int64_t n, int end_bit, bool vals_iota,
                              int* temp, int* err, cudaStream_t s) {
  const int passes = radix_passes(end_bit);
  if (n <= 0 || passes == 0) return cudaSuccess;
  const int items = sort_items<K>(n);
  const int64_t tiles = cdiv(n, (int64_t)kSortThreads * items);
  if (tiles > INT32_MAX / kRadixBins || n > (int64_t)kStatValue || passes > kMaxPasses) return cudaErrorInvalidValue;
  int* counts = temp;
  int* tile_ctr = counts + passes * kRadixBins;
  unsigned* status = reinterpret_cast<unsigned*>(tile_ctr + 32);
  cudaError_t e = cudaMemsetAsync(temp, 0, (size_t)radix_temp_ints<K>(n, end_bit) * sizeof(int), s);
  if (e != cudaSuccess) return e;
  // the digits spread evenly over the passes (each at most kRadixMaxBits)
  const int per = (end_bit + passes - 1) / passes;
  // up to 8 CTAs per SM: each adds its histograms to the global counts once
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = 8 * (int64_t)sms;
  const int64_t chunks = cdiv(n, (int64_t)kCountThreads * kCountRun);
  const int count_ctas = (int)(chunks < want ? chunks : want);
  k_radix_counts<K><<<count_ctas, kCountThreads, 0, s>>>(keys, n, end_bit, per, passes, counts);
  K *kin = keys, *kout = keys_alt;
  int *vin = vals, *vout = vals_alt;
  for (int p = 0; p < passes; ++p) {
    const int shift = p * per;
    const int bits = end_bit - shift < per ? end_bit - shift : per;
    const int* vp = (p == 0 && vals_iota) ? nullptr : vin;
    unsigned* st = status + (int64_t)p * tiles * kRadixBins;
    if (items == 10)
      e = launch_onesweep<K, 10>(tiles, kin, vp, kout, vout, n, shift, bits, counts + p * kRadixBins, st, tile_ctr + p,
                                 err, s);
    else if (items == 6)
      e = launch_onesweep<K, 6>(tiles, kin, vp, kout, vout, n, shift, bits, counts + p * kRadixBins, st, tile_ctr + p,
                                err, s);
    else
      e = launch_onesweep<K, 4>(tiles, kin, vp, kout, vout, n, shift, bits, counts + p * kRadixBins, st, tile_ctr + p,
                                err, s);
    if (e != cudaSuccess) return e;
    K* tk = kin;
    kin = kout;
    kout = tk;
    int* tv = vin;
    vin = vout;
    vout = tv;
  }
  return cudaSuccess;
}

template int64_t radix_temp_ints<uint32_t>(int64_t, int);
template int64_t radix_temp_ints<uint64_t>(int64_t, int);
template cudaError_t launch_radix_sort<uint32_t>(uint32_t*, int*, uint32_t*, int*, int64_t, int, bool, int*, int*,
                                                 cudaStream_t);
template cudaError_t launch_radix_sort<uint64_t>(uint64_t*, int*, uint64_t*, int*, int64_t, int, bool, int*, int*,
                                                 cudaStream_t);

}  // namespace apic
