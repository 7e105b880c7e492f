// Radix sort and exclusive scan of libapiccontact (sm_103a).
//
// The per-step sort orders particles by their key (grid block of the
// scene's page-table box, body, cell in block), so that every work item is
// a run of particles of one body in one grid block, cell by cell.  It is a
// stable least-significant-digit radix sort over the key's significant bits
// (end_bit), with digits of at most 8 bits, three launches per digit:
//
//   k_radix_hist     per tile of keys, the count of every digit value
//                    (digit-major table hist[d * n_tiles + tile]);
//   scan             exclusive sum of that table: the output position of the
//                    first key of digit d in tile t (all keys of smaller
//                    digits, then those of digit d in earlier tiles);
//   k_radix_scatter  each key's rank among the keys of its digit in its tile
//                    (warp by warp, in index order, so the sort is stable),
//                    the tile staged in shared memory in sorted order, then
//                    written out with runs of equal digits contiguous.
//
// Values are the particles' original indices, so the sorted permutation is
// unique for given keys (ties keep index order).  The first pass takes its
// values as the index itself instead of reading them.
//
// The exclusive scan (run counts, block flags, the digit tables) is a
// reduce-then-scan in three launches: tile sums, one CTA scanning the tile
// sums, then every tile scanned from its offset.  No kernel waits on another
// CTA; every launch depends only on the launches before it in the stream.
#include <cuda_runtime.h>
#include <stdint.h>

#include "apic_internal.h"

namespace apic {
namespace {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kRadixMaxBits = 8;
constexpr int kRadixBins = 1 << kRadixMaxBits;
static_assert(kSortThreads == kRadixBins, "phase B of the scatter gives each thread one digit");

// Keys per thread and per tile: 32-bit keys 16 per thread (4096 a tile),
// 64-bit keys 8 (2048), so that the tile's staging stays in static shared
// memory (48 KB).
template <class K>
struct SortTile {
  static constexpr int kItems = sizeof(K) == 4 ? 16 : 8;
  static constexpr int kTile = kSortThreads * kItems;
  static constexpr int kWarpTile = 32 * kItems;
};

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Lanes of the warp whose digit equals this lane's, among the valid lanes
// (0 for an invalid lane): one ballot per digit bit.  Every lane of the warp
// must call it (bits is the same on all lanes).
__device__ __forceinline__ unsigned digit_peers(unsigned d, int bits, bool valid) {
  unsigned peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
  for (int b = 0; b < kRadixMaxBits; ++b) {
    if (b < bits) {
      const unsigned set = __ballot_sync(0xffffffffu, (d >> b) & 1u);
      peers &= ((d >> b) & 1u) ? set : ~set;
    }
  }
  return valid ? peers : 0u;
}

template <class K>
__device__ __forceinline__ unsigned digit_of(K k, int shift, unsigned mask) {
  return (unsigned)(k >> shift) & mask;
}

template <class K>
__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const K* __restrict__ keys, int64_t n, int shift,
                                                              int bits, int n_tiles, int* __restrict__ hist) {
  using TT = SortTile<K>;
  __shared__ int cnt[kRadixBins];
  const unsigned mask = (1u << bits) - 1u;
  const int tile = blockIdx.x;
  for (int d = threadIdx.x; d < kRadixBins; d += kSortThreads) cnt[d] = 0;
  __syncthreads();
  const int64_t base = (int64_t)tile * TT::kTile;
  const int lane = threadIdx.x & 31;
#pragma unroll 4
  for (int i = 0; i < TT::kItems; ++i) {
    const int64_t idx = base + (int64_t)i * kSortThreads + threadIdx.x;
    const bool valid = idx < n;
    const unsigned d = valid ? digit_of(keys[idx], shift, mask) : 0u;
    // one shared atomic per distinct digit of the warp
    const unsigned peers = digit_peers(d, bits, valid);
    if (valid && lane == __ffs(peers) - 1) atomicAdd(&cnt[d], __popc(peers));
  }
  __syncthreads();
  for (int d = threadIdx.x; d <= (int)mask; d += kSortThreads) hist[(int64_t)d * n_tiles + tile] = cnt[d];
}

// Exclusive scan of one value per thread over the CTA (kSortThreads); also
// returns the total.
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
    int t = lane < kSortWarps ? warp_tot[lane] : 0;
    int ti = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, ti, o);
      if (lane >= o) ti += y;
    }
    if (lane < kSortWarps) warp_tot[lane] = ti - t;  // exclusive warp offsets
    if (lane == kSortWarps - 1) warp_tot[kSortWarps] = ti;
  }
  __syncthreads();
  const int r = warp_tot[w] + incl - x;
  if (total) *total = warp_tot[kSortWarps];
  return r;
}

template <class K>
__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(const K* __restrict__ kin, const int* __restrict__ vin,
                                                                 K* __restrict__ kout, int* __restrict__ vout,
                                                                 int64_t n, int shift, int bits, int n_tiles,
                                                                 const int* __restrict__ hist) {
  using TT = SortTile<K>;
  __shared__ int wcnt[kSortWarps][kRadixBins];  // per warp: keys of each digit so far, then offsets
  __shared__ int tstart[kRadixBins];            // first tile position of each digit
  __shared__ int gbase[kRadixBins];             // output position of the tile's first key of each digit
  __shared__ int warp_tot[kSortWarps + 1];
  __shared__ K skey[TT::kTile];
  __shared__ int sval[TT::kTile];
  const unsigned mask = (1u << bits) - 1u;
  const int tile = blockIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < kSortWarps * kRadixBins; i += kSortThreads) (&wcnt[0][0])[i] = 0;
  __syncthreads();
  const int64_t base = (int64_t)tile * TT::kTile;
  const int tile_n = (int)(n - base < TT::kTile ? n - base : TT::kTile);
  // Phase A: warp w ranks the keys [w kWarpTile, (w + 1) kWarpTile) of the
  // tile, 32 at a time in index order.
  K key[TT::kItems];
  int val[TT::kItems];
  int rank[TT::kItems];
#pragma unroll
  for (int r = 0; r < TT::kItems; ++r) {
    const int t = w * TT::kWarpTile + r * 32 + lane;
    const bool valid = t < tile_n;
    key[r] = valid ? kin[base + t] : K(0);
    val[r] = valid ? (vin ? vin[base + t] : (int)(base + t)) : 0;
    const unsigned d = digit_of(key[r], shift, mask);
    const unsigned peers = digit_peers(d, bits, valid);
    const int prior = valid ? wcnt[w][d] : 0;
    rank[r] = prior + __popc(peers & lanemask_lt());
    __syncwarp();
    if (valid && lane == __ffs(peers) - 1) wcnt[w][d] = prior + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // Phase B: per digit, exclusive offsets of the warps, the tile's digit
  // runs (exclusive scan over digits) and the output base of each run.
  int dtot = 0;
  {
    const int d = threadIdx.x;  // kSortThreads == kRadixBins
    int run = 0;
#pragma unroll
    for (int q = 0; q < kSortWarps; ++q) {
      const int c = wcnt[q][d];
      wcnt[q][d] = run;
      run += c;
    }
    dtot = run;
    gbase[d] = d <= (int)mask ? hist[(int64_t)d * n_tiles + tile] : 0;
  }
  tstart[threadIdx.x] = cta_exclusive_scan(dtot, warp_tot, nullptr);
  __syncthreads();
  // Phase C: stage the tile in sorted order.
#pragma unroll
  for (int r = 0; r < TT::kItems; ++r) {
    const int t = w * TT::kWarpTile + r * 32 + lane;
    if (t < tile_n) {
      const unsigned d = digit_of(key[r], shift, mask);
      const int pos = tstart[d] + wcnt[w][d] + rank[r];
      skey[pos] = key[r];
      sval[pos] = val[r];
    }
  }
  __syncthreads();
  // Phase D: write out; consecutive threads write consecutive positions of a
  // digit's run.
  for (int i = threadIdx.x; i < tile_n; i += kSortThreads) {
    const K k = skey[i];
    const unsigned d = digit_of(k, shift, mask);
    const int64_t o = (int64_t)gbase[d] + (i - tstart[d]);
    kout[o] = k;
    vout[o] = sval[i];
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
    const int e = cta_exclusive_scan(x, warp_tot, &total);
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
  int run = sums[blockIdx.x] + cta_exclusive_scan(s, warp_tot, nullptr);
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

template <class K>
int64_t radix_temp_ints(int64_t n, int end_bit) {
  const int64_t tiles = cdiv(n > 0 ? n : 1, SortTile<K>::kTile);
  const int64_t hist = tiles * kRadixBins;
  return hist + scan_temp_ints(hist);
}

template <class K>
cudaError_t launch_radix_sort(K* keys, int* vals, K* keys_alt, int* vals_alt, int64_t n, int end_bit, bool vals_iota,
                              int* temp, cudaStream_t s) {
  const int passes = radix_passes(end_bit);
  if (n <= 0 || passes == 0) return cudaSuccess;
  const int64_t tiles = cdiv(n, SortTile<K>::kTile);
  if (tiles * kRadixBins > INT32_MAX) return cudaErrorInvalidValue;
  int* hist = temp;
  int* scan_tmp = temp + tiles * kRadixBins;
  // spread the bits evenly over the passes (each <= 8)
  const int per = (end_bit + passes - 1) / passes;
  K *kin = keys, *kout = keys_alt;
  int *vin = vals, *vout = vals_alt;
  for (int p = 0, shift = 0; p < passes; ++p) {
    const int bits = end_bit - shift < per ? end_bit - shift : per;
    const int64_t nh = tiles * ((int64_t)1 << bits);
    k_radix_hist<K><<<(unsigned)tiles, kSortThreads, 0, s>>>(kin, n, shift, bits, (int)tiles, hist);
    cudaError_t e = launch_exclusive_scan(hist, hist, nh, scan_tmp, s);
    if (e != cudaSuccess) return e;
    k_radix_scatter<K><<<(unsigned)tiles, kSortThreads, 0, s>>>(kin, (p == 0 && vals_iota) ? nullptr : vin, kout,
                                                                 vout, n, shift, bits, (int)tiles, hist);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    K* tk = kin;
    kin = kout;
    kout = tk;
    int* tv = vin;
    vin = vout;
    vout = tv;
    shift += bits;
  }
  return cudaSuccess;
}

template int64_t radix_temp_ints<uint32_t>(int64_t, int);
template int64_t radix_temp_ints<uint64_t>(int64_t, int);
template cudaError_t launch_radix_sort<uint32_t>(uint32_t*, int*, uint32_t*, int*, int64_t, int, bool, int*,
                                                 cudaStream_t);
template cudaError_t launch_radix_sort<uint64_t>(uint64_t*, int*, uint64_t*, int*, int64_t, int, bool, int*,
                                                 cudaStream_t);

}  // namespace apic
