// CUDA kernels of libapiccontact (sm_103a).
//
// The per-step pipeline (host side in api.cu):
//   cells -> keys -> radix sort -> gather SoA -> item heads -> grid-block
//   activation -> mass P2G -> P2G(V) -> N+1 fused transfer passes, each
//   followed by a node normalisation (v_i = p_i / m_i).
//
// Notation follows the paper: particles p, background nodes i, weights N_i
// (App. B), generalized velocity V = {v, B} with B_p = C_p D_p and
// D_p = (h^2/2) I, the series V_hat = V + G V + sum G W_n (Sec. 2.3) and the
// undesirable part of Sec. 2.4.  Inside the kernels C is carried as
// Ch = h C (velocity units) and node offsets in cell units d = (x_i - x_p)/h,
// so P2G adds N m (v + Ch d) and G2P gives Ch_hat = 2 sum N v_i (x) d.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <type_traits>

#include "apic_internal.h"

namespace apic {

#ifdef APIC_DEBUG_BOUNDS
__device__ unsigned g_dbg_kernels;  // bounds-check bits of this translation unit
namespace {
__device__ __forceinline__ void dbg_record(unsigned bit) { atomicOr(&g_dbg_kernels, bit); }
}  // namespace
#endif

unsigned kernels_debug_flags(int clear) {
#ifdef APIC_DEBUG_BOUNDS
  unsigned v = 0;
  if (cudaMemcpyFromSymbol(&v, g_dbg_kernels, sizeof(v)) != cudaSuccess) return ~0u;
  if (clear) {
    const unsigned z = 0;
    if (cudaMemcpyToSymbol(g_dbg_kernels, &z, sizeof(z)) != cudaSuccess) return ~0u;
  }
  return v;
#else
  (void)clear;
  return 0;
#endif
}

namespace {

__device__ __forceinline__ float bits_to(float, uint32_t b) { return __uint_as_float(b); }
__device__ __forceinline__ double bits_to(double, uint32_t b) {
  return __longlong_as_double((long long)b);
}
__device__ __forceinline__ uint32_t to_bits(float v) { return __float_as_uint(v); }
__device__ __forceinline__ uint32_t to_bits(double v) { return (uint32_t)__double_as_longlong(v); }

// Programmatic dependent launch (sm_90 and later).  A grid launched with the
// programmatic-serialization attribute may start while the grid before it in
// the stream still runs; grid_dep_wait() returns once every grid it depends
// on has completed with its memory visible, and grid_dep_launch() lets the
// next grid start.  Both do nothing in a grid launched without the attribute.
// Before grid_dep_wait() a kernel reads only what the grid-sizing sequence
// wrote (which completed before the first grid of the chain started) and
// writes nothing to global memory.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

// App. B quadratic B-spline weights of the nodes i-1, i, i+1, i+2 for the
// in-cell offset t = x/h - floor(x/h), written out (with the 1/4 factor on
// the middle two, the reading under which they sum to one):
//   (1-t)^2/4,  (2-t^2)/4,  (1+2t-t^2)/4,  t^2/4
// and the node offsets d_k = (x_{i-1+k} - x_p)/h = k - 1 - t.
template <class T>
__device__ __forceinline__ void bspline(T t, T w[4], T d[4]) {
  const T s = T(1) - t;
  w[0] = T(0.25) * s * s;
  w[1] = T(0.25) * (T(2) - t * t);
  w[2] = T(0.25) * (T(1) + t * (T(2) - t));
  w[3] = T(0.25) * t * t;
  d[0] = -T(1) - t;
  d[1] = -t;
  d[2] = T(1) - t;
  d[3] = T(2) - t;
}

// Derivatives of the same four weights with respect to t (cell units):
//   -(1-t)/2,  -t/2,  (1-t)/2,  t/2.
template <class T>
__device__ __forceinline__ void bspline_grad(T t, T g[4]) {
  g[0] = -T(0.5) * (T(1) - t);
  g[1] = -T(0.5) * t;
  g[2] = T(0.5) * (T(1) - t);
  g[3] = T(0.5) * t;
}

// Sec. 2.4: the undesirable part of the proposed change (dv, dCh).  dCh is
// always undesirable; dv loses its admissible part inside the Coulomb cone
// when dv.n <= 0.  With sep23 the Sec. 2.3 rule is used instead.
template <class T>
__device__ __forceinline__ void undesirable(const T dv[3], const T dC[9], const T n[3], T mu,
                                            int sep23, T wv[3], T wC[9]) {
  const T dn = dv[0] * n[0] + dv[1] * n[1] + dv[2] * n[2];
  if (sep23) {
    const T f = dn > T(0) ? T(1) : T(0);
#pragma unroll
    for (int a = 0; a < 3; ++a) wv[a] = f * dv[a];
#pragma unroll
    for (int a = 0; a < 9; ++a) wC[a] = f * dC[a];
    return;
  }
  if (dn <= T(0)) {
    T vt[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) vt[a] = dv[a] - dn * n[a];
    // the admissible tangential part keeps min(|vt|, -mu dn) / |vt| of vt
    T keep;
    if constexpr (sizeof(T) == 4) {
      // FP32: min(1, -mu dn / |vt|) with the reciprocal square root
      // (rsqrtf: no IEEE square root and divide, whose slow paths branch);
      // |vt|^2 below the smallest normal float is taken at that floor
      const float nt2 = vt[0] * vt[0] + vt[1] * vt[1] + vt[2] * vt[2];
      keep = nt2 > 0.f ? fminf(1.f, -mu * dn * rsqrtf(fmaxf(nt2, 1.17549435e-38f))) : 0.f;
    } else {
      const T nt = sqrt(vt[0] * vt[0] + vt[1] * vt[1] + vt[2] * vt[2]);
      const T s = fmin(nt, -mu * dn);
      keep = nt > T(0) ? s / nt : T(0);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) wv[a] = vt[a] - keep * vt[a];
  } else {
#pragma unroll
    for (int a = 0; a < 3; ++a) wv[a] = dv[a];
  }
#pragma unroll
  for (int a = 0; a < 9; ++a) wC[a] = dC[a];
}

template <class T>
__device__ __forceinline__ void load12(const V4<T>* planes, int n, int s, T v[3], T C[9]) {
  const V4<T> a = planes[s], b = planes[n + s], c = planes[2 * n + s];
  v[0] = a.x; v[1] = a.y; v[2] = a.z;
  C[0] = a.w; C[1] = b.x; C[2] = b.y;
  C[3] = b.z; C[4] = b.w; C[5] = c.x;
  C[6] = c.y; C[7] = c.z; C[8] = c.w;
}

template <class T>
__device__ __forceinline__ void store12(V4<T>* planes, int n, int s, const T v[3], const T C[9]) {
  planes[s] = V4<T>{v[0], v[1], v[2], C[0]};
  planes[n + s] = V4<T>{C[1], C[2], C[3], C[4]};
  planes[2 * n + s] = V4<T>{C[5], C[6], C[7], C[8]};
}

// Tile node t = (a, b, c) in [0,7)^3, relative to node 4B-1 of the item's
// block B, lies in neighbour block ((a+3)>>2, (b+3)>>2, (c+3)>>2) of the
// 3x3x3 around B at local node ((a+3)&3, (b+3)&3, (c+3)&3).  Computed in
// registers (a table in memory would add a load per node to the busiest
// unit).  Node index of tile node t, or -1 when its block is not active.
__device__ __forceinline__ int tile_node(const int* snb, int t) {
  const int c = t / (kTile * kTile), r = t - c * (kTile * kTile);
  const int b = r / kTile, a = r - b * kTile;
  const int nb = snb[((c + 3) >> 2) * 9 + ((b + 3) >> 2) * 3 + ((a + 3) >> 2)];
  const int local = (((c + 3) & 3) << 4) | (((b + 3) & 3) << 2) | ((a + 3) & 3);
  return nb < 0 ? -1 : nb * kNodesPerBlock + local;
}

// G2P from the shared tile: v_hat = sum N v_i, Ch_hat = 2 sum N v_i (x) d,
// sum-factorised over x, then y, then z.
template <class T, bool AFF>
__device__ __forceinline__ void g2p_tile(const V4<T>* sv, int base, const T wx[4], const T dx[4],
                                         const T wy[4], const T dy[4], const T wz[4],
                                         const T dz[4], T hv[3], T hC[9]) {
  T s0[3] = {0, 0, 0}, sx[3] = {0, 0, 0}, sy[3] = {0, 0, 0}, sz[3] = {0, 0, 0};
  T wdx[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) wdx[k] = wx[k] * dx[k];
#pragma unroll
  for (int kz = 0; kz < 4; ++kz) {
#pragma unroll
    for (int ky = 0; ky < 4; ++ky) {
      T ax[3] = {0, 0, 0}, adx[3] = {0, 0, 0};
#pragma unroll
      for (int kx = 0; kx < 4; ++kx) {
        const V4<T> g = sv[base + kz * (kTile * kTile) + ky * kTile + kx];
        ax[0] += wx[kx] * g.x;
        ax[1] += wx[kx] * g.y;
        ax[2] += wx[kx] * g.z;
        if (AFF) {
          adx[0] += wdx[kx] * g.x;
          adx[1] += wdx[kx] * g.y;
          adx[2] += wdx[kx] * g.z;
        }
      }
      const T wyz = wy[ky] * wz[kz];
#pragma unroll
      for (int a = 0; a < 3; ++a) s0[a] += wyz * ax[a];
      if (AFF) {
        const T wyzdy = wyz * dy[ky], wyzdz = wyz * dz[kz];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          sx[a] += wyz * adx[a];
          sy[a] += wyzdy * ax[a];
          sz[a] += wyzdz * ax[a];
        }
      }
    }
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    hv[a] = s0[a];
    hC[3 * a + 0] = T(2) * sx[a];
    hC[3 * a + 1] = T(2) * sy[a];
    hC[3 * a + 2] = T(2) * sz[a];
  }
}

// The FP32 form of g2p_tile with paired FMAs: per node, (ax_x, ax_y) and
// (adx_x, adx_y) take (v_x, v_y) times (N, N) and (N d, N d), and
// (ax_z, adx_z) takes (v_z, v_z) times (N, N d) -- three paired FMAs where
// g2p_tile issues six.  Needs node velocities stored as (v_x, v_y, v_z, v_z).
__device__ __forceinline__ void g2p_tile_f32(const V4<float>* sv, int base, const float wx[4], const float dx[4],
                                             const float wy[4], const float dy[4], const float wz[4],
                                             const float dz[4], float hv[3], float hC[9]) {
  float2 wxx[4], wdd[4], wxd[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float wd = wx[k] * dx[k];
    wxx[k] = make_float2(wx[k], wx[k]);
    wdd[k] = make_float2(wd, wd);
    wxd[k] = make_float2(wx[k], wd);
  }
  float2 s0 = make_float2(0.f, 0.f), sx = s0, sy = s0, sz = s0;
  float s0z = 0.f, sxz = 0.f, syz = 0.f, szz = 0.f;
#pragma unroll
  for (int kz = 0; kz < 4; ++kz) {
#pragma unroll
    for (int ky = 0; ky < 4; ++ky) {
      float2 a01 = make_float2(0.f, 0.f), d01 = a01, az = a01;
#pragma unroll
      for (int kx = 0; kx < 4; ++kx) {
        const V4<float> g = sv[base + kz * (kTile * kTile) + ky * kTile + kx];
        const float2 gxy = make_float2(g.x, g.y), gzz = make_float2(g.z, g.w);
        a01 = __ffma2_rn(gxy, wxx[kx], a01);
        d01 = __ffma2_rn(gxy, wdd[kx], d01);
        az = __ffma2_rn(gzz, wxd[kx], az);
      }
      const float wyz = wy[ky] * wz[kz];
      const float wyzdy = wyz * dy[ky], wyzdz = wyz * dz[kz];
      s0 = __ffma2_rn(a01, make_float2(wyz, wyz), s0);
      sx = __ffma2_rn(d01, make_float2(wyz, wyz), sx);
      sy = __ffma2_rn(a01, make_float2(wyzdy, wyzdy), sy);
      sz = __ffma2_rn(a01, make_float2(wyzdz, wyzdz), sz);
      s0z += wyz * az.x;
      sxz += wyz * az.y;
      syz += wyzdy * az.x;
      szz += wyzdz * az.x;
    }
  }
  hv[0] = s0.x;
  hv[1] = s0.y;
  hv[2] = s0z;
  hC[0] = 2.f * sx.x;
  hC[1] = 2.f * sy.x;
  hC[2] = 2.f * sz.x;
  hC[3] = 2.f * sx.y;
  hC[4] = 2.f * sy.y;
  hC[5] = 2.f * sz.y;
  hC[6] = 2.f * sxz;
  hC[7] = 2.f * syz;
  hC[8] = 2.f * szz;
}

// Quadratic B-spline weight of one node row k (0..3, i.e. node i-1+k) as a
// polynomial in t, N_k(t) = c0 + c1 t + c2 t^2 (the App. B functions expanded).
template <class T>
__device__ __forceinline__ void row_poly(int k, T& c0, T& c1, T& c2) {
  c0 = k == 0 ? T(0.25) : k == 1 ? T(0.5) : k == 2 ? T(0.25) : T(0);
  c1 = k == 0 ? T(-0.5) : k == 2 ? T(0.5) : T(0);
  c2 = k == 0 ? T(0.25) : k == 3 ? T(0.25) : T(-0.25);
}

__device__ __forceinline__ void flush_mom(float*, V4<float>* gp, V4<double>* gp64,
                                          const uint32_t* gmask, int node, float x, float y,
                                          float z) {
  if (gp64 != nullptr && __popc(gmask[node]) >= 2) {
    atomicAdd(&gp64[node].x, (double)x);
    atomicAdd(&gp64[node].y, (double)y);
    atomicAdd(&gp64[node].z, (double)z);
  } else {
    atomicAdd(reinterpret_cast<float4*>(&gp[node]), make_float4(x, y, z, 0.f));
  }
}
__device__ __forceinline__ void flush_mom(double*, V4<double>* gp, V4<double>*, const uint32_t*,
                                          int node, double x, double y, double z) {
  atomicAdd(&gp[node].x, x);
  atomicAdd(&gp[node].y, y);
  atomicAdd(&gp[node].z, z);
}

// Stash rows of particle j are padded by one slot every 16 particles, so the
// two half-warps of a warp (16 particles apart) read different banks.
__device__ __forceinline__ int sidx(int j) { return j + (j >> 4); }

// Phase-2 register accumulators of one lane: nodes kx = 0..3 of its stencil
// row, K components.  A particle adds wx_k A_c + (wx_k dx_k) B_c to node k,
// component c.  The FP32 form packs node pairs (0,1) and (2,3) into float2
// and uses the paired FP32 FMA of sm_100+.
template <class T, int K>
struct RowAcc {
  T a[4][K];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int c = 0; c < K; ++c) a[k][c] = T(0);
  }
  __device__ __forceinline__ void add(const V4<T>& X, const V4<T>& XD, const T* A, const T* B) {
    const T wx[4] = {X.x, X.y, X.z, X.w}, wd[4] = {XD.x, XD.y, XD.z, XD.w};
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int c = 0; c < K; ++c) a[k][c] += wx[k] * A[c] + (B ? wd[k] * B[c] : T(0));
  }
  __device__ __forceinline__ T get(int k, int c) const { return a[k][c]; }
};

template <int K>
struct RowAcc<float, K> {
  float2 a01[K], a23[K];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int c = 0; c < K; ++c) a01[c] = a23[c] = make_float2(0.f, 0.f);
  }
  __device__ __forceinline__ void add(const V4<float>& X, const V4<float>& XD, const float* A, const float* B) {
    const float2 x01 = make_float2(X.x, X.y), x23 = make_float2(X.z, X.w);
    const float2 d01 = make_float2(XD.x, XD.y), d23 = make_float2(XD.z, XD.w);
#pragma unroll
    for (int c = 0; c < K; ++c) {
      const float2 Ac = make_float2(A[c], A[c]);
      a01[c] = __ffma2_rn(x01, Ac, a01[c]);
      a23[c] = __ffma2_rn(x23, Ac, a23[c]);
      if (B) {
        const float2 Bc = make_float2(B[c], B[c]);
        a01[c] = __ffma2_rn(d01, Bc, a01[c]);
        a23[c] = __ffma2_rn(d23, Bc, a23[c]);
      }
    }
  }
  __device__ __forceinline__ float get(int k, int c) const {
    return k == 0 ? a01[c].x : k == 1 ? a01[c].y : k == 2 ? a23[c].x : a23[c].y;
  }
};

// ---- Fixed-point node sums (FP32 path) ----
// A pass scatters, per particle and node, N m (w_c + sum_k Ch_ck d_k) with
// N <= 1 and |d_k| <= 2 (cell units), so every component is bounded by
//   b_p = m_p max_c (|w_c| + 2 sum_k |Ch_ck|).
// The default path uses the bound per work item: the item's shared P2G tile
// holds 32-bit integers at a scale from the sum of its particles' b_p (see
// k_items).  The deterministic mode uses it per scene, with int64 sums:
// If every b_p of a scene is at most B, a node sum over the scene's n
// particles stays below n B; the scale S = 2^e with S n B <= 2^62 then keeps
// it inside int64, and integer atomics add the scaled terms exactly, in any
// order.  B comes from the bound measured in the pass before (or, for the
// mass pass, from the inputs themselves), times a headroom of 2^lg; a term
// over B is recorded, the step is repeated with a larger headroom, and
// outputs are written only by a pass in which nothing was recorded.
__device__ __forceinline__ float fx_bound(float m, const float* w, const float* Ch) {
  float b = 0.f;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float t = fabsf(w[c]) + 2.f * (fabsf(Ch[3 * c]) + fabsf(Ch[3 * c + 1]) + fabsf(Ch[3 * c + 2]));
    b = (t > b || t != t) ? t : b;  // a NaN term propagates (fmaxf would drop it)
  }
  return m * b * 1.0001f;  // margin over the rounding of the terms themselves
}
// Scale of slot `slot` of one scene's bounds (fxs), headroom 2^lg, n terms
// per node at most: S = 2^e, the largest power of two with S n B <= 2^62
// (e at most 100, B at most 2^90); *allowed = the largest b_p it admits.
// FP32 and integer arithmetic only (every CTA and the normalisation compute
// the same S).
__device__ __forceinline__ float fx_scale(const unsigned* fxs, int slot, int lg, int n, float* allowed) {
  float B = __uint_as_float(fxs[slot]);
  if (slot >= 2) B = fmaxf(B, __uint_as_float(fxs[1]) * 0x1p-30f);  // W negligible next to V
  B = fminf(ldexpf(fmaxf(B, 1e-30f), lg), 0x1p90f);  // n B stays finite in FP32
  *allowed = B;
  int k;
  const float f = frexpf((float)max(n, 1) * B, &k);  // n B = f 2^k, f in [0.5, 1)
  (void)f;
  // n B <= 2^k, so S = 2^(62 - k) gives S n B <= 2^62 (up to the rounding of
  // n B, well inside int64's 2^63)
  return ldexpf(1.f, min(62 - k, 100));
}
// Headroom of a pass scattering W: the retry widens it for the scenes whose
// first attempt recorded an excess.
__device__ __forceinline__ int fx_head(const int* fx_err, int attempt, int scene) {
  return attempt > 0 && __ldcg(fx_err + scene) != 0 ? kFxRetryHeadLog2 : kFxHeadLog2;
}
// x S rounded to the nearest integer (ties to even).  x S is exact in FP32 (S
// is a power of two) and holds 24 significant bits, so above 2^24 it already
// is an integer m 2^e that shifts into place.
__device__ __forceinline__ unsigned long long to_fx(float x, float S) {
  const float r = rintf(x * S);
  if (fabsf(r) < 16777216.f) return (unsigned long long)(long long)__float2int_rn(r);
  const unsigned b = __float_as_uint(r);
  const int e = (int)((b >> 23) & 0xffu) - 150;  // r = m 2^e, 1 <= e
  const unsigned long long v = (unsigned long long)((b & 0x7fffffu) | 0x800000u) << min(e, 63);
  return (b >> 31) ? (unsigned long long)(-(long long)v) : v;
}
// A fixed-point sum back to FP32 (hi and lo words, deterministic rounding).
__device__ __forceinline__ float from_fx(long long g, float inv_S) {
  const float hi = (float)(int)(g >> 32), lo = (float)(unsigned)(g & 0xffffffffull);
  return fmaf(hi, 4294967296.f, lo) * inv_S;
}

// One work item = up to CHUNK * RPL sorted particles of one body whose
// cells lie in one grid block.  A CTA of CHUNK threads runs it in two
// phases:
//
//  phase 1, one thread per particle, RPL particles per thread (lanes sorted
//    by cell, so neighbouring lanes read the same tile nodes): G2P from the
//    7^3-node shared tile of grid velocities, the Sec. 2.3 series update of
//    Delta, the Sec. 2.4 projection giving W, and a stash of (t, m, W) in
//    shared memory;
//  phase 2, cell-centric P2G: a group of 16 / RPL lanes walks 16
//    consecutive stashed particles; each lane owns RPL stencil rows
//    (., ky, kz) of the current cell and keeps their 4 nodes x 3 components
//    in registers, adding them to the shared P2G tile only when the cell
//    changes.  No two lanes of a group ever add to the same node.  With
//    RPL = 2 a group is 8 lanes, so a stashed record is read by 8 lanes
//    instead of 16, and a warp walks 64 particles.
//
// The shared P2G tile is then added to the global grid (FP64 at nodes that
// two or more bodies touch, on the FP32 path).
//
// CHUNK is the CTA size, CHUNK * RPL the largest item, MINB the number of
// resident CTAs per SM the kernel is compiled for (its register cap); the
// autotuner picks among the variants of apic_internal.h.
//
// DET (deterministic mode, FP32): the shared tile and the global node sums
// hold scaled int64 terms (fixed point) instead of floating-point sums.
//
// items_body runs one work item with the whole CTA; k_items runs one item
// per CTA or, persistent (PERSIST), a grid of resident CTAs: CTA b starts
// with item b and then draws tickets for the items after the first
// gridDim.x, one at a time, until the items run out.
template <class T, int MODE, int MINB, int CHUNK, bool ROWTAB, bool DET, int RPL>
__device__ __forceinline__ void items_body(const IterParams<T>& p, const int item) {
  static_assert(RPL == 1 || RPL == 2, "one or two stencil rows per lane");
  constexpr int kItem = CHUNK * RPL;  // particles of the largest item
  constexpr int kStashN = kItem + kItem / 16;
  constexpr int kGroup = 16 / RPL;    // lanes that walk one run of 16 particles in phase 2
  constexpr bool kG2P = MODE == kModeFirst || MODE == kModeMid || MODE == kModeLast || MODE == kModeOnly;
  constexpr bool kP2G = MODE == kModeMassV || MODE == kModeFirst || MODE == kModeMid;
  constexpr bool kMass = MODE == kModeMassV;  // also accumulates m_i and the body mask
  constexpr int kComp = kMass ? 4 : 3;         // momentum (x, y, z) [, mass]
  __shared__ V4<T> sv[kG2P ? kTile3 : 1];
  __shared__ uint32_t smask[MODE == kModeMu ? kTile3 : 1];
  __shared__ T smass[MODE == kModeNormals ? kTile3 : 1];  // the item's body's node masses
  // FP32 series passes: the tile's node body masks (final since the mass
  // pass), fetched with the velocities, for the flush's FP64 choice
  constexpr bool kMaskPre = sizeof(T) == 4 && !DET && (MODE == kModeFirst || MODE == kModeMid);
  __shared__ uint32_t smk[kMaskPre ? kTile3 : 1];
  // FP32 default path: the tile's momentum sums are 32-bit fixed point with a
  // per-item power-of-two scale (native integer atomics; a float add to
  // shared memory is a compare-and-swap loop).  The mass sums of the mass
  // pass stay float, stored in the same int array: a node's mass is used in
  // ratios (the per-pair friction blend, mass normals) and sets its body
  // bit, so a mass term below a fixed-point unit must not vanish.
  constexpr bool kFix = sizeof(T) == 4 && !DET && kP2G;
  using Acc = typename std::conditional<DET, long long, typename std::conditional<kFix, int, T>::type>::type;
  __shared__ Acc sacc[kP2G ? kComp : 1][kTile3];
  __shared__ unsigned s_fxmax;
  __shared__ float s_bw[kFix ? CHUNK / 32 : 1];  // per-warp sums of the term bounds
  __shared__ V4<T> stash[kP2G ? (ROWTAB ? 7 : 6) : 1][kP2G ? kStashN : 1];
  __shared__ int sloc[kItem];
  __shared__ int snb[27];
  // Passes that write the outputs keep each warp's results in shared memory
  // and store them in caller order sorted by caller index (rows of 13
  // values: no bank conflicts between lanes).
  constexpr bool kWarpOut = RPL == 1 && (MODE == kModeLast || MODE == kModeOnly);
  __shared__ T sout[kWarpOut ? CHUNK / 32 : 1][kWarpOut ? 32 * 13 : 1];
  __shared__ long long skey[kWarpOut ? CHUNK / 32 : 1][kWarpOut ? 32 : 1];
  const int tid = threadIdx.x;
  // node index of tile node t (-1: inactive block; the debug build also
  // refuses an index outside the node arrays)
  auto node_of = [&](int t) {
    const int nd = tile_node(snb, t);
    return nd >= 0 && !APIC_DBG_CHECK(nd < p.n_nodes, kDbgTileNode) ? -1 : nd;
  };
  const int n = p.n_particles;
  // R9 friction blend of one particle at tile cell `base` from the tile's
  // node masks: mu_p = sum_{b' != b} mu(b,b') M_b'p / sum_{b' != b} M_b'p with
  // M_b'p = sum_i N_ip m_{b',i}; mu(b,b) when no other body is near.
  auto friction_blend = [&](const uint32_t* masks, const V4<T>& pt, int base, int body, const SceneDev& S,
                            float fxSm) -> T {
    T wx[4], dx[4], wy[4], dy[4], wz[4], dz[4];
    bspline(pt.x, wx, dx);
    bspline(pt.y, wy, dy);
    bspline(pt.z, wz, dz);
    T num = T(0), den = T(0);
    const uint32_t own = 1u << body;
#pragma unroll 1
    for (int q = 0; q < 64; ++q) {
      const int kx = q & 3, ky = (q >> 2) & 3, kz = q >> 4;
      const int tq = base + kz * (kTile * kTile) + ky * kTile + kx;
      uint32_t other = masks[tq] & ~own;
      if (!other) continue;
      const int node = node_of(tq);
      T wxk = kx == 0 ? wx[0] : kx == 1 ? wx[1] : kx == 2 ? wx[2] : wx[3];
      T wyk = ky == 0 ? wy[0] : ky == 1 ? wy[1] : ky == 2 ? wy[2] : wy[3];
      T wzk = kz == 0 ? wz[0] : kz == 1 ? wz[1] : kz == 2 ? wz[2] : wz[3];
      const T w = wxk * wyk * wzk;
      while (other) {
        const int bo = __ffs(other) - 1;
        other &= other - 1;
        const T M = DET ? (T)from_fx(p.gmb_fx[(int64_t)bo * p.n_nodes + node], 1.f / fxSm)
                        : p.gmb[(int64_t)bo * p.n_nodes + node];
        num += w * p.mu_table[S.mu_off + body * S.n_bodies + bo] * M;
        den += w * M;
      }
    }
    return den > T(0) ? num / den : p.mu_table[S.mu_off + body * S.n_bodies + body];
  };
  if (item >= p.n_items) {
    grid_dep_wait();
    return;
  }
  const int4 info = p.item_info[item];
  const SceneDev& S = p.sc[info.z];
  const Box box = S.box;
  const int body = info.y;
  const int s0 = p.item_start[item];
  const int s1 = item + 1 < p.n_items ? p.item_start[item + 1] : n;
  const int count = s1 - s0;  // <= kItem
  if (!APIC_DBG_CHECK(count >= 1 && count <= kItem, kDbgSlot)) {
    grid_dep_wait();
    return;
  }
  // phase-1 slot of this thread's r-th particle: warp w holds the slots
  // [32 RPL w, 32 RPL (w + 1)), the ones its phase-2 groups walk
  const int wslot = (tid >> 5) * (32 * RPL) + (tid & 31);
  // Particles are sorted by cell (z-major) inside an item, so its stencils
  // reach only tile layers c in [lz(first), lz(last) + 3]: fetch, clear and
  // flush just those.
  const int t_lo = (int)(to_bits(p.pn[s0].w) >> 4) * (kTile * kTile);
  const int t_hi = ((int)(to_bits(p.pn[s1 - 1].w) >> 4) + 4) * (kTile * kTile);
  // Issue this thread's particle loads first so that they are in flight
  // while the CTA fetches its grid tile.
  constexpr bool kReadD = MODE == kModeMid || MODE == kModeLast;
  constexpr bool kReadV = MODE == kModeMassV || MODE == kModeFirst || MODE == kModeOnly;
  V4<T> ptr_[RPL], pnr_[RPL], q0r[RPL], q1r[RPL], q2r[RPL];
#pragma unroll
  for (int r = 0; r < RPL; ++r) {
    ptr_[r] = pnr_[r] = q0r[r] = q1r[r] = q2r[r] = V4<T>{};
    const int j = wslot + 32 * r;
    if (j < count) {
      const int s = s0 + j;
      ptr_[r] = p.pt[s];
      pnr_[r] = p.pn[s];
      if (kReadV) {
        q0r[r] = p.V[s];
        q1r[r] = p.V[n + s];
        q2r[r] = p.V[2 * n + s];
      }
    }
  }
  if (tid < 27) {
    // the 3x3x3 blocks around the item's block (info.x is its global page
    // index; every particle block keeps a one-block margin inside its box)
    const int ox = tid % 3 - 1, oy = (tid / 3) % 3 - 1, oz = tid / 9 - 1;
    const long long pg = (long long)info.x + ((long long)oz * box.ny + oy) * box.nx + ox;
    snb[tid] = APIC_DBG_CHECK(pg >= 0 && pg < p.n_pages, kDbgPage) ? p.page[pg] : -1;
  }
  if (kP2G)
    for (int t = t_lo + tid; t < t_hi; t += CHUNK)
#pragma unroll
      for (int a = 0; a < kComp; ++a) sacc[a][t] = Acc(0);
  if (DET && tid == 0) s_fxmax = 0u;
  // D, the node velocities, the node masks and the grid sums come from the
  // grids before this one
  grid_dep_wait();
  // Fixed-point scales of this CTA's scene: S for momentum terms, Sm for
  // masses; fx_ok is the largest term bound S admits.
  float fxS = 0.f, fxSm = 0.f, fx_ok = 0.f;
  bool fx_bad = false;
  if constexpr (DET) {
    const unsigned* fxs = p.fx_max + (int64_t)info.z * p.fx_stride;
    float unused;
    if (MODE == kModeMassV || MODE == kModeMu || MODE == kModeNormals) fxSm = fx_scale(fxs, 0, 0, S.n, &unused);
    if (MODE == kModeMassV) fxS = fx_scale(fxs, 1, 0, S.n, &fx_ok);
    if (MODE == kModeFirst || MODE == kModeMid)
      fxS = fx_scale(fxs, p.fx_slot, fx_head(p.fx_err, p.fx_attempt, info.z), S.n, &fx_ok);
  }
  if (kReadD) {
#pragma unroll
    for (int r = 0; r < RPL; ++r) {
      const int j = wslot + 32 * r;
      if (j < count) {
        const int s = s0 + j;
        q0r[r] = p.D[s];
        q1r[r] = p.D[n + s];
        q2r[r] = p.D[2 * n + s];
      }
    }
  }
  __syncthreads();
  if (kG2P) {
    if constexpr (sizeof(T) == 4) {
      // global -> shared without staging in registers (cp.async, 16 bytes:
      // V4<float> is 16-byte aligned in both spaces); all of this thread's
      // copies are in flight together
      for (int t = t_lo + tid; t < t_hi; t += CHUNK) {
        const int node = node_of(t);
        if (node >= 0) {
          const unsigned dst = (unsigned)__cvta_generic_to_shared(&sv[t]);
          asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(&p.gv[node]) : "memory");
          if constexpr (kMaskPre) {
            const unsigned dm = (unsigned)__cvta_generic_to_shared(&smk[t]);
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dm), "l"(&p.gmask[node]) : "memory");
          }
        } else {
          sv[t] = V4<T>{T(0), T(0), T(0), T(0)};
          if constexpr (kMaskPre) smk[t] = 0u;
        }
      }
      asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
    } else {
      for (int t = t_lo + tid; t < t_hi; t += CHUNK) {
        const int node = node_of(t);
        sv[t] = node >= 0 ? p.gv[node] : V4<T>{T(0), T(0), T(0), T(0)};
      }
    }
    __syncthreads();
  }
  // the first pass with the friction blend folded in: does any other body
  // reach this item's tile? (uniform over the CTA)
  bool fold_other = false;
  if constexpr (kMaskPre && MODE == kModeFirst) {
    if (p.fold_mu && S.mu_off >= 0) {
      const uint32_t own = 1u << body;
      int o = 0;
      for (int t = t_lo + tid; t < t_hi; t += CHUNK) o |= (smk[t] & ~own) != 0u;
      fold_other = __syncthreads_or(o) != 0;
    }
  }
  if (MODE == kModeNormals) {
    for (int t = t_lo + tid; t < t_hi; t += CHUNK) {
      const int node = node_of(t);
      T mi = T(0);
      if (node >= 0) {
        const int64_t k = (int64_t)body * p.n_nodes + node;
        mi = DET ? (T)from_fx(p.gmb_fx[k], 1.f / fxSm) : p.gmb[k];
      }
      smass[t] = mi;
    }
    __syncthreads();
  }
  if (MODE == kModeMu) {
    const uint32_t own = 1u << body;
    int other = 0;
    for (int t = t_lo + tid; t < t_hi; t += CHUNK) {
      const int node = node_of(t);
      const uint32_t m = node >= 0 ? p.gmask[node] : 0u;
      smask[t] = m;
      other |= (m & ~own) != 0u;
    }
    if (!__syncthreads_or(other)) {
      // no other body anywhere in the tile: every particle keeps mu(b, b),
      // as the blend below would give it (no other body's mass in reach)
#pragma unroll
      for (int r = 0; r < RPL; ++r)
        if (wslot + 32 * r < count)
          p.mup_out[s0 + wslot + 32 * r] =
              S.mu_off < 0 ? (T)S.mu : p.mu_table[S.mu_off + body * S.n_bodies + body];
      return;
    }
  }

  // ---------------- phase 1: one thread per particle ----------------
  float bsum = 0.f;  // kFix: sum of this thread's particle term bounds
  long long okey = LLONG_MAX;  // kWarpOut: (caller index << 5) | lane of this thread's output
#pragma unroll
  for (int r = 0; r < RPL; ++r) {
    const int j = wslot + 32 * r;
    const V4<T> pt = ptr_[r], pn = pnr_[r];
    V4<T> q0 = q0r[r], q1 = q1r[r], q2 = q2r[r];
    if (j < count) {
      const int s = s0 + j;
      const uint32_t loc = to_bits(pn.w);
      int base = (int)(loc >> 4) * (kTile * kTile) + (int)((loc >> 2) & 3) * kTile + (int)(loc & 3);
      if (!APIC_DBG_CHECK(loc < 64u, kDbgSlot)) base = 0;  // (a cell outside its block)
      sloc[j] = base;
      if (MODE == kModeMu && S.mu_off < 0) {
        p.mup_out[s] = (T)S.mu;  // a scene with one scalar mu
      } else if (MODE == kModeMu) {
        p.mup_out[s] = friction_blend(smask, pt, base, body, S, fxSm);
      } else if (MODE == kModeNormals) {
        // rho = sum N m_b and g = sum grad N m_b (cell units) over the body's
        // own node masses, sum-factorised; n = -g/|g| on the surface, else 0
        T wx[4], dx[4], wy[4], dy[4], wz[4], dz[4], gx[4], gy[4], gz[4];
        bspline(pt.x, wx, dx);
        bspline(pt.y, wy, dy);
        bspline(pt.z, wz, dz);
        bspline_grad(pt.x, gx);
        bspline_grad(pt.y, gy);
        bspline_grad(pt.z, gz);
        T rho = T(0), g0 = T(0), g1 = T(0), g2 = T(0);
#pragma unroll
        for (int kz = 0; kz < 4; ++kz) {
          T r = T(0), ry = T(0), rx = T(0);  // sum over y of N_y (N_x m), of gN_y (N_x m), of N_y (gN_x m)
#pragma unroll
          for (int ky = 0; ky < 4; ++ky) {
            T a = T(0), ad = T(0);
#pragma unroll
            for (int kx = 0; kx < 4; ++kx) {
              const T mi = smass[base + kz * (kTile * kTile) + ky * kTile + kx];
              a += wx[kx] * mi;
              ad += gx[kx] * mi;
            }
            r += wy[ky] * a;
            ry += gy[ky] * a;
            rx += wy[ky] * ad;
          }
          rho += wz[kz] * r;
          g0 += wz[kz] * rx;
          g1 += wz[kz] * ry;
          g2 += gz[kz] * r;
        }
        const T len = sqrt(g0 * g0 + g1 * g1 + g2 * g2);
        const bool surf = rho > T(0) && len > (T)S.nthr * rho;
        const T inv = surf ? -T(1) / len : T(0);
        const T nn[3] = {g0 * inv, g1 * inv, g2 * inv};
        if (p.normals_out) {
          const int64_t idx = p.perm[s] - S.part_off;
          T* o = static_cast<T*>(S.v_out);
          if (APIC_DBG_CHECK(idx >= 0 && idx < S.n, kDbgPerm))
#pragma unroll
            for (int a = 0; a < 3; ++a) o[3 * idx + a] = nn[a];
        } else {
          p.pn_out[s] = V4<T>{nn[0], nn[1], nn[2], pn.w};
        }
      } else if (MODE == kModeMassV) {
        T wx[4], dx[4];
        bspline(pt.x, wx, dx);
        if constexpr (kFix) {
          const float vv[3] = {q0.x, q0.y, q0.z};
          const float Cc[9] = {q0.w, q1.x, q1.y, q1.z, q1.w, q2.x, q2.y, q2.z, q2.w};
          bsum += fx_bound(pt.w, vv, Cc);
        }
        if constexpr (ROWTAB) {
          T wy[4], dy[4], wz[4], dz[4];
          bspline(pt.y, wy, dy);
          bspline(pt.z, wz, dz);
          stash[0][sidx(j)] = V4<T>{pt.w * wy[0], pt.w * wy[1], pt.w * wy[2], pt.w * wy[3]};
          stash[ROWTAB ? 6 : 0][sidx(j)] = V4<T>{wz[0], wz[1], wz[2], wz[3]};
          if (!p.pic) {
            // fold the particle's own offset into v: v_c - Ch_c1 t_y - Ch_c2 t_z
            q0.x -= q1.x * pt.y + q1.y * pt.z;
            q0.y -= q1.w * pt.y + q2.x * pt.z;
            q0.z -= q2.z * pt.y + q2.w * pt.z;
          }
        } else {
          stash[0][sidx(j)] = pt;
        }
        stash[4][sidx(j)] = V4<T>{wx[0], wx[1], wx[2], wx[3]};
        stash[5][sidx(j)] = V4<T>{wx[0] * dx[0], wx[1] * dx[1], wx[2] * dx[2], wx[3] * dx[3]};
        // W = V, in phase 2's record layout (below)
        stash[1][sidx(j)] = V4<T>{q0.x, q0.y, q1.x, q1.w};
        stash[2][sidx(j)] = V4<T>{q1.y, q2.x, q0.w, q1.z};
        stash[3][sidx(j)] = V4<T>{q0.z, q2.z, q2.w, q2.y};
      } else {
        T wx[4], dx[4], wy[4], dy[4], wz[4], dz[4];
        bspline(pt.x, wx, dx);
        bspline(pt.y, wy, dy);
        bspline(pt.z, wz, dz);
        T hv[3], hC[9];
        if (p.pic)
          g2p_tile<T, false>(sv, base, wx, dx, wy, dy, wz, dz, hv, hC);
        else if constexpr (sizeof(T) == 4)
          g2p_tile_f32(sv, base, wx, dx, wy, dy, wz, dz, hv, hC);
        else
          g2p_tile<T, true>(sv, base, wx, dx, wy, dy, wz, dz, hv, hC);
        const T nrm[3] = {pn.x, pn.y, pn.z};
        T mu;
        if (kMaskPre && MODE == kModeFirst && p.fold_mu) {
          if constexpr (kMaskPre) {
            mu = S.mu_off < 0 ? (T)S.mu
                 : fold_other ? friction_blend(smk, pt, base, body, S, fxSm)
                              : p.mu_table[S.mu_off + body * S.n_bodies + body];
          } else {
            mu = (T)S.mu;
          }
          p.mup_out[s] = mu;  // for the passes after this one
        } else {
          mu = p.mup ? p.mup[s] : (T)S.mu;
        }
        T dv[3], dC[9];
        bool out = false;
        if (MODE == kModeFirst || MODE == kModeOnly) {
          // Delta_0 = H V - V
          const T v[3] = {q0.x, q0.y, q0.z};
          const T C[9] = {q0.w, q1.x, q1.y, q1.z, q1.w, q2.x, q2.y, q2.z, q2.w};
#pragma unroll
          for (int a = 0; a < 3; ++a) dv[a] = hv[a] - v[a];
#pragma unroll
          for (int a = 0; a < 9; ++a) dC[a] = p.pic ? T(0) : hC[a] - C[a];
          out = MODE == kModeOnly;
        } else {
          // Delta_m = Delta_{m-1} + H W_m - W_m, W_m recomputed from Delta_{m-1}
          const T pv[3] = {q0.x, q0.y, q0.z};
          const T pC[9] = {q0.w, q1.x, q1.y, q1.z, q1.w, q2.x, q2.y, q2.z, q2.w};
          T wv[3], wC[9];
          undesirable(pv, pC, nrm, mu, p.sep23, wv, wC);
#pragma unroll
          for (int a = 0; a < 3; ++a) dv[a] = pv[a] + hv[a] - wv[a];
#pragma unroll
          for (int a = 0; a < 9; ++a) dC[a] = p.pic ? T(0) : pC[a] + hC[a] - wC[a];
          out = MODE == kModeLast;
        }
        if (DET && out && __ldcg(p.fx_err + p.fx_attempt * (p.n_scenes + 1) + p.n_scenes) != 0) {
          // an earlier pass of this attempt exceeded its fixed-point range in
          // some scene: the step is repeated (or fails), and no scene's outputs
          // are written by this attempt
        } else if (out) {
          // V_hat = V + Delta_N, back in caller order, C = Ch / h
          T v[3], C[9];
          load12(p.V, n, s, v, C);
          const int64_t idx = p.perm[s] - S.part_off;
          T* vo = static_cast<T*>(S.v_out);
          T* Co = static_cast<T*>(S.C_out);
          const T inv_h = (T)S.inv_h;
          if constexpr (kWarpOut) {
            // stored by the whole warp below
            T* so = &sout[tid >> 5][(tid & 31) * 13];
#pragma unroll
            for (int a = 0; a < 3; ++a) so[a] = v[a] + dv[a];
#pragma unroll
            for (int a = 0; a < 9; ++a) so[3 + a] = (C[a] + dC[a]) * inv_h;
            if (APIC_DBG_CHECK(idx >= 0 && idx < S.n, kDbgPerm)) okey = (idx << 5) | (tid & 31);
          } else if (APIC_DBG_CHECK(idx >= 0 && idx < S.n, kDbgPerm)) {
#pragma unroll
            for (int a = 0; a < 3; ++a) vo[3 * idx + a] = v[a] + dv[a];
#pragma unroll
            for (int a = 0; a < 9; ++a) Co[9 * idx + a] = (C[a] + dC[a]) * inv_h;
          }
        } else {
          store12(p.D, n, s, dv, dC);
          T u[3], uC[9];
          undesirable(dv, dC, nrm, mu, p.sep23, u, uC);
          if constexpr (kFix) bsum += fx_bound(pt.w, u, uC);
          if constexpr (DET) {
            const float b = fx_bound(pt.w, u, uC);
            fx_bad = fx_bad || !(b <= fx_ok);
            atomicMax(&s_fxmax, __float_as_uint(b));
          }
          if constexpr (ROWTAB) {
            stash[0][sidx(j)] = V4<T>{pt.w * wy[0], pt.w * wy[1], pt.w * wy[2], pt.w * wy[3]};
            stash[ROWTAB ? 6 : 0][sidx(j)] = V4<T>{wz[0], wz[1], wz[2], wz[3]};
            if (!p.pic) {  // fold the particle's own offset into u: u_c - Ch_c1 t_y - Ch_c2 t_z
              u[0] -= uC[1] * pt.y + uC[2] * pt.z;
              u[1] -= uC[4] * pt.y + uC[5] * pt.z;
              u[2] -= uC[7] * pt.y + uC[8] * pt.z;
            }
          } else {
            stash[0][sidx(j)] = pt;
          }
          // W = (u, uC) in phase 2's record layout (below)
          stash[1][sidx(j)] = V4<T>{u[0], u[1], uC[1], uC[4]};
          stash[2][sidx(j)] = V4<T>{uC[2], uC[5], uC[0], uC[3]};
          stash[3][sidx(j)] = V4<T>{u[2], uC[7], uC[8], uC[6]};
          stash[4][sidx(j)] = V4<T>{wx[0], wx[1], wx[2], wx[3]};
          stash[5][sidx(j)] = V4<T>{wx[0] * dx[0], wx[1] * dx[1], wx[2] * dx[2], wx[3] * dx[3]};
        }
      }
    }
  }
  if constexpr (kWarpOut) {
    // The warp's outputs in caller order.  Sorted by caller index (a bitonic
    // sort of the 32 keys across the warp), runs of consecutive particles
    // (the caller's numbering is usually spatially coherent) become runs of
    // consecutive addresses, and lane k of each store instruction writes the
    // k-th value of the warp's sorted outputs: whole sectors instead of every
    // third or ninth float of many.  Measured on the 4 M-node scene: the last
    // pass about 105 us faster, 4.34 -> 4.18 ms a step.
    const int lane = tid & 31;
    long long key = okey;
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1)
#pragma unroll
      for (int jj = k >> 1; jj > 0; jj >>= 1) {
        const long long other = __shfl_xor_sync(0xffffffffu, key, jj);
        const bool keep_min = ((lane & jj) == 0) == ((lane & k) == 0);
        key = keep_min ? min(key, other) : max(key, other);
      }
    const int cnt = __popc(__ballot_sync(0xffffffffu, okey != LLONG_MAX));
    skey[tid >> 5][lane] = key;
    __syncwarp();
    T* vo = static_cast<T*>(S.v_out);
    T* Co = static_cast<T*>(S.C_out);
    const T* so = sout[tid >> 5];
    const long long* sk = skey[tid >> 5];
    for (int f = lane; f < 3 * cnt; f += 32) {
      const int r = f / 3, a = f - 3 * r;
      const long long kk = sk[r];
      vo[3 * (kk >> 5) + a] = so[(int)(kk & 31) * 13 + a];
    }
    for (int f = lane; f < 9 * cnt; f += 32) {
      const int r = f / 9, a = f - 9 * r;
      const long long kk = sk[r];
      Co[9 * (kk >> 5) + a] = so[(int)(kk & 31) * 13 + 3 + a];
    }
  }
  if (!kP2G) return;
  // Group g of phase 2 walks particles 16g .. 16g+15, which lanes of its own
  // warp stashed in phase 1: ordering within the warp is enough, except for
  // the fixed-point scale, which needs every warp's bound.
  float fxT = 0.f, fxInvT = 0.f;  // kFix: tile scale T = 2^e and 1/T
  bool fx_nonfinite = false;
  if constexpr (kFix) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bsum += __shfl_xor_sync(0xffffffffu, bsum, o);
    if ((tid & 31) == 0) s_bw[tid >> 5] = bsum;
    __syncthreads();
    float B = 0.f;
#pragma unroll
    for (int w = 0; w < CHUNK / 32; ++w) B += s_bw[w];
    // every node sum of the tile, and every partial sum a lane adds, is at
    // most B / 8: a particle adds at most N b_p to a node, and N <= 1/8
    // (each one-dimensional App. B weight is at most 1/2).  With B < 2^k,
    // T = 2^(33 - k) keeps them below 2^30 in magnitude.
    fx_nonfinite = !(B <= 3.0e38f);
    // B = f 2^k with f in [0.5, 1): k is B's biased exponent - 126 (a zero or
    // subnormal B gives k = -126, and the cap e = 126 applies); T and 1/T are
    // built from their exponent bits
    const int k = (int)((__float_as_uint(B) >> 23) & 0xffu) - 126;
    const int e = fx_nonfinite ? 0 : min(33 - k, 126);
    fxT = __uint_as_float((unsigned)(e + 127) << 23);
    fxInvT = __uint_as_float((unsigned)(127 - e) << 23);
  } else {
    __syncwarp();
  }

  // ---------------- phase 2: cell-centric P2G ----------------
  {
    const int grp = tid / kGroup, lg = tid % kGroup;
    const int ky = lg & 3, kz0 = lg >> 2;  // rows (ky, kz0 + k 4 / RPL), k < RPL
    T cy0, cy1, cy2, cz0[RPL], cz1[RPL], cz2[RPL], oz[RPL];
    int kzr[RPL];
    row_poly(ky, cy0, cy1, cy2);
#pragma unroll
    for (int k = 0; k < RPL; ++k) {
      kzr[k] = kz0 + k * (4 / RPL);
      row_poly(kzr[k], cz0[k], cz1[k], cz2[k]);
      oz[k] = T(kzr[k] - 1);
    }
    const T oy = T(ky - 1);
    const bool aff = !p.pic;
    RowAcc<T, 3> acc[RPL];
    RowAcc<T, 1> macc[RPL];  // mass, when this pass also scatters mass (kModeMassV)
#pragma unroll
    for (int k = 0; k < RPL; ++k) {
      acc[k].zero();
      macc[k].zero();
    }
    const int j0 = grp * 16, j1 = min(j0 + 16, count);
    auto flush = [&](int base) {
#pragma unroll
      for (int kk = 0; kk < RPL; ++kk) {
        const int row = base + kzr[kk] * (kTile * kTile) + ky * kTile;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          if constexpr (DET) {
#pragma unroll
            for (int c = 0; c < 3; ++c)
              atomicAdd(reinterpret_cast<unsigned long long*>(&sacc[c][row + k]), to_fx(acc[kk].get(k, c), fxS));
            if constexpr (MODE == kModeMassV)
              atomicAdd(reinterpret_cast<unsigned long long*>(&sacc[3][row + k]), to_fx(macc[kk].get(k, 0), fxSm));
          } else if constexpr (kFix) {
#pragma unroll
            for (int c = 0; c < 3; ++c) atomicAdd(&sacc[c][row + k], __float2int_rn(acc[kk].get(k, c) * fxT));
            if constexpr (MODE == kModeMassV)
              atomicAdd(reinterpret_cast<float*>(&sacc[3][row + k]), macc[kk].get(k, 0));
          } else {
#pragma unroll
            for (int c = 0; c < 3; ++c) atomicAdd(&sacc[c][row + k], acc[kk].get(k, c));
            if constexpr (MODE == kModeMassV) atomicAdd(&sacc[3][row + k], macc[kk].get(k, 0));
          }
        }
        acc[kk].zero();
        macc[kk].zero();
      }
    };
    // stash row index sidx(j) = j + (j >> 4); j >> 4 is fixed over a group's 16
    const int jofs = j0 >> 4;
    // phase 2 for stashed particle j: this lane's rows of its 4^3 stencil
    auto accumulate = [&](const int j) {
      const int sj = j + jofs;
      const V4<T> X = stash[4][sj], XD = stash[5][sj];
      T wyzm[RPL], ty = T(0), tz = T(0);
      if constexpr (ROWTAB) {
        // this lane's row weights m N_y(ky) N_z(kz), from the stashed factors
        // (the particle's own offset is already folded into u)
        const T wym = reinterpret_cast<const T*>(&stash[0][sj])[ky];
#pragma unroll
        for (int k = 0; k < RPL; ++k)
          wyzm[k] = wym * reinterpret_cast<const T*>(&stash[ROWTAB ? 6 : 0][sj])[kzr[k]];
      } else {
        const V4<T> a = stash[0][sj];
        const T wym = a.w * (cy0 + a.y * (cy1 + a.y * cy2));
#pragma unroll
        for (int k = 0; k < RPL; ++k) wyzm[k] = wym * (cz0[k] + a.z * (cz1[k] + a.z * cz2[k]));
        ty = a.y;
        tz = a.z;
      }
      if constexpr (kMass) {
#pragma unroll
        for (int k = 0; k < RPL; ++k) {
          const T A[1] = {wyzm[k]};
          macc[k].add(X, XD, A, nullptr);
        }
      }
      {
        // W = (u, Ch) as the records w0 = (u_0, u_1, Ch_01, Ch_11),
        // w1 = (Ch_02, Ch_12, Ch_00, Ch_10), w2 = (u_2, Ch_21, Ch_22, Ch_20), so
        // that components 0 and 1 pair up for the paired FP32 operations.
        // Node k of a row gets wx_k A + wx_k dx_k B with
        //   A_c = m wy wz (u_c + Ch_c1 dy + Ch_c2 dz),  B_c = m wy wz Ch_c0.
        const V4<T> w0 = stash[1][sj], w1 = stash[2][sj], w2 = stash[3][sj];
        const T dy = oy - ty;
#pragma unroll
        for (int k = 0; k < RPL; ++k) {
          const T dz = oz[k] - tz;
          T A[3], B[3];
          if (aff) {
            if constexpr (sizeof(T) == 4) {
              const float2 m2 = make_float2(wyzm[k], wyzm[k]);
              float2 a01 = __ffma2_rn(make_float2(w0.z, w0.w), make_float2(dy, dy), make_float2(w0.x, w0.y));
              a01 = __fmul2_rn(__ffma2_rn(make_float2(w1.x, w1.y), make_float2(dz, dz), a01), m2);
              const float2 b01 = __fmul2_rn(make_float2(w1.z, w1.w), m2);
              A[0] = a01.x;
              A[1] = a01.y;
              B[0] = b01.x;
              B[1] = b01.y;
            } else {
              A[0] = wyzm[k] * (w0.x + w0.z * dy + w1.x * dz);
              A[1] = wyzm[k] * (w0.y + w0.w * dy + w1.y * dz);
              B[0] = wyzm[k] * w1.z;
              B[1] = wyzm[k] * w1.w;
            }
            A[2] = wyzm[k] * (w2.x + w2.y * dy + w2.z * dz);
            B[2] = wyzm[k] * w2.w;
            acc[k].add(X, XD, A, B);
          } else {
            A[0] = wyzm[k] * w0.x;
            A[1] = wyzm[k] * w0.y;
            A[2] = wyzm[k] * w2.x;
            acc[k].add(X, XD, A, nullptr);
          }
        }
      }
    };
    if constexpr (RPL == 1) {
      // Runs of equal cells from a warp ballot of the run heads (phase-1 slot
      // j is thread j's, in this warp): a group walks each run without
      // checking for a change of cell and flushes once at its end.
      const bool head = tid < count && ((tid & 15) == 0 || sloc[tid] != sloc[tid - 1]);
      const unsigned heads = __ballot_sync(0xffffffffu, head);
      const unsigned hm = (heads >> (j0 & 31)) & 0xffffu;  // this group's 16 slots
      int a = j0;
      while (a < j1) {
        const unsigned later = hm & ~((2u << (a - j0)) - 1u);  // heads after slot a
        const int b = later ? min(j0 + __ffs(later) - 1, j1) : j1;
        const int base = sloc[a];
        for (int j = a; j < b; ++j) accumulate(j);
        flush(base);
        a = b;
      }
    } else {
      int cur = -1;
      for (int j = j0; j < j1; ++j) {
        const int base = sloc[j];
        if (base != cur) {
          if (cur >= 0) flush(cur);
          cur = base;
        }
        accumulate(j);
      }
      if (cur >= 0) flush(cur);
    }
  }
  __syncthreads();

  // ---------------- add the tile to the global grid ----------------
  // (only the P2G modes get here)
  if constexpr (DET && kP2G) {
    if (fx_bad) {
      int* row = p.fx_err + p.fx_attempt * (p.n_scenes + 1);
      atomicOr(row + info.z, 1);
      atomicOr(row + p.n_scenes, 1);  // any scene of this attempt
    }
    if (MODE != kModeMassV && tid == 0) atomicMax(p.fx_max + (int64_t)info.z * p.fx_stride + p.fx_slot + 1, s_fxmax);
    for (int t = t_lo + tid; t < t_hi; t += CHUNK) {
      const int node = node_of(t);
      if (node < 0) continue;
      unsigned long long* g = reinterpret_cast<unsigned long long*>(p.gp64) + 4 * (int64_t)node;
      if constexpr (MODE == kModeMassV) {
        const long long mv = sacc[3][t];
        if (mv != 0) {
          atomicAdd(g + 3, (unsigned long long)mv);
          atomicOr(&p.gmask[node], 1u << body);
          if (p.gmb_fx)
            atomicAdd(reinterpret_cast<unsigned long long*>(p.gmb_fx + (int64_t)body * p.n_nodes + node),
                      (unsigned long long)mv);
        }
      }
#pragma unroll
      for (int c = 0; c < 3; ++c)
        if (sacc[c][t] != 0) atomicAdd(g + c, (unsigned long long)sacc[c][t]);
    }
  } else if constexpr (!DET && kP2G) {
    for (int t = t_lo + tid; t < t_hi; t += CHUNK) {
      const int node = node_of(t);
      if (node < 0) continue;
      if constexpr (kMass) {
        T mv;
        if constexpr (kFix) mv = __int_as_float(sacc[3][t]);
        else mv = sacc[3][t];
        if (mv != T(0)) {
          atomicAdd(&p.gm[node], mv);
          atomicOr(&p.gmask[node], 1u << body);
          if (p.gmb) atomicAdd(&p.gmb[(int64_t)body * p.n_nodes + node], mv);
        }
      }
      // the node's sums in the working type (from the fixed-point integers:
      // int -> float, times the power of two 1/T; a non-finite bound in the
      // item gives its nodes NaN, as float sums would)
      T x, y, z;
      bool any;
      if constexpr (kFix) {
        const int ix = sacc[0][t], iy = sacc[1][t], iz = sacc[2][t];
        any = (ix | iy | iz) != 0 || fx_nonfinite;
        const float inv = fx_nonfinite ? __int_as_float(0x7fc00000) : fxInvT;
        x = (float)ix * inv;
        y = (float)iy * inv;
        z = (float)iz * inv;
      } else {
        x = sacc[0][t];
        y = sacc[1][t];
        z = sacc[2][t];
        any = x != T(0) || y != T(0) || z != T(0);
      }
      const double xd = (double)x, yd = (double)y, zd = (double)z;  // (used by the FP64 branches only)
      if (any) {
        if (kMass && p.gp64 != nullptr) {
          // the body mask is not final yet: P2G of V goes to FP64 everywhere
          atomicAdd(&p.gp64[node].x, xd);
          atomicAdd(&p.gp64[node].y, yd);
          atomicAdd(&p.gp64[node].z, zd);
        } else if constexpr (kMaskPre) {
          if (p.gp64 != nullptr && __popc(smk[t]) >= 2) {
            atomicAdd(&p.gp64[node].x, xd);
            atomicAdd(&p.gp64[node].y, yd);
            atomicAdd(&p.gp64[node].z, zd);
          } else {
            atomicAdd(reinterpret_cast<float4*>(&p.gp[node]), make_float4((float)x, (float)y, (float)z, 0.f));
          }
        } else {
          flush_mom(static_cast<T*>(nullptr), p.gp, p.gp64, p.gmask, node, x, y, z);
        }
      }
    }
  }
}

template <class T, int MODE, int MINB, int CHUNK, bool ROWTAB, bool DET = false, int RPL = 1, bool PERSIST = false>
__global__ void __launch_bounds__(CHUNK, MINB) k_items(const IterParams<T> p) {
  grid_dep_launch();
  if constexpr (PERSIST) {
    // Tickets are drawn after the item's grid_dep_wait, so the grid before
    // this one, which used the same counter, has completed.  The launch
    // draws n_items tickets in all (n_items - gridDim.x that name an item,
    // one past the end per CTA), so the counter wraps back to 0.
    __shared__ int s_next;
    int item = blockIdx.x;
    while (item < p.n_items) {
      items_body<T, MODE, MINB, CHUNK, ROWTAB, DET, RPL>(p, item);
      if (p.n_items <= (int)gridDim.x) break;  // one item per CTA: no tickets
      if (threadIdx.x == 0) {
        grid_dep_wait();  // (already passed, unless the item exited early)
        s_next = (int)gridDim.x + (int)atomicInc(p.ticket, (unsigned)(p.n_items - 1));
      }
      __syncthreads();  // also: the next item reuses the shared tiles
      item = s_next;
      __syncthreads();  // every thread has read it before thread 0 writes it again
    }
  } else {
    items_body<T, MODE, MINB, CHUNK, ROWTAB, DET, RPL>(p, blockIdx.x);
  }
}

// v_i = p_i / m_i (0 where m_i = 0), then clear p_i for the next pass.
// The node velocity is stored as (v_x, v_y, v_z, v_z): the repeated v_z lets
// G2P pair it with (N, N d) in one paired FMA.
// Nodes that two or more bodies touch take their momentum from the FP64
// accumulators (FP32 path).
template <class T>
__global__ void k_normalize(int64_t n_nodes, const T* gm, const uint32_t* gmask, V4<T>* gp,
                            V4<double>* gp64, V4<T>* gv, int all64) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  grid_dep_launch();
  grid_dep_wait();
  if (i >= n_nodes) return;
  const T m = gm[i];
  V4<T> v{T(0), T(0), T(0), T(0)};
  if (gp64 != nullptr && (all64 || __popc(gmask[i]) >= 2)) {
    const V4<double> q = gp64[i];
    if (m > T(0)) {
      const double md = (double)m;
      const T vz = (T)(q.z / md);
      v = V4<T>{(T)(q.x / md), (T)(q.y / md), vz, vz};
    }
    gp64[i] = V4<double>{0.0, 0.0, 0.0, 0.0};
  } else {
    const V4<T> q = gp[i];
    if (m > T(0)) v = V4<T>{q.x / m, q.y / m, q.z / m, q.z / m};
  }
  gp[i] = V4<T>{T(0), T(0), T(0), T(0)};
  gv[i] = v;
}

template <class T>
__device__ __forceinline__ bool bad_mass(T m) {
  return !(m > T(0)) || !isfinite((double)m);
}

// Scene of batch particle i / of global page-table entry g (binary search
// over the scenes' offsets; empty scenes share the next scene's offset).
__device__ __forceinline__ int scene_of_particle(const SceneDev* sc, int ns, long long i) {
  int lo = 0, hi = ns - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (sc[mid].part_off <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}
__device__ __forceinline__ int scene_of_page(const SceneDev* sc, int ns, long long g) {
  int lo = 0, hi = ns - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (sc[mid].page_off <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Deterministic mode: node velocities from the fixed-point sums of the pass
// that used bound slot `slot` (all64: the mass pass, which also gives m_i),
// with the scales that pass used; clears the sums for the next pass.
__global__ void k_normalize_fx(int64_t n_nodes, const int* __restrict__ blist, const SceneDev* __restrict__ sc,
                               int ns, float* gm, long long* gfx, V4<float>* gv, const unsigned* fx_max,
                               const int* fx_err, int fx_stride, int slot, int attempt, int all64) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  grid_dep_launch();
  grid_dep_wait();
  if (i >= n_nodes) return;
  const int scene = scene_of_page(sc, ns, blist[i / kNodesPerBlock]);
  const unsigned* fxs = fx_max + (int64_t)scene * fx_stride;
  const int n = sc[scene].n;
  float unused;
  long long* g = gfx + 4 * i;
  float m;
  if (all64) {
    m = from_fx(g[3], 1.f / fx_scale(fxs, 0, 0, n, &unused));
    gm[i] = m;
    g[3] = 0;
  } else {
    m = gm[i];
  }
  const float S = fx_scale(fxs, slot, all64 ? 0 : fx_head(fx_err, attempt, scene), n, &unused);
  V4<float> v{0.f, 0.f, 0.f, 0.f};
  if (m > 0.f) {
    const float inv = 1.f / S;
    const float vz = from_fx(g[2], inv) / m;
    v = V4<float>{from_fx(g[0], inv) / m, from_fx(g[1], inv) / m, vz, vz};
  }
  g[0] = g[1] = g[2] = 0;
  gv[i] = v;
}

// Deterministic mode: per scene, the largest mass (slot 0) and the largest
// term bound b_p of V (slot 1); a bound that is not finite, or beyond the
// 2^90 the scales cover, sets the scene's range flag (err_row[scene]) and
// the attempt's (err_row[ns]).  Each CTA covers a contiguous run of sorted particles and
// keeps the maxima of its first scene in shared memory.
__global__ void k_fx_prep(int64_t n, const SceneDev* __restrict__ sc, int ns, const int* __restrict__ perm,
                          const V4<float>* __restrict__ pt, const V4<float>* __restrict__ V, unsigned* fx_max,
                          int fx_stride, int* err_row, int per_cta) {
  __shared__ unsigned smax[2];
  __shared__ int first_scene;
  const int64_t s0 = (int64_t)blockIdx.x * per_cta;
  const int64_t s1 = min(s0 + per_cta, n);
  if (threadIdx.x == 0) {
    smax[0] = smax[1] = 0u;
    first_scene = s0 < n ? scene_of_particle(sc, ns, perm[s0]) : -1;
  }
  __syncthreads();
  for (int64_t s = s0 + threadIdx.x; s < s1; s += blockDim.x) {
    const int scene = scene_of_particle(sc, ns, perm[s]);
    const V4<float> q0 = V[s], q1 = V[n + s], q2 = V[2 * n + s];
    const float w[3] = {q0.x, q0.y, q0.z};
    const float Ch[9] = {q0.w, q1.x, q1.y, q1.z, q1.w, q2.x, q2.y, q2.z, q2.w};
    const float m = pt[s].w;
    const float b = fx_bound(m, w, Ch);
    if (!(b <= 0x1p90f) || !(m <= 0x1p90f)) {  // NaN, inf or beyond the scales
      atomicOr(err_row + scene, 1);
      atomicOr(err_row + ns, 1);  // any scene of this attempt
    }
    const unsigned bm = __float_as_uint(m), bv = __float_as_uint(b);
    if (scene == first_scene) {
      atomicMax(&smax[0], bm);
      atomicMax(&smax[1], bv);
    } else {
      atomicMax(fx_max + (int64_t)scene * fx_stride, bm);
      atomicMax(fx_max + (int64_t)scene * fx_stride + 1, bv);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && first_scene >= 0) {
    atomicMax(fx_max + (int64_t)first_scene * fx_stride, smax[0]);
    atomicMax(fx_max + (int64_t)first_scene * fx_stride + 1, smax[1]);
  }
}

// floor(x 2^k) for a double x, from its bits with integer instructions only:
// |x| 2^k = mant 2^sh exactly, so the floor is a shift, less one for a
// negative x whose shifted-out bits are not all zero.  The caller keeps the
// result inside +-2^62 (sh <= 9 here).
__device__ __forceinline__ long long floor_pow2_scaled(double x, int k) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((u >> 52) & 0x7ff);
  const unsigned long long mant = (u & 0xfffffffffffffull) | (e != 0 ? (1ull << 52) : 0ull);
  const int sh = (e != 0 ? e : 1) - 1075 + k;
  unsigned long long a;
  bool frac;
  if (sh >= 0) {
    a = mant << sh;
    frac = false;
  } else if (sh > -64) {
    a = mant >> -sh;
    frac = (mant & ((1ull << -sh) - 1ull)) != 0;
  } else {
    a = 0;
    frac = mant != 0;
  }
  return (u >> 63) ? -(long long)(a + (frac ? 1ull : 0ull)) : (long long)a;
}

// Cell of every particle (x/h in FP64, floor), validation, and the bounding
// box of each scene's particle blocks.  A CTA whose particles all belong to
// one scene reduces the box in shared memory and adds it with one set of
// atomics; CTAs that straddle scenes add per particle.  With keys (the boxes
// reused from the step before) the kernel writes the sort keys instead and
// skips the box.
template <class T>
__global__ void k_cells(int64_t n, const SceneDev* __restrict__ sc, int ns, int4* cellb, V4<T>* ptc, int* sbbox,
                        int* errp, int check, void* keys, int key_bytes, int max_bodies) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t p_first = blockIdx.x * (int64_t)blockDim.x;
  const int64_t p_last = min(p_first + blockDim.x, n) - 1;
  __shared__ int uniform_scene;
  if (threadIdx.x == 0) {
    const int a = scene_of_particle(sc, ns, p_first), b = scene_of_particle(sc, ns, p_last);
    uniform_scene = a == b ? a : -1;
  }
  __syncthreads();
  int lo[3] = {INT32_MAX, INT32_MAX, INT32_MAX}, hi[3] = {INT32_MIN, INT32_MIN, INT32_MIN};
  int err = 0;
  int scene = uniform_scene;
  if (p < n) {
    if (scene < 0) scene = scene_of_particle(sc, ns, p);
    const SceneDev& S = sc[scene];
    const int64_t i = p - S.part_off;
    int c[3];
    float t[3];
    // 1/h a power of two 2^lg (h = 1/512 and the like): x / h is exact and
    // its scaled floor comes from the bits of x with integer instructions
    const unsigned long long hb = (unsigned long long)__double_as_longlong(S.inv_h);
    const int he = (int)((hb >> 52) & 0x7ff);
    const bool pow2 = (hb & 0xfffffffffffffull) == 0 && he != 0 && he != 0x7ff;
    const int lg = he - 1023;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      // floor(x 2^32 / h) as a 64-bit integer holds floor(x / h) above bit 32
      // and the offset in the cell's first 32 bits below.  x 2^32 / h is x / h
      // scaled exactly, so its exponent is that of x / h plus 32.  |x/h| < 2^29
      // keeps cells, blocks and their margins inside int32; the tests read
      // exponent bits (and refuse inf and NaN).  The FP64 pipe is narrow on
      // this GPU: the general path takes two FP64 instructions an axis, the
      // power-of-two path none.
      const double xd = S.x[3 * i + d];
      bool bad;
      long long q = 0;
      if (pow2) {
        const int e = (int)((__double_as_longlong(xd) >> 52) & 0x7ff);
        bad = e == 0x7ff || e - 1023 + lg >= 29;
        if (!bad) q = floor_pow2_scaled(xd, lg + 32);
      } else {
        const double xs = xd * (S.inv_h * 4294967296.0);
        bad = (int)((__double_as_longlong(xs) >> 52) & 0x7ff) >= 1023 + 29 + 32;
        if (!bad) q = __double2ll_rd(xs);
      }
      if (bad) {
        err |= kErrPos;
        c[d] = 0;
        t[d] = 0.f;
      } else {
        c[d] = (int)(q >> 32);
        t[d] = (float)(unsigned)(q & 0xffffffffll) * 0x1p-32f;
      }
      lo[d] = hi[d] = c[d] >> 2;
    }
    const int b = S.body[i];
    if (b < 0 || b >= S.n_bodies) err |= kErrBody;
    if (bad_mass(static_cast<const T*>(S.m)[i])) err |= kErrMass;
    if (check && S.v && S.C) {
      const T* v = static_cast<const T*>(S.v) + 3 * i;
      const T* C = static_cast<const T*>(S.C) + 9 * i;
      bool fin = true;
#pragma unroll
      for (int a = 0; a < 3; ++a) fin = fin && isfinite(v[a]);
#pragma unroll
      for (int a = 0; a < 9; ++a) fin = fin && isfinite(C[a]);
      if (S.nrm) {  // (NULL when the normals are computed on the device)
        const T* nr = static_cast<const T*>(S.nrm) + 3 * i;
#pragma unroll
        for (int a = 0; a < 3; ++a) fin = fin && isfinite(nr[a]);
        const T n2 = nr[0] * nr[0] + nr[1] * nr[1] + nr[2] * nr[2];
        if (fin && n2 != T(0) && fabs(n2 - T(1)) > T(1e-3)) err |= kErrNormal;
      }
      if (!fin) err |= kErrFinite;
    }
    if (keys != nullptr) {
      // the scene's page-table box is known (reused from the step before):
      // the sort key here, as k_keys computes it from the cell
      const Box box = S.box;
      int bx = (c[0] >> 2) - box.ox, by = (c[1] >> 2) - box.oy, bz = (c[2] >> 2) - box.oz;
      if (bx < 1 || by < 1 || bz < 1 || bx > box.nx - 2 || by > box.ny - 2 || bz > box.nz - 2) {
        err |= kErrBox;  // a block left the reused box: the host sizes fresh boxes
        bx = min(max(bx, 1), box.nx - 2);
        by = min(max(by, 1), box.ny - 2);
        bz = min(max(bz, 1), box.nz - 2);
      }
      const int64_t gpage = S.page_off + ((int64_t)bz * box.ny + by) * box.nx + bx;
      const uint32_t loc = (uint32_t)(((c[2] & 3) << 4) | ((c[1] & 3) << 2) | (c[0] & 3));
      const uint64_t key = (((uint64_t)gpage * (uint64_t)max_bodies + (uint64_t)(b < 0 ? 0 : b)) << 6) | loc;
      if (key_bytes == 8) static_cast<uint64_t*>(keys)[p] = key;
      else static_cast<uint32_t*>(keys)[p] = (uint32_t)key;
    } else {
      cellb[p] = make_int4(c[0], c[1], c[2], b);
    }
    // FP32 path: the offset in the cell and the mass, in caller order, for
    // the gather (one aligned 16-byte record instead of x and m)
    if (ptc) ptc[p] = V4<T>{(T)t[0], (T)t[1], (T)t[2], static_cast<const T*>(S.m)[i]};
    if (uniform_scene < 0 && keys == nullptr) {
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        atomicMin(&sbbox[6 * scene + d], lo[d]);
        atomicMax(&sbbox[6 * scene + 3 + d], hi[d]);
      }
    }
  }
  if (keys != nullptr) {
    // the boxes are reused and known: no box reduction, only errors
    if (err) atomicOr(errp, err);
    return;
  }
  if (uniform_scene < 0) {
    if (err) atomicOr(errp, err);
    return;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      lo[d] = min(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], off));
      hi[d] = max(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], off));
    }
    err |= __shfl_xor_sync(0xffffffffu, err, off);
  }
  __shared__ int red[7][32];
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      red[d][w] = lo[d];
      red[3 + d][w] = hi[d];
    }
    red[6][w] = err;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const int l = threadIdx.x;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      lo[d] = l < nw ? red[d][l] : INT32_MAX;
      hi[d] = l < nw ? red[3 + d][l] : INT32_MIN;
    }
    err = l < nw ? red[6][l] : 0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        lo[d] = min(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], off));
        hi[d] = max(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], off));
      }
      err |= __shfl_xor_sync(0xffffffffu, err, off);
    }
    if (l == 0 && lo[0] != INT32_MAX) {
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        atomicMin(&sbbox[6 * uniform_scene + d], lo[d]);
        atomicMax(&sbbox[6 * uniform_scene + 3 + d], hi[d]);
      }
      if (err) atomicOr(errp, err);
    }
  }
}

// Sort key: ((global page index of the cell's block) * max_bodies + body) << 6
// | cell-in-block.  Sorting by it groups particles by scene, block and body,
// and orders each group by cell (z-major).
template <class K>
__global__ void k_keys(int64_t n, const SceneDev* __restrict__ sc, int ns, const int4* __restrict__ cellb,
                       int max_bodies, K* keys, int* vals, int* err) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n) return;
  const SceneDev& S = sc[scene_of_particle(sc, ns, p)];
  const Box box = S.box;
  const int4 c = cellb[p];
  int bx = (c.x >> 2) - box.ox, by = (c.y >> 2) - box.oy, bz = (c.z >> 2) - box.oz;
  // every particle block must keep a one-block margin inside the box
  if (bx < 1 || by < 1 || bz < 1 || bx > box.nx - 2 || by > box.ny - 2 || bz > box.nz - 2) {
    atomicOr(err, kErrBox);
    bx = min(max(bx, 1), box.nx - 2);
    by = min(max(by, 1), box.ny - 2);
    bz = min(max(bz, 1), box.nz - 2);
  }
  const int64_t gpage = S.page_off + ((int64_t)bz * box.ny + by) * box.nx + bx;
  const uint32_t loc = (uint32_t)(((c.z & 3) << 4) | ((c.y & 3) << 2) | (c.x & 3));
  keys[p] = (K)((((uint64_t)gpage * (uint64_t)max_bodies + (uint64_t)c.w) << 6) | loc);
  vals[p] = (int)p;
}

// Sorted structure-of-arrays: offset in cell and mass, normal and cell bits,
// and V = (v, h C) in three float4 planes.
template <class T>
__global__ void k_gather(int64_t n, const SceneDev* __restrict__ sc, int ns, const int* __restrict__ perm,
                         const V4<T>* __restrict__ ptc, const void* __restrict__ skeys, int key_bytes, V4<T>* pt,
                         V4<T>* pn, V4<T>* V) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int64_t g = perm[s];
  if (!APIC_DBG_CHECK(g >= 0 && g < n, kDbgPerm)) return;
  const SceneDev& S = sc[scene_of_particle(sc, ns, g)];
  const int64_t i = g - S.part_off;
  uint32_t loc;
  if (ptc != nullptr) {
    // FP32 path: offset and mass from the cell kernel's record, the cell in
    // the block from the sorted key's low six bits
    pt[s] = ptc[g];
    loc = key_bytes == 8 ? (uint32_t)(static_cast<const uint64_t*>(skeys)[s] & 63u)
                         : static_cast<const uint32_t*>(skeys)[s] & 63u;
  } else {
    // FP64 path: the exact FP64 difference x / h - floor(x / h)
    const double* x = S.x;
    int cc[3];
    T tt[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double xs = x[3 * i + d] * S.inv_h;
      cc[d] = __double2int_rd(xs);
      tt[d] = (T)(xs - (double)cc[d]);
    }
    pt[s] = V4<T>{tt[0], tt[1], tt[2], static_cast<const T*>(S.m)[i]};
    loc = (uint32_t)(((cc[2] & 3) << 4) | ((cc[1] & 3) << 2) | (cc[0] & 3));
  }
  if (V == nullptr) {  // normals and V planes gathered later (k_gather_v)
    pn[s] = V4<T>{T(0), T(0), T(0), bits_to(T(0), loc)};
    return;
  }
  const T* nrm = static_cast<const T*>(S.nrm);  // NULL: normals computed on the device later
  pn[s] = nrm ? V4<T>{nrm[3 * i + 0], nrm[3 * i + 1], nrm[3 * i + 2], bits_to(T(0), loc)}
              : V4<T>{T(0), T(0), T(0), bits_to(T(0), loc)};
  const T hh = (T)S.h;
  const T* v = static_cast<const T*>(S.v);
  const T* C = static_cast<const T*>(S.C);
  T vv[3], Ch[9];
#pragma unroll
  for (int a = 0; a < 3; ++a) vv[a] = v[3 * i + a];
#pragma unroll
  for (int a = 0; a < 9; ++a) Ch[a] = C[9 * i + a] * hh;
  store12(V, (int)n, (int)s, vv, Ch);
}

// The normals (into pn's first three components; what & 2) and the V = (v,
// h C) planes (what & 1), in sorted order, when v, C and the normals arrive
// after the sizing sequence has started.
template <class T>
__global__ void k_gather_v(int64_t n, const SceneDev* __restrict__ sc, int ns, const int* __restrict__ perm,
                           V4<T>* pn, V4<T>* V, int what) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int64_t g = perm[s];
  const SceneDev& S = sc[scene_of_particle(sc, ns, g)];
  const int64_t i = g - S.part_off;
  const T* nrm = static_cast<const T*>(S.nrm);
  if ((what & 2) && nrm) {  // NULL: normals computed on the device later
    pn[s].x = nrm[3 * i + 0];
    pn[s].y = nrm[3 * i + 1];
    pn[s].z = nrm[3 * i + 2];
  }
  if (!(what & 1)) return;
  const T hh = (T)S.h;
  const T* v = static_cast<const T*>(S.v);
  const T* C = static_cast<const T*>(S.C);
  T vv[3], Ch[9];
#pragma unroll
  for (int a = 0; a < 3; ++a) vv[a] = v[3 * i + a];
#pragma unroll
  for (int a = 0; a < 9; ++a) Ch[a] = C[9 * i + a] * hh;
  store12(V, (int)n, (int)s, vv, Ch);
}

// Work items, from the sorted keys.  A run is a maximal range of equal
// (grid block, body); a run of len particles splits into k = ceil(len /
// chunk) items of equal size (within one), item j starting at ceil(j len /
// k), so no item is a short tail.  k_run_items: at each run head s, the run's
// end (binary search over the sorted keys) and k; 0 elsewhere.
template <class K>
__global__ void k_run_items(int64_t n, const K* __restrict__ keys, int chunk, int* cnt, int* rend) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= n) return;
  const K q = keys[s] >> 6;
  if (s > 0 && (keys[s - 1] >> 6) == q) {
    cnt[s] = 0;
    return;
  }
  int64_t lo = s + 1, hi = n;  // first index past the run
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if ((keys[mid] >> 6) == q) lo = mid + 1; else hi = mid;
  }
  cnt[s] = (int)((lo - s + chunk - 1) / chunk);
  rend[s] = (int)lo;
}

// The items of each run at their offsets (exclusive sum of cnt): start and
// (global page index of the block, body, scene, 0); the last thread stores
// the item count.
template <class K>
__global__ void k_item_write(int64_t n, const K* __restrict__ keys, const int* __restrict__ cnt,
                             const int* __restrict__ off, const int* __restrict__ rend, int max_bodies,
                             const SceneDev* __restrict__ sc, int ns, int* item_start, int4* item_info,
                             int* n_items) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int k = cnt[s];
  if (s == n - 1) *n_items = off[s] + k;
  if (k == 0) return;
  const int64_t len = rend[s] - s;
  const uint64_t q = (uint64_t)(keys[s] >> 6);
  const long long gpage = (long long)(q / (uint64_t)max_bodies);
  const int4 info = make_int4((int)gpage, (int)(q % (uint64_t)max_bodies), scene_of_page(sc, ns, gpage), 0);
  const int o = off[s];
  for (int j = 0; j < k; ++j) {
    item_start[o + j] = (int)(s + (j * len + k - 1) / k);
    item_info[o + j] = info;
  }
}

// Mark the grid blocks the stencils of one work item reach: one warp per
// item.  Particles of an item share a block B; a particle in cell-in-block l
// reaches block B-1 along an axis when l = 0 and B+1 when l >= 2, so the
// warp ORs those six conditions over its particles and marks the implied
// subset of the 3x3x3 blocks around B (once per item, not per particle).
template <class K>
__global__ void k_mark_items(const int* __restrict__ item_start, const int4* __restrict__ item_info,
                             const int* __restrict__ n_items_p, const K* __restrict__ keys, int64_t n,
                             const SceneDev* __restrict__ sc, int* flags) {
  const int lane = threadIdx.x & 31;
  const int n_items = *n_items_p;
  const int warps = (int)((gridDim.x * (int64_t)blockDim.x) >> 5);
  for (int i = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5); i < n_items; i += warps) {
    const int s0 = item_start[i];
    const int s1 = i + 1 < n_items ? item_start[i + 1] : (int)n;
    unsigned need = 0;
    for (int s = s0 + lane; s < s1; s += 32) {
      const unsigned loc = (unsigned)(keys[s] & 63);
      const unsigned lx = loc & 3, ly = (loc >> 2) & 3, lz = loc >> 4;
      need |= (lx == 0) | ((lx >= 2) << 1) | ((ly == 0) << 2) | ((ly >= 2) << 3) | ((lz == 0) << 4) |
              ((lz >= 2) << 5);
    }
    need = __reduce_or_sync(0xffffffffu, need);
    if (lane < 27) {
      const int dx = lane % 3 - 1, dy = (lane / 3) % 3 - 1, dz = lane / 9 - 1;
      const bool ok = (dx == 0 || (dx < 0 ? (need & 1) : (need & 2))) &&
                      (dy == 0 || (dy < 0 ? (need & 4) : (need & 8))) &&
                      (dz == 0 || (dz < 0 ? (need & 16) : (need & 32)));
      if (ok) {
        const int4 info = item_info[i];
        const SceneDev& S = sc[info.z];
        const Box box = S.box;
        const int blin = (int)(info.x - S.page_off);
        const int bx = blin % box.nx, by = (blin / box.nx) % box.ny, bz = blin / (box.nx * box.ny);
        flags[S.page_off + ((int64_t)(bz + dz) * box.ny + (by + dy)) * box.nx + (bx + dx)] = 1;
      }
    }
  }
}

// Stream compaction after an exclusive scan of 0/1 flags: list the flagged
// indices in order, optionally write each index's compact id (or -1) into
// `page`, and store the count.
__global__ void k_compact(int64_t n, const int* __restrict__ flags, const int* __restrict__ offs,
                          int* list, int* page, int* count) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int f = flags[i], o = offs[i];
  if (f) list[o] = (int)i;
  if (page) page[i] = f ? o : -1;
  if (i == n - 1) *count = o + f;
}

// FP64 totals P = sum m v, L = sum m [x cross v + (h^2/2) axial(C)] and the
// generalised kinetic energy E = sum m (|v|^2 + (h^2/2) |C|_F^2) / 2 (the
// energy of the mass inner product under which H is a contraction).
template <class T>
__global__ void k_momentum(int64_t n, const double* __restrict__ x, const T* __restrict__ v,
                           const T* __restrict__ C, const T* __restrict__ m, double h2half,
                           double* out7) {
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    const double mm = (double)m[p];
    const double x0 = x[3 * p], x1 = x[3 * p + 1], x2 = x[3 * p + 2];
    const double v0 = (double)v[3 * p], v1 = (double)v[3 * p + 1], v2 = (double)v[3 * p + 2];
    const T* c = C + 9 * p;
    acc[0] += mm * v0;
    acc[1] += mm * v1;
    acc[2] += mm * v2;
    acc[3] += mm * (x1 * v2 - x2 * v1 + h2half * ((double)c[7] - (double)c[5]));
    acc[4] += mm * (x2 * v0 - x0 * v2 + h2half * ((double)c[2] - (double)c[6]));
    acc[5] += mm * (x0 * v1 - x1 * v0 + h2half * ((double)c[3] - (double)c[1]));
    double cc = 0.0;
#pragma unroll
    for (int a = 0; a < 9; ++a) cc += (double)c[a] * (double)c[a];
    acc[6] += 0.5 * mm * (v0 * v0 + v1 * v1 + v2 * v2 + h2half * cc);
  }
#pragma unroll
  for (int k = 0; k < 7; ++k)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], off);
  __shared__ double red[7][32];
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int k = 0; k < 7; ++k) red[k][w] = acc[k];
  __syncthreads();
  if (threadIdx.x < 32) {
#pragma unroll
    for (int k = 0; k < 7; ++k) {
      double v = threadIdx.x < nw ? red[k][threadIdx.x] : 0.0;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
      if (threadIdx.x == 0) atomicAdd(&out7[k], v);
    }
  }
}

// Per-scene diagnostics: multi-body nodes and active blocks (from the
// compact block list) and work items.
__global__ void k_scene_counts(int n_blocks, const int* __restrict__ blist, const uint32_t* __restrict__ gmask,
                               int n_items, const int4* __restrict__ item_info, const SceneDev* __restrict__ sc,
                               int ns, unsigned long long* out) {
  const int stride = gridDim.x * blockDim.x;
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < n_blocks; b += stride) {
    const int scene = scene_of_page(sc, ns, blist[b]);
    int mb = 0;
    for (int k = 0; k < kNodesPerBlock; ++k) mb += __popc(gmask[(int64_t)b * kNodesPerBlock + k]) >= 2;
    if (mb) atomicAdd(&out[3 * scene + 0], (unsigned long long)mb);
    atomicAdd(&out[3 * scene + 1], 1ull);
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_items; i += stride)
    atomicAdd(&out[3 * item_info[i].z + 2], 1ull);
}

// x += dt v (the serving loop's optional advection after a contact step).
template <class T>
__global__ void k_advect(int64_t n, double* __restrict__ x, const T* __restrict__ v, double dt) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < 3 * n) x[i] += dt * (double)v[i];
}

inline unsigned grid_for(int64_t n, int threads) {
  return (unsigned)((n + threads - 1) / threads);
}

}  // namespace

template <class T>
cudaError_t launch_cells(int64_t n, const SceneDev* sc, int ns, int4* cellb, V4<T>* ptc, int* sbbox, int* err,
                         int check, void* keys, int key_bytes, int max_bodies, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_cells<T><<<grid_for(n, 256), 256, 0, s>>>(n, sc, ns, cellb, ptc, sbbox, err, check, keys, key_bytes,
                                               max_bodies);
  return cudaGetLastError();
}

template <class K>
cudaError_t launch_keys(int64_t n, const SceneDev* sc, int ns, const int4* cellb, int max_bodies, K* keys,
                        int* vals, int* err, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_keys<K><<<grid_for(n, 256), 256, 0, s>>>(n, sc, ns, cellb, max_bodies, keys, vals, err);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_gather(int64_t n, const SceneDev* sc, int ns, const int* perm, const V4<T>* ptc, const void* skeys,
                          int key_bytes, V4<T>* pt, V4<T>* pn, V4<T>* V, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_gather<T><<<grid_for(n, 256), 256, 0, s>>>(n, sc, ns, perm, ptc, skeys, key_bytes, pt, pn, V);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_gather_v(int64_t n, const SceneDev* sc, int ns, const int* perm, V4<T>* pn, V4<T>* V,
                            int what, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_gather_v<T><<<grid_for(n, 256), 256, 0, s>>>(n, sc, ns, perm, pn, V, what);
  return cudaGetLastError();
}

template <class K>
cudaError_t launch_run_items(int64_t n, const K* keys, int chunk, int* cnt, int* rend, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (chunk < 16 || chunk > kChunk) return cudaErrorInvalidValue;
  k_run_items<K><<<grid_for(n, 256), 256, 0, s>>>(n, keys, chunk, cnt, rend);
  return cudaGetLastError();
}

template <class K>
cudaError_t launch_item_write(int64_t n, const K* keys, const int* cnt, const int* off, const int* rend,
                              int max_bodies, const SceneDev* sc, int ns, int* item_start, int4* item_info,
                              int* n_items, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_item_write<K><<<grid_for(n, 256), 256, 0, s>>>(n, keys, cnt, off, rend, max_bodies, sc, ns, item_start,
                                                   item_info, n_items);
  return cudaGetLastError();
}

template <class K>
cudaError_t launch_mark_items(const int* item_start, const int4* item_info, const int* n_items, const K* keys,
                              int64_t n, int max_items, const SceneDev* sc, int* flags, cudaStream_t s) {
  if (max_items <= 0) return cudaSuccess;
  const int64_t warps = std::min<int64_t>(max_items, 152 * 64);
  k_mark_items<K><<<(unsigned)((warps * 32 + 255) / 256), 256, 0, s>>>(item_start, item_info, n_items, keys, n,
                                                                       sc, flags);
  return cudaGetLastError();
}

cudaError_t launch_compact(int64_t n, const int* flags, const int* offs, int* list, int* page, int* count,
                           cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_compact<<<grid_for(n, 256), 256, 0, s>>>(n, flags, offs, list, page, count);
  return cudaGetLastError();
}

// One launch, with programmatic stream serialization when `overlap` (the
// grid may start while the one before it in the stream still runs; see
// grid_dep_wait).
template <class... P, class... A>
cudaError_t launch_ex(void (*kernel)(P...), unsigned grid, unsigned block, bool overlap, cudaStream_t s,
                      A... args) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = overlap ? 1 : 0;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, args...);
  return e != cudaSuccess ? e : cudaGetLastError();
}

// Resident CTAs of a persistent grid: MINB per SM (the kernel's register
// cap), never more than the items.
inline unsigned persistent_grid(int n_items, int minb) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    sms = 1;
  return (unsigned)std::min<long long>((long long)n_items, (long long)sms * minb);
}

template <class T, int MINB, int CHUNK, bool ROWTAB, int RPL, bool PERSIST>
cudaError_t launch_items_cfg(const IterParams<T>& p, int mode, bool overlap, cudaStream_t s) {
  const unsigned grid = PERSIST ? persistent_grid(p.n_items, MINB) : (unsigned)p.n_items;
  switch (mode) {
#define APIC_MODE(m) \
  case m: return launch_ex(k_items<T, m, MINB, CHUNK, ROWTAB, false, RPL, PERSIST>, grid, CHUNK, overlap, s, p);
    APIC_MODE(kModeFirst)
    APIC_MODE(kModeMid)
    APIC_MODE(kModeLast)
    APIC_MODE(kModeOnly)
    APIC_MODE(kModeMu)
    APIC_MODE(kModeMassV)
    APIC_MODE(kModeNormals)
#undef APIC_MODE
    default: return cudaErrorInvalidValue;
  }
}

// Deterministic mode: the modes of the FP32 step, variant 0's CTA shape.
template <class T>
cudaError_t launch_items_fx(const IterParams<T>& p, int mode, bool overlap, cudaStream_t s) {
  constexpr int B = kVariantMinBlocks[0], C = kVariantThreads[0];
  const unsigned grid = (unsigned)p.n_items;
  switch (mode) {
#define APIC_MODE(m) \
  case m: return launch_ex(k_items<T, m, B, C, false, true>, grid, C, overlap, s, p);
    APIC_MODE(kModeFirst)
    APIC_MODE(kModeMid)
    APIC_MODE(kModeLast)
    APIC_MODE(kModeOnly)
    APIC_MODE(kModeMu)
    APIC_MODE(kModeMassV)
    APIC_MODE(kModeNormals)
#undef APIC_MODE
    default: return cudaErrorInvalidValue;
  }
}

template <class T>
cudaError_t launch_items(const IterParams<T>& p, int mode, int variant, bool overlap, cudaStream_t s) {
  if (p.n_items <= 0) return cudaSuccess;
  if (variant < 0 || variant >= kNumVariants) return cudaErrorInvalidValue;
  if constexpr (sizeof(T) == 4) {
    if (p.fx_max != nullptr) return variant == 0 ? launch_items_fx<T>(p, mode, overlap, s) : cudaErrorInvalidValue;
  }
  if constexpr (sizeof(T) == 4) {
    // the FP32 path is built in every variant
#define APIC_VARIANT(v)                                                                               \
  launch_items_cfg<T, kVariantMinBlocks[v], kVariantThreads[v], kVariantRowTab[v], kVariantRPL[v],       \
                   kVariantPersist[v]>(p, mode, overlap, s)
    switch (variant) {
      case 1: return APIC_VARIANT(1);
      case 2: return APIC_VARIANT(2);
      case 3: return APIC_VARIANT(3);
      case 4: return APIC_VARIANT(4);
      case 5: return APIC_VARIANT(5);
      case 6: return APIC_VARIANT(6);
      case 7: return APIC_VARIANT(7);
      case 8: return APIC_VARIANT(8);
      default: break;
    }
  }
  // the FP64 path (parity and small scenes) only in variant 0
  return APIC_VARIANT(0);
#undef APIC_VARIANT
}

// ---- partitions of one scene: the ghost sum of shared grid blocks ----

__global__ void k_halo_map(int n_blocks, const int* __restrict__ blist, const SceneDev* __restrict__ sc, int ns,
                           const int* __restrict__ page, int* __restrict__ rep) {
  const int cb = blockIdx.x * blockDim.x + threadIdx.x;
  if (cb >= n_blocks) return;
  const long long pg = blist[cb];
  const int s = scene_of_page(sc, ns, pg);
  const Box b = sc[s].box;
  const long long local = pg - sc[s].page_off;
  const int gx = (int)(local % b.nx) + b.ox, gy = (int)((local / b.nx) % b.ny) + b.oy,
            gz = (int)(local / ((long long)b.nx * b.ny)) + b.oz;
  int r = -1;
  for (int s2 = 0; s2 < s && r < 0; ++s2) {
    const Box b2 = sc[s2].box;
    const int lx = gx - b2.ox, ly = gy - b2.oy, lz = gz - b2.oz;
    if (lx < 0 || ly < 0 || lz < 0 || lx >= b2.nx || ly >= b2.ny || lz >= b2.nz) continue;
    r = page[sc[s2].page_off + ((long long)lz * b2.ny + ly) * b2.nx + lx];
  }
  rep[cb] = r;
}

template <class T>
__global__ void k_halo_add(int n_blocks, const int* __restrict__ rep, V4<T>* gp, V4<double>* gp64, T* gm,
                           uint32_t* gmask, T* gmb, int max_bodies, int64_t n_nodes, int mass) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)n_blocks * kNodesPerBlock) return;
  const int r = rep[t / kNodesPerBlock];
  if (r < 0) return;
  const int64_t i = t, j = (int64_t)r * kNodesPerBlock + t % kNodesPerBlock;
  const V4<T> q = gp[i];
  atomicAdd(&gp[j].x, q.x);
  atomicAdd(&gp[j].y, q.y);
  atomicAdd(&gp[j].z, q.z);
  if (gp64) {
    const V4<double> d = gp64[i];
    atomicAdd(&gp64[j].x, d.x);
    atomicAdd(&gp64[j].y, d.y);
    atomicAdd(&gp64[j].z, d.z);
  }
  if (mass) {
    atomicAdd(&gm[j], gm[i]);
    atomicOr(&gmask[j], gmask[i]);
    if (gmb)
      for (int b = 0; b < max_bodies; ++b) atomicAdd(&gmb[b * n_nodes + j], gmb[b * n_nodes + i]);
  }
}

template <class T>
__global__ void k_halo_copy(int n_blocks, const int* __restrict__ rep, V4<T>* gp, V4<double>* gp64, T* gm,
                            uint32_t* gmask, T* gmb, int max_bodies, int64_t n_nodes, int mass) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)n_blocks * kNodesPerBlock) return;
  const int r = rep[t / kNodesPerBlock];
  if (r < 0) return;
  const int64_t i = t, j = (int64_t)r * kNodesPerBlock + t % kNodesPerBlock;
  gp[i] = gp[j];
  if (gp64) gp64[i] = gp64[j];
  if (mass) {
    gm[i] = gm[j];
    gmask[i] = gmask[j];
    if (gmb)
      for (int b = 0; b < max_bodies; ++b) gmb[b * n_nodes + i] = gmb[b * n_nodes + j];
  }
}

cudaError_t launch_halo_map(int n_blocks, const int* blist, const SceneDev* sc, int ns, const int* page, int* rep,
                            cudaStream_t s) {
  if (n_blocks <= 0) return cudaSuccess;
  k_halo_map<<<(n_blocks + 255) / 256, 256, 0, s>>>(n_blocks, blist, sc, ns, page, rep);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_halo_sum(int n_blocks, const int* rep, V4<T>* gp, V4<double>* gp64, T* gm, uint32_t* gmask,
                            T* gmb, int max_bodies, int64_t n_nodes, bool mass, cudaStream_t s) {
  if (n_blocks <= 0) return cudaSuccess;
  const int64_t n = (int64_t)n_blocks * kNodesPerBlock;
  k_halo_add<T><<<grid_for(n, 256), 256, 0, s>>>(n_blocks, rep, gp, gp64, gm, gmask, gmb, max_bodies, n_nodes,
                                                  mass ? 1 : 0);
  k_halo_copy<T><<<grid_for(n, 256), 256, 0, s>>>(n_blocks, rep, gp, gp64, gm, gmask, gmb, max_bodies, n_nodes,
                                                   mass ? 1 : 0);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_normalize(int64_t n_nodes, const T* gm, const uint32_t* gmask, V4<T>* gp,
                             V4<double>* gp64, V4<T>* gv, int all64, bool overlap, cudaStream_t s) {
  if (n_nodes <= 0) return cudaSuccess;
  return launch_ex(k_normalize<T>, grid_for(n_nodes, 256), 256, overlap, s, n_nodes, gm, gmask, gp, gp64, gv,
                   all64);
}

cudaError_t launch_fx_prep(int64_t n, const SceneDev* sc, int ns, const int* perm, const V4<float>* pt,
                           const V4<float>* V, unsigned* fx_max, int fx_stride, int* err_row, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int per_cta = 4096;
  k_fx_prep<<<grid_for(n, per_cta), 256, 0, s>>>(n, sc, ns, perm, pt, V, fx_max, fx_stride, err_row, per_cta);
  return cudaGetLastError();
}

cudaError_t launch_normalize_fx(int64_t n_nodes, const int* blist, const SceneDev* sc, int ns, float* gm,
                                long long* gfx, V4<float>* gv, const unsigned* fx_max, const int* fx_err,
                                int fx_stride, int slot, int attempt, int all64, bool overlap, cudaStream_t s) {
  if (n_nodes <= 0) return cudaSuccess;
  return launch_ex(k_normalize_fx, grid_for(n_nodes, 256), 256, overlap, s, n_nodes, blist, sc, ns, gm, gfx, gv,
                   fx_max, fx_err, fx_stride, slot, attempt, all64);
}

template <class T>
cudaError_t launch_momentum(int64_t n, const double* x, const T* v, const T* C, const T* m, double h,
                            double* out7, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  unsigned g = grid_for(n, 256);
  if (g > 608) g = 608;
  k_momentum<T><<<g, 256, 0, s>>>(n, x, v, C, m, 0.5 * h * h, out7);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_advect(int64_t n, double* x, const T* v, double dt, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_advect<T><<<grid_for(3 * n, 256), 256, 0, s>>>(n, x, v, dt);
  return cudaGetLastError();
}

cudaError_t launch_scene_counts(int n_blocks, const int* blist, const uint32_t* gmask, int n_items,
                                const int4* item_info, const SceneDev* sc, int ns, unsigned long long* out,
                                cudaStream_t s) {
  const int work = std::max(n_blocks, n_items);
  if (work <= 0) return cudaSuccess;
  const unsigned g = (unsigned)std::min<int64_t>(grid_for(work, 256), 152 * 8);
  k_scene_counts<<<g, 256, 0, s>>>(n_blocks, blist, gmask, n_items, item_info, sc, ns, out);
  return cudaGetLastError();
}

// Sec. 2.3 node normals, step 1: per boundary triangle (a, b, c), half the
// cross product (b - a) x (c - a) -- the face's area times its outward unit
// normal -- added to each of its nodes in FP64.  A triangle with an index
// outside [0, n) is skipped and flagged.
__global__ void k_face_normals(int64_t n_tri, const int32_t* tri, const double* x, int64_t n, double* acc,
                               int* err) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < n_tri; f += stride) {
    const int32_t v[3] = {tri[3 * f], tri[3 * f + 1], tri[3 * f + 2]};
    if (v[0] < 0 || v[1] < 0 || v[2] < 0 || v[0] >= n || v[1] >= n || v[2] >= n) {
      atomicOr(err, kErrBody);
      continue;
    }
    double e1[3], e2[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const double xa = x[3 * (int64_t)v[0] + k];
      e1[k] = x[3 * (int64_t)v[1] + k] - xa;
      e2[k] = x[3 * (int64_t)v[2] + k] - xa;
    }
    const double an[3] = {0.5 * (e1[1] * e2[2] - e1[2] * e2[1]), 0.5 * (e1[2] * e2[0] - e1[0] * e2[2]),
                          0.5 * (e1[0] * e2[1] - e1[1] * e2[0])};
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int k = 0; k < 3; ++k) atomicAdd(&acc[3 * (int64_t)v[c] + k], an[k]);
  }
}

// Step 2: n_p = s_p / |s_p|, 0 where the weighted sum vanishes (nodes on no
// face, or on zero-area faces only).
template <class T>
__global__ void k_unit_normals(int64_t n, const double* acc, T* out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double s0 = acc[3 * i], s1 = acc[3 * i + 1], s2 = acc[3 * i + 2];
  const double len = sqrt(s0 * s0 + s1 * s1 + s2 * s2);
  const double r = len > 0.0 ? 1.0 / len : 0.0;
  out[3 * i] = (T)(s0 * r);
  out[3 * i + 1] = (T)(s1 * r);
  out[3 * i + 2] = (T)(s2 * r);
}

cudaError_t launch_face_normals(int64_t n_tri, const int32_t* tri, const double* x, int64_t n, double* acc,
                                int* err, cudaStream_t s) {
  if (n_tri <= 0) return cudaSuccess;
  const unsigned g = (unsigned)std::min<int64_t>(grid_for(n_tri, 256), 152 * 16);
  k_face_normals<<<g, 256, 0, s>>>(n_tri, tri, x, n, acc, err);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_unit_normals(int64_t n, const double* acc, T* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_unit_normals<T><<<grid_for(n, 256), 256, 0, s>>>(n, acc, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Augury dynamics (Sec. 2.2, eq. apic_accel, eq. Newmark read as velocity
// Verlet) with a linear-spring foreground.  One step:
//   kick+drift:  V += dt/2 A; x += dt v            (fixed nodes: V = 0)
//   springs:     f = sum k (|d| - L0) d / |d|      (FP64 sums)
//   predict:     a = f / m + g; V_bar = V + c {a, 0}, c = dt/2 + tau
//   contact:     V_hat = contact step of V_bar      (the library's step)
//   finish:      A = {a, 0} + (V_hat - V_bar) / tau; V += dt/2 A
// (with c = tau and no kicks for the initial acceleration).

template <class T>
__global__ void k_aug_kick_drift(int64_t n, double* x, T* v, T* C, const T* av, const T* aC, const uint8_t* fixed,
                                 T half_dt, double dt) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n) return;
  const bool held = fixed != nullptr && fixed[p] != 0;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const T vn = held ? T(0) : v[3 * p + c] + half_dt * av[3 * p + c];
    v[3 * p + c] = vn;
    x[3 * p + c] += dt * (double)vn;
  }
#pragma unroll
  for (int c = 0; c < 9; ++c) C[9 * p + c] = held ? T(0) : C[9 * p + c] + half_dt * aC[9 * p + c];
}

__global__ void k_aug_springs(int64_t n_springs, const int32_t* springs, const double* rest, const double* k,
                              const double* x, int64_t n, double* f, int* err) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n_springs; s += stride) {
    const int32_t i = springs[2 * s], j = springs[2 * s + 1];
    if (i < 0 || j < 0 || i >= n || j >= n) {
      atomicOr(err, kErrBody);
      continue;
    }
    double d[3], len2 = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      d[c] = x[3 * (int64_t)j + c] - x[3 * (int64_t)i + c];
      len2 += d[c] * d[c];
    }
    const double len = sqrt(len2);
    if (!(len > 0.0)) continue;
    const double fs = k[s] * (len - rest[s]) / len;  // pulls i toward j when stretched
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      atomicAdd(&f[3 * (int64_t)i + c], fs * d[c]);
      atomicAdd(&f[3 * (int64_t)j + c], -fs * d[c]);
    }
  }
}

template <class T>
__global__ void k_aug_predict(int64_t n, const double* f, const T* m, double gx, double gy, double gz, const T* v,
                              T* am, T* vbar, T c_bar) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n) return;
  const double g[3] = {gx, gy, gz};
  const double mp = (double)m[p];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const T a = (T)(f[3 * p + c] / mp + g[c]);
    am[3 * p + c] = a;
    vbar[3 * p + c] = v[3 * p + c] + c_bar * a;
  }
}

template <class T>
__global__ void k_aug_finish(int64_t n, const T* am, const T* vbar, const T* vhat, const T* Chat, const uint8_t* fixed,
                             T inv_tau, T half_dt, T* v, T* C, T* av, T* aC) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n) return;
  const bool held = fixed != nullptr && fixed[p] != 0;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const T a = held ? T(0) : am[3 * p + c] + (vhat[3 * p + c] - vbar[3 * p + c]) * inv_tau;
    av[3 * p + c] = a;
    v[3 * p + c] += half_dt * a;
  }
#pragma unroll
  for (int c = 0; c < 9; ++c) {
    const T a = held ? T(0) : (Chat[9 * p + c] - C[9 * p + c]) * inv_tau;
    aC[9 * p + c] = a;
    C[9 * p + c] += half_dt * a;
  }
}

// out[0] += sum 1/2 m |v|^2, out[1] += sum 1/2 k (|d| - L0)^2, out[2] += -sum m g.x
template <class T>
__global__ void k_aug_energy(int64_t n, const double* x, const T* v, const T* m, double gx, double gy, double gz,
                             int64_t n_springs, const int32_t* springs, const double* rest, const double* k,
                             double* out) {
  double e[3] = {0.0, 0.0, 0.0};
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (int64_t p = t0; p < n; p += stride) {
    const double mp = (double)m[p];
    double v2 = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) v2 += (double)v[3 * p + c] * (double)v[3 * p + c];
    e[0] += 0.5 * mp * v2;
    e[2] -= mp * (gx * x[3 * p] + gy * x[3 * p + 1] + gz * x[3 * p + 2]);
  }
  for (int64_t s = t0; s < n_springs; s += stride) {
    const int32_t i = springs[2 * s], j = springs[2 * s + 1];
    if (i < 0 || j < 0 || i >= n || j >= n) continue;
    double len2 = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double d = x[3 * (int64_t)j + c] - x[3 * (int64_t)i + c];
      len2 += d * d;
    }
    const double ex = sqrt(len2) - rest[s];
    e[1] += 0.5 * k[s] * ex * ex;
  }
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    double val = e[q];
    for (int o = 16; o > 0; o >>= 1) val += __shfl_down_sync(0xffffffffu, val, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&out[q], val);
  }
}

template <class T>
cudaError_t launch_aug_kick_drift(int64_t n, double* x, T* v, T* C, const T* av, const T* aC, const uint8_t* fixed,
                                  T half_dt, double dt, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_aug_kick_drift<T><<<grid_for(n, 256), 256, 0, s>>>(n, x, v, C, av, aC, fixed, half_dt, dt);
  return cudaGetLastError();
}

cudaError_t launch_aug_springs(int64_t n_springs, const int32_t* springs, const double* rest, const double* k,
                               const double* x, int64_t n, double* f, int* err, cudaStream_t s) {
  if (n_springs <= 0) return cudaSuccess;
  const unsigned g = (unsigned)std::min<int64_t>(grid_for(n_springs, 256), 152 * 16);
  k_aug_springs<<<g, 256, 0, s>>>(n_springs, springs, rest, k, x, n, f, err);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_aug_predict(int64_t n, const double* f, const T* m, const double* g, const T* v, T* am, T* vbar,
                               T c_bar, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_aug_predict<T><<<grid_for(n, 256), 256, 0, s>>>(n, f, m, g[0], g[1], g[2], v, am, vbar, c_bar);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_aug_finish(int64_t n, const T* am, const T* vbar, const T* vhat, const T* Chat,
                              const uint8_t* fixed, T inv_tau, T half_dt, T* v, T* C, T* av, T* aC,
                              cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_aug_finish<T><<<grid_for(n, 256), 256, 0, s>>>(n, am, vbar, vhat, Chat, fixed, inv_tau, half_dt, v, C, av, aC);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_aug_energy(int64_t n, const double* x, const T* v, const T* m, const double* g, int64_t n_springs,
                              const int32_t* springs, const double* rest, const double* k, double* out,
                              cudaStream_t s) {
  const unsigned gr = (unsigned)std::min<int64_t>(grid_for(std::max<int64_t>(std::max<int64_t>(n, n_springs), 1), 256), 608);
  k_aug_energy<T><<<gr, 256, 0, s>>>(n, x, v, m, g[0], g[1], g[2], n_springs, springs, rest, k, out);
  return cudaGetLastError();
}

// Table-driven copies (host staging of caller arrays in page-locked memory):
// blockIdx.y picks the entry, the x-blocks stride over its bytes.  With
// 4-byte granularity the copy moves 16-byte words whenever either end is
// 16-byte aligned (that end, usually the host side of the link, gets whole
// 16-byte accesses; the other is split into 4-byte ones), then a 4-byte tail;
// otherwise bytes.
// Copy bytes [0, len) of src to dst with the threads t0, t0 + stride, ...:
// 16-byte accesses when both ends allow them (four in flight per thread, so
// that a small grid still fills the host link), 4-byte ones when only one
// does, then a 4-byte tail; bytes when the ends are not 4-byte aligned.
__device__ __forceinline__ void copy_range(const void* srcp, void* dstp, long long len, int64_t t0, int64_t stride) {
  const uintptr_t sa = (uintptr_t)srcp, da = (uintptr_t)dstp;
  if (((sa | da | (uintptr_t)len) & 3) == 0) {
    const bool s16 = (sa & 15) == 0, d16 = (da & 15) == 0;
    const uint32_t* src = static_cast<const uint32_t*>(srcp);
    uint32_t* dst = static_cast<uint32_t*>(dstp);
    int64_t done_words = 0;
    const int64_t n16 = len / 16;
    if (s16 && d16) {
      const uint4* s4 = static_cast<const uint4*>(srcp);
      uint4* d4 = static_cast<uint4*>(dstp);
      for (int64_t i = t0; i < n16; i += 4 * stride) {
        uint4 w[4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (i + k * stride < n16) w[k] = s4[i + k * stride];
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (i + k * stride < n16) d4[i + k * stride] = w[k];
      }
      done_words = 4 * n16;
    } else if (s16 || d16) {
      for (int64_t i = t0; i < n16; i += stride) {
        uint4 w;
        if (s16) {
          w = static_cast<const uint4*>(srcp)[i];
        } else {
          w = make_uint4(src[4 * i], src[4 * i + 1], src[4 * i + 2], src[4 * i + 3]);
        }
        if (d16) {
          static_cast<uint4*>(dstp)[i] = w;
        } else {
          dst[4 * i] = w.x;
          dst[4 * i + 1] = w.y;
          dst[4 * i + 2] = w.z;
          dst[4 * i + 3] = w.w;
        }
      }
      done_words = 4 * n16;
    }
    for (int64_t i = done_words + t0; i < len / 4; i += stride) dst[i] = src[i];
  } else {
    const unsigned char* src = static_cast<const unsigned char*>(srcp);
    unsigned char* dst = static_cast<unsigned char*>(dstp);
    for (int64_t i = t0; i < len; i += stride) dst[i] = src[i];
  }
}

// One entry per grid row, its bytes spread over the row's CTAs.
__global__ void k_copy_table(const CopyEntry* __restrict__ table, int n_entries) {
  const int e = blockIdx.y;
  if (e >= n_entries) return;
  const CopyEntry c = table[e];
  copy_range(c.src, c.dst, c.bytes, blockIdx.x * (int64_t)blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x);
}

// With a CTA budget: the entries' bytes as one sequence of kCopyChunk-byte
// chunks (an entry's last one may be short); CTA b copies the contiguous
// chunks [b C / G, (b + 1) C / G) of the C chunks, walking the entries in
// order (chunk0 is each entry's first chunk).
constexpr long long kCopyChunk = 64 << 10;
__global__ void k_copy_chunks(const CopyEntry* __restrict__ table, int n_entries, long long n_chunks) {
  __shared__ int s_e;
  const long long c0 = (long long)blockIdx.x * n_chunks / gridDim.x;
  const long long c1 = (long long)(blockIdx.x + 1) * n_chunks / gridDim.x;
  if (c0 >= c1) return;
  if (threadIdx.x == 0) {
    int lo = 0, hi = n_entries - 1;  // the last entry whose first chunk is <= c0
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (table[mid].chunk0 <= c0) lo = mid;
      else hi = mid - 1;
    }
    s_e = lo;
  }
  __syncthreads();
  int e = s_e;
  CopyEntry ent = table[e];
  for (long long c = c0; c < c1; ++c) {
    while (e + 1 < n_entries && table[e + 1].chunk0 <= c) ent = table[++e];
    const long long off = (c - ent.chunk0) * kCopyChunk;
    const long long len = ent.bytes - off < kCopyChunk ? ent.bytes - off : kCopyChunk;
    if (len > 0)
      copy_range(static_cast<const char*>(ent.src) + off, static_cast<char*>(ent.dst) + off, len, threadIdx.x,
                 blockDim.x);
  }
}

cudaError_t launch_copy_table(CopyEntry* table, int n_entries, long long max_bytes, cudaStream_t s,
                              int max_ctas) {
  if (n_entries <= 0 || max_bytes <= 0) return cudaSuccess;
  if (n_entries > 65535) return cudaErrorInvalidValue;
  if (max_ctas > 0) {
    long long chunks = 0;
    for (int e = 0; e < n_entries; ++e) {
      table[e].chunk0 = chunks;
      chunks += (table[e].bytes + kCopyChunk - 1) / kCopyChunk;
    }
    if (chunks == 0) return cudaSuccess;
    const unsigned g = (unsigned)std::min<long long>(chunks, max_ctas);
    k_copy_chunks<<<g, 256, 0, s>>>(table, n_entries, chunks);
    return cudaGetLastError();
  }
  const long long gx = std::min<long long>(std::max<long long>((max_bytes + 16383) / 16384, 1), 304);
  k_copy_table<<<dim3((unsigned)gx, (unsigned)n_entries), 256, 0, s>>>(table, n_entries);
  return cudaGetLastError();
}

#define APIC_INST_T(T)                                                                                  \
  template cudaError_t launch_cells<T>(int64_t, const SceneDev*, int, int4*, V4<T>*, int*, int*, int,     \
                                       void*, int, int, cudaStream_t);                                  \
  template cudaError_t launch_gather<T>(int64_t, const SceneDev*, int, const int*, const V4<T>*,         \
                                        const void*, int, V4<T>*, V4<T>*, V4<T>*, cudaStream_t);         \
  template cudaError_t launch_gather_v<T>(int64_t, const SceneDev*, int, const int*, V4<T>*, V4<T>*,     \
                                          int, cudaStream_t);                                                \
  template cudaError_t launch_items<T>(const IterParams<T>&, int, int, bool, cudaStream_t);             \
  template cudaError_t launch_halo_sum<T>(int, const int*, V4<T>*, V4<double>*, T*, uint32_t*, T*, int,   \
                                          int64_t, bool, cudaStream_t);                                 \
  template cudaError_t launch_normalize<T>(int64_t, const T*, const uint32_t*, V4<T>*, V4<double>*,     \
                                           V4<T>*, int, bool, cudaStream_t);                            \
  template cudaError_t launch_momentum<T>(int64_t, const double*, const T*, const T*, const T*, double, \
                                          double*, cudaStream_t);                                       \
  template cudaError_t launch_advect<T>(int64_t, double*, const T*, double, cudaStream_t);                \
  template cudaError_t launch_unit_normals<T>(int64_t, const double*, T*, cudaStream_t);                 \
  template cudaError_t launch_aug_kick_drift<T>(int64_t, double*, T*, T*, const T*, const T*, const uint8_t*, T,  \
                                                double, cudaStream_t);                                    \
  template cudaError_t launch_aug_predict<T>(int64_t, const double*, const T*, const double*, const T*, T*, T*, \
                                             T, cudaStream_t);                                            \
  template cudaError_t launch_aug_finish<T>(int64_t, const T*, const T*, const T*, const T*, const uint8_t*, T, \
                                            T, T*, T*, T*, T*, cudaStream_t);                              \
  template cudaError_t launch_aug_energy<T>(int64_t, const double*, const T*, const T*, const double*, int64_t, \
                                            const int32_t*, const double*, const double*, double*, cudaStream_t);
APIC_INST_T(float)
APIC_INST_T(double)

#define APIC_INST_K(K)                                                                                     \
  template cudaError_t launch_keys<K>(int64_t, const SceneDev*, int, const int4*, int, K*, int*, int*,     \
                                      cudaStream_t);                                                       \
  template cudaError_t launch_run_items<K>(int64_t, const K*, int, int*, int*, cudaStream_t);            \
  template cudaError_t launch_item_write<K>(int64_t, const K*, const int*, const int*, const int*, int,     \
                                            const SceneDev*, int, int*, int4*, int*, cudaStream_t);         \
  template cudaError_t launch_mark_items<K>(const int*, const int4*, const int*, const K*, int64_t, int,   \
                                            const SceneDev*, int*, cudaStream_t);
APIC_INST_K(uint32_t)
APIC_INST_K(uint64_t)

}  // namespace apic
