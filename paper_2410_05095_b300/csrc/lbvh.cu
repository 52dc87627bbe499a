// LBVH build and refit (§IV-B-3 acceleration-structure build; §IV-C per-body
// world matrices each frame), restated as a Karras (2012) linear BVH:
//   transform -> centroid bounds -> 63-bit Morton codes -> stable LSD radix
//   sort -> radix-tree topology -> bottom-up boxes -> collapse into the 4-wide
//   tree the traversal walks.
// The refit re-runs only the transform and the 4-wide tree's boxes, bottom
// up, with the topology of the last build.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "fire_internal.cuh"

namespace fire {
namespace {

// x' = fma(m0,x, fma(m1,y, fma(m2,z, m3))) per row of the 3x4 matrix.
__device__ __forceinline__ float3 xform(const float* __restrict__ m, float4 v) {
  return f3(fmaf(m[0], v.x, fmaf(m[1], v.y, fmaf(m[2], v.z, m[3]))),
            fmaf(m[4], v.x, fmaf(m[5], v.y, fmaf(m[6], v.z, m[7]))),
            fmaf(m[8], v.x, fmaf(m[9], v.y, fmaf(m[10], v.z, m[11]))));
}

__device__ __forceinline__ float3 fmin3(float3 a, float3 b) { return f3(fminf(a.x, b.x), fminf(a.y, b.y), fminf(a.z, b.z)); }
__device__ __forceinline__ float3 fmax3(float3 a, float3 b) { return f3(fmaxf(a.x, b.x), fmaxf(a.y, b.y), fmaxf(a.z, b.z)); }

// ----------------------------------------------------------------------------
// Validation of the inputs of fire_scene_create: count out-of-range indices
// and non-finite positions (the host turns a non-zero count into an error).
// ----------------------------------------------------------------------------
__global__ void k_validate(const float4* __restrict__ rest, int64_t nv, const uint32_t* __restrict__ idx,
                           const uint32_t* __restrict__ tmat, int64_t nt, const uint16_t* __restrict__ vb,
                           int nmat, int nbody, uint32_t* bad) {
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  uint32_t n = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nv || i < nt; i += stride) {
    if (i < nv) {
      float4 v = rest[i];
      n += !(isfinite(v.x) && isfinite(v.y) && isfinite(v.z));
      n += vb[i] >= (uint32_t)nbody;
    }
    if (i < nt) {
      n += idx[3 * i] >= (uint64_t)nv;
      n += idx[3 * i + 1] >= (uint64_t)nv;
      n += idx[3 * i + 2] >= (uint64_t)nv;
      n += tmat[i] >= (uint32_t)nmat;
    }
  }
  if (n) atomicAdd(bad, n);
}

// ----------------------------------------------------------------------------
// Build step 1: transform, triangle boxes, centroids, exact centroid bounds.
// centroid c = 0.5 * (min + max) per axis.
// ----------------------------------------------------------------------------
// Grid-stride over triangles; min/max are reduced per thread, per warp
// (shuffles) and per block (shared memory) before one set of atomics per
// block on the ordered-integer images (exact, order-independent).
__global__ void __launch_bounds__(256) k_centroids(const float4* __restrict__ rest, const uint32_t* __restrict__ idx,
                                                   const uint16_t* __restrict__ vb, const float* __restrict__ xf,
                                                   int64_t nt, float4* __restrict__ cen, uint32_t* __restrict__ bounds) {
  __shared__ uint32_t red[8][6];
  uint32_t lo[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, hi[3] = {0u, 0u, 0u};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nt; i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t a = idx[3 * i], b = idx[3 * i + 1], d = idx[3 * i + 2];
    float3 w0 = xform(xf + 12 * vb[a], rest[a]);
    float3 w1 = xform(xf + 12 * vb[b], rest[b]);
    float3 w2 = xform(xf + 12 * vb[d], rest[d]);
    float3 mn = fmin3(w0, fmin3(w1, w2)), mx = fmax3(w0, fmax3(w1, w2));
    float3 c = f3(0.5f * (mn.x + mx.x), 0.5f * (mn.y + mx.y), 0.5f * (mn.z + mx.z));
    cen[i] = make_float4(c.x, c.y, c.z, 0.0f);
    uint32_t o[3] = {f2ord(c.x), f2ord(c.y), f2ord(c.z)};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      lo[k] = min(lo[k], o[k]);
      hi[k] = max(hi[k], o[k]);
    }
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    for (int off = 16; off; off >>= 1) {
      lo[k] = min(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], off));
      hi[k] = max(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], off));
    }
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      red[w][k] = lo[k];
      red[w][3 + k] = hi[k];
    }
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    const int k = threadIdx.x;
    uint32_t v = red[0][k];
    for (int q = 1; q < (int)(blockDim.x >> 5); ++q) v = k < 3 ? min(v, red[q][k]) : max(v, red[q][k]);
    if (k < 3) atomicMin(bounds + k, v);
    else atomicMax(bounds + k, v);
  }
}

// Spread the low 21 bits of x to every third bit (bit k -> bit 3k).
__device__ __forceinline__ uint64_t spread3(uint32_t x) {
  uint64_t v = x & 0x1fffffull;
  v = (v | (v << 32)) & 0x1f00000000ffffull;
  v = (v | (v << 16)) & 0x1f0000ff0000ffull;
  v = (v | (v << 8)) & 0x100f00f00f00f00full;
  v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
  v = (v | (v << 2)) & 0x1249249249249249ull;
  return v;
}

// q = min(floor((c - lo) * s), 2^m - 1) with s = 2^m / (hi - lo) (0 if
// hi == lo): FP32 subtract, FP32 multiply, truncation.
__device__ __forceinline__ uint32_t quantise(float c, float lo, float s, uint32_t qmax) {
  float f = (c - lo) * s;
  if (!(f > 0.0f)) return 0u;
  if (f >= (float)qmax) return qmax;
  return (uint32_t)f;
}

// Build step 2: Morton code with m bits per axis (x -> bit 3k+2, y -> 3k+1,
// z -> 3k) and, with more than one rigid body, a body field of B bits
// (body = that of the triangle's first vertex) between its top 3c bits
// (coarse) and the rest (fine):
//   key = coarse << (B + 3(m-c)) | body << 3(m-c) | fine.
// Inside each coarse cell (1/2^c of the bounds per axis) a body's triangles
// are consecutive in the sorted order and form one subtree, so a refit under
// the bodies' rigid motions only widens the nodes of the coarse levels by
// the drift between bodies.  The host picks B = bits of (nbody - 1),
// m = min(21, (63 - B) / 3), c = 4 (two-level bottom levels: c = 0, one
// subtree per body); one body: B = 0, m = 21, the plain Morton code.
__global__ void k_morton(const float4* __restrict__ cen, int64_t nt, const uint32_t* __restrict__ bounds,
                         const uint32_t* __restrict__ idx, const uint16_t* __restrict__ vb, int prefix_bits,
                         int m, int coarse_bits, uint64_t* __restrict__ keys, uint32_t* __restrict__ vals,
                         uint64_t* __restrict__ keys_orig) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nt) return;
  const float cells = (float)(1u << m);
  const uint32_t qmax = (1u << m) - 1u;
  float lo[3], s[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    lo[k] = ord2f(bounds[k]);
    float hi = ord2f(bounds[3 + k]);
    s[k] = (hi > lo[k]) ? cells / (hi - lo[k]) : 0.0f;
  }
  float4 c = cen[i];
  uint64_t code = (spread3(quantise(c.x, lo[0], s[0], qmax)) << 2) |
                  (spread3(quantise(c.y, lo[1], s[1], qmax)) << 1) | spread3(quantise(c.z, lo[2], s[2], qmax));
  if (prefix_bits > 0) {
    const int fine = 3 * (m - coarse_bits);
    const uint64_t low = fine > 0 ? code & ((1ull << fine) - 1) : 0ull;
    code = ((code >> fine) << (prefix_bits + fine)) | ((uint64_t)vb[idx[3 * i]] << fine) | low;
  }
  keys[i] = code;
  keys_orig[i] = code;
  vals[i] = (uint32_t)i;
}

// ----------------------------------------------------------------------------
// Stable LSD radix sort of (63-bit key, u32 value): 7 passes of 9 bits.
//   upsweep   : per-tile digit histogram -> hist[digit * ntiles + tile]
//   scan      : per digit, exclusive scan over tiles; digit totals
//   downsweep : per tile, stable local ranks (warp match + per-warp counts),
//               scatter to digit_start + tile_prefix + warp_prefix + rank
// Tile = 256 threads x 16 items; item order inside a tile is warp-major,
// then round, then lane, which equals global order (stability).
// ----------------------------------------------------------------------------
__device__ __forceinline__ uint32_t digit_of(uint64_t k, int shift) { return (uint32_t)(k >> shift) & (kSortBins - 1); }

__global__ void __launch_bounds__(kSortThreads) k_sort_upsweep(const uint64_t* __restrict__ keys, int64_t n, int shift,
                                                               uint32_t* __restrict__ hist, int ntiles) {
  __shared__ uint32_t h[kSortBins];
  for (int d = threadIdx.x; d < kSortBins; d += kSortThreads) h[d] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * kSortTile;
#pragma unroll 4
  for (int r = 0; r < kSortItems; ++r) {
    int64_t i = base + (int64_t)r * kSortThreads + threadIdx.x;
    if (i < n) atomicAdd(&h[digit_of(keys[i], shift)], 1u);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < kSortBins; d += kSortThreads) hist[(int64_t)d * ntiles + blockIdx.x] = h[d];
}

// One block per digit: exclusive scan of hist[d][0..ntiles) in place; total -> totals[d].
__global__ void __launch_bounds__(1024) k_sort_scan(uint32_t* __restrict__ hist, int ntiles, uint32_t* __restrict__ totals) {
  __shared__ uint32_t wsum[32];
  __shared__ uint32_t carry;
  uint32_t* row = hist + (int64_t)blockIdx.x * ntiles;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int base = 0; base < ntiles; base += 1024) {
    int i = base + threadIdx.x;
    uint32_t v = i < ntiles ? row[i] : 0u;
    uint32_t x = v;
    for (int off = 1; off < 32; off <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, x, off);
      if (lane >= off) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
      uint32_t s = wsum[lane];
      for (int off = 1; off < 32; off <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, s, off);
        if (lane >= off) s += y;
      }
      wsum[lane] = s;  // inclusive warp sums
    }
    __syncthreads();
    uint32_t excl = carry + (w ? wsum[w - 1] : 0u) + x - v;
    if (i < ntiles) row[i] = excl;
    __syncthreads();
    if (threadIdx.x == 0) carry += wsum[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) totals[blockIdx.x] = carry;
}

__global__ void __launch_bounds__(kSortThreads) k_sort_downsweep(const uint64_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                                                                 uint64_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                                 int64_t n, int shift, const uint32_t* __restrict__ hist,
                                                                 int ntiles, const uint32_t* __restrict__ totals) {
  constexpr int W = kSortThreads / 32;
  __shared__ uint32_t wcnt[W][kSortBins];
  __shared__ uint32_t dbase[kSortBins];
  __shared__ uint32_t scan_tmp[kSortThreads];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int d = threadIdx.x; d < kSortBins; d += kSortThreads)
#pragma unroll
    for (int k = 0; k < W; ++k) wcnt[k][d] = 0;
  // digit start = exclusive scan of totals (each thread owns 2 consecutive digits)
  {
    uint32_t t0 = totals[2 * threadIdx.x], t1 = totals[2 * threadIdx.x + 1];
    uint32_t s = t0 + t1, x = s;
    for (int off = 1; off < 32; off <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, x, off);
      if (lane >= off) x += y;
    }
    if (lane == 31) scan_tmp[w] = x;
    __syncthreads();
    uint32_t wpre = 0;
    for (int k = 0; k < w; ++k) wpre += scan_tmp[k];
    uint32_t excl = wpre + x - s;
    dbase[2 * threadIdx.x] = excl + hist[(int64_t)(2 * threadIdx.x) * ntiles + blockIdx.x];
    dbase[2 * threadIdx.x + 1] = excl + t0 + hist[(int64_t)(2 * threadIdx.x + 1) * ntiles + blockIdx.x];
  }
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kSortTile + (int64_t)w * (kSortItems * 32);
  uint64_t key[kSortItems];
  uint32_t val[kSortItems], pre[kSortItems];
  const unsigned lt = (1u << lane) - 1u;
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    int64_t i = base + r * 32 + lane;
    bool ok = i < n;
    key[r] = ok ? kin[i] : 0;
    val[r] = ok ? vin[i] : 0;
    uint32_t d = ok ? digit_of(key[r], shift) : 0xffffffffu;
    unsigned peers = __match_any_sync(0xffffffffu, d);
    uint32_t before = ok ? wcnt[w][d] : 0u;
    __syncwarp();
    if (ok && (peers & lt) == 0) wcnt[w][d] = before + __popc(peers);
    __syncwarp();
    pre[r] = before + __popc(peers & lt);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < kSortBins; d += kSortThreads) {
    uint32_t run = 0;
#pragma unroll
    for (int k = 0; k < W; ++k) {
      uint32_t c = wcnt[k][d];
      wcnt[k][d] = run;
      run += c;
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    int64_t i = base + r * 32 + lane;
    if (i < n) {
      uint32_t d = digit_of(key[r], shift);
      uint32_t pos = dbase[d] + wcnt[w][d] + pre[r];
      if (pos < n) {  // always true for a consistent histogram; keeps stores in bounds regardless
        kout[pos] = key[r];
        vout[pos] = val[r];
      }
    }
  }
}

// ----------------------------------------------------------------------------
// Topology (Karras 2012): one thread per internal node i in [0, T-2].
// delta(i, j) = clz64(k_i ^ k_j), or 64 + clz32(i ^ j) for equal keys,
// -1 outside [0, T-1].
// ----------------------------------------------------------------------------
__device__ __forceinline__ int kdelta(const uint64_t* __restrict__ k, int64_t n, int64_t i, int64_t j) {
  if (j < 0 || j >= n) return -1;
  uint64_t a = k[i], b = k[j];
  if (a != b) return __clzll((long long)(a ^ b));
  return 64 + __clz((int)((uint32_t)i ^ (uint32_t)j));
}

__global__ void k_karras(const uint64_t* __restrict__ k, int64_t n, Node* __restrict__ nodes,
                         int32_t* __restrict__ leaf_slot, int32_t* __restrict__ node_slot) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n - 1) return;
  int d = (kdelta(k, n, i, i + 1) - kdelta(k, n, i, i - 1)) >= 0 ? 1 : -1;
  int dmin = kdelta(k, n, i, i - d);
  int64_t lmax = 2;
  while (kdelta(k, n, i, i + lmax * d) > dmin) lmax <<= 1;
  int64_t l = 0;
  for (int64_t t = lmax >> 1; t >= 1; t >>= 1)
    if (kdelta(k, n, i, i + (l + t) * d) > dmin) l += t;
  int64_t j = i + l * d;
  int dnode = kdelta(k, n, i, j);
  int64_t s = 0, t = l;
  do {
    t = (t + 1) >> 1;
    if (kdelta(k, n, i, i + (s + t) * d) > dnode) s += t;
  } while (t > 1);
  int64_t gamma = i + s * d + (d < 0 ? -1 : 0);
  int64_t lo = i < j ? i : j, hi = i < j ? j : i;
  if (gamma < lo || gamma >= hi) return;  // impossible for sorted keys; slots stay -1
  int32_t c0, c1;
  if (lo == gamma) { c0 = ~(int32_t)gamma; leaf_slot[gamma] = (int32_t)(2 * i); }
  else { c0 = (int32_t)gamma; node_slot[gamma] = (int32_t)(2 * i); }
  if (hi == gamma + 1) { c1 = ~(int32_t)(gamma + 1); leaf_slot[gamma + 1] = (int32_t)(2 * i + 1); }
  else { c1 = (int32_t)(gamma + 1); node_slot[gamma + 1] = (int32_t)(2 * i + 1); }
  nodes[i].b.z = __int_as_float(c0);
  nodes[i].d.z = __int_as_float(c1);
  if (i == 0) node_slot[0] = -1;
}

// Permute the index buffer and materials into leaf (sorted) order.
__global__ void k_gather_sorted(const uint32_t* __restrict__ order, const uint32_t* __restrict__ idx,
                                const uint32_t* __restrict__ tmat, int64_t nt, uint4* __restrict__ sidx,
                                uint32_t* __restrict__ smat, int32_t* __restrict__ rank) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nt) return;
  uint32_t o = order[i];
  sidx[i] = make_uint4(idx[3 * (int64_t)o], idx[3 * (int64_t)o + 1], idx[3 * (int64_t)o + 2], o);
  smat[i] = tmat[o];
  rank[o] = (int32_t)i;
}

// Write one child sector of a node: box, link and subtree height (a whole
// 32-B sector, two 16-B stores).
__device__ __forceinline__ void store_child(Node* node, int side, float3 lo, float3 hi, int link, int height) {
  float4* s = side == 0 ? &node->a : &node->c;
  s[0] = make_float4(lo.x, lo.y, lo.z, hi.x);
  s[1] = make_float4(hi.y, hi.z, __int_as_float(link), __int_as_float(height));
}

// Box (union of both children) and height of a node, read through L2.
__device__ __forceinline__ void load_node_box(const Node* nd, float3& lo, float3& hi, int& height) {
  float4 a = __ldcg(&nd->a), b = __ldcg(&nd->b), c = __ldcg(&nd->c), d = __ldcg(&nd->d);
  lo = f3(fminf(a.x, c.x), fminf(a.y, c.y), fminf(a.z, c.z));
  hi = f3(fmaxf(a.w, c.w), fmaxf(b.x, d.x), fmaxf(b.y, d.y));
  height = 1 + max(__float_as_int(b.w), __float_as_int(d.w));
}

// ----------------------------------------------------------------------------
// Build refit: one thread per leaf (sorted position).  Transform the
// triangle, write its 48-B record, store its box in the parent's slot; then
// climb: the second thread to arrive at a node (odd counter value) unions
// the node's two child boxes into the grandparent's slot and records the
// node's height there.  Min/max are exact, so the boxes do not depend on the
// arrival order.  (Per frame, the level-synchronous refit below is used.)
// ----------------------------------------------------------------------------
__global__ void k_refit_build(const float4* __restrict__ rest, const uint16_t* __restrict__ vb,
                              const float* __restrict__ xf, const uint4* __restrict__ sidx,
                              const uint32_t* __restrict__ smat, int64_t nt, float4* __restrict__ tris,
                              Node* nodes, const int32_t* __restrict__ leaf_slot,
                              const int32_t* __restrict__ node_slot, uint32_t* counters,
                              float* __restrict__ xfb, int nxf, int body_in_w) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < nxf) xfb[i] = xf[i];  // the frame buffer's copy of the body matrices
  const int lane = threadIdx.x & 31;
  const bool valid = i < nt;
  float3 lo = f3(0, 0, 0), hi = f3(0, 0, 0);
  int32_t slot = -1;
  if (valid) {
    uint4 id = sidx[i];
    float3 w0 = xform(xf + 12 * vb[id.x], rest[id.x]);
    float3 w1 = xform(xf + 12 * vb[id.y], rest[id.y]);
    float3 w2 = xform(xf + 12 * vb[id.z], rest[id.z]);
    float3 e1 = sub3(w1, w0), e2 = sub3(w2, w0);
    tris[3 * i] = make_float4(w0.x, w0.y, w0.z, __uint_as_float(id.w));
    tris[3 * i + 1] = make_float4(e1.x, e1.y, e1.z, __uint_as_float(smat[i]));
    tris[3 * i + 2] = make_float4(e2.x, e2.y, e2.z, body_in_w ? __uint_as_float((uint32_t)vb[id.x]) : 0.0f);
    lo = fmin3(w0, fmin3(w1, w2));
    hi = fmax3(w0, fmax3(w1, w2));
    slot = nt > 1 ? leaf_slot[i] : 0;
  }
  if (nt == 1) {  // single leaf: node 0 holds it on both sides
    if (valid) {
      store_child(nodes, 0, lo, hi, ~0, 0);
      store_child(nodes, 1, lo, hi, ~0, 0);
    }
    return;
  }
  // Two sibling leaves in neighbouring lanes (leaf i on side 0, leaf i+1 on
  // side 1 of the same node) finish their node inside the warp: the side-0
  // lane stores both boxes and climbs on; that node's counter is never used
  // (the same pairs occur in every refit of the topology).
  const int32_t s_next = __shfl_down_sync(0xffffffffu, slot, 1);
  const int32_t s_prev = __shfl_up_sync(0xffffffffu, slot, 1);
  const float3 nlo = f3(__shfl_down_sync(0xffffffffu, lo.x, 1), __shfl_down_sync(0xffffffffu, lo.y, 1),
                        __shfl_down_sync(0xffffffffu, lo.z, 1));
  const float3 nhi = f3(__shfl_down_sync(0xffffffffu, hi.x, 1), __shfl_down_sync(0xffffffffu, hi.y, 1),
                        __shfl_down_sync(0xffffffffu, hi.z, 1));
  if (!valid) return;
  const bool pair_lo = slot >= 0 && (slot & 1) == 0 && lane < 31 && i + 1 < nt && s_next == slot + 1;
  const bool pair_hi = slot >= 0 && (slot & 1) == 1 && lane > 0 && s_prev == slot - 1;
  if (pair_hi) return;
  int h = 0;
  int link = (int)~i;
  if (pair_lo) {
    if ((slot >> 1) >= nt - 1) return;  // never for a complete topology
    Node* node = nodes + (slot >> 1);
    store_child(node, 0, lo, hi, (int)~i, 0);
    store_child(node, 1, nlo, nhi, (int)~(i + 1), 0);
    lo = fmin3(lo, nlo);
    hi = fmax3(hi, nhi);
    h = 1;
    link = slot >> 1;
    slot = node_slot[slot >> 1];
    if (slot < 0) return;  // the pair was the root
  }
  while (true) {
    if (slot < 0 || (slot >> 1) >= nt - 1) return;  // never for a complete topology
    int32_t p = slot >> 1;
    Node* node = nodes + p;
    store_child(node, slot & 1, lo, hi, link, h);
    // release the box to the sibling's thread / acquire the sibling's box
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    uint32_t old = atomicAdd(counters + p, 1u);
    if ((old & 1u) == 0) return;  // first arrival: the sibling finishes this node
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    load_node_box(node, lo, hi, h);
    link = p;
    slot = node_slot[p];
    if (slot < 0) return;  // root done
  }
}

// ----------------------------------------------------------------------------
// 4-wide traversal tree, collapsed from the binary tree at build (one launch
// per level): a 4-wide node starts from a binary node's two children and
// opens the internal member with the largest box surface area until it has
// four members or only leaves.  Each member keeps the binary slot that holds
// its box, so a frame's boxes are copied from the binary refit (k_fill4).
// ----------------------------------------------------------------------------
__device__ __forceinline__ float box_area(float4 a, float4 b) {  // sector: lo xyz hi.x | hi.y hi.z
  float dx = a.w - a.x, dy = b.x - a.y, dz = b.y - a.z;
  return dx * dy + dy * dz + dz * dx;
}

__device__ __forceinline__ void collapse_one(const Node* __restrict__ nodes, const int32_t* __restrict__ in_pairs,
                                             uint32_t i, int32_t* __restrict__ out_pairs, uint32_t* nout,
                                             uint32_t* alloc, Node4* __restrict__ nodes4, int64_t cap4) {
  const int b = in_pairs[2 * i], q = in_pairs[2 * i + 1];
  int link[4] = {kEmptyLink, kEmptyLink, kEmptyLink, kEmptyLink}, src[4] = {-1, -1, -1, -1};
  float area[4] = {0, 0, 0, 0};
  for (int side = 0; side < 2; ++side) {
    const float4* s = side == 0 ? &nodes[b].a : &nodes[b].c;
    float4 a = s[0], bb = s[1];
    link[side] = __float_as_int(bb.z);
    src[side] = 2 * b + side;
    area[side] = box_area(a, bb);
  }
  int m = 2;
  while (m < 4) {
    int j = -1;
    float best = -1.0f;
    for (int k = 0; k < m; ++k)
      if (link[k] >= 0 && area[k] > best) { best = area[k]; j = k; }
    if (j < 0) break;
    const int f = link[j];
    float4 a0 = nodes[f].a, b0 = nodes[f].b, a1 = nodes[f].c, b1 = nodes[f].d;
    link[j] = __float_as_int(b0.z);
    src[j] = 2 * f;
    area[j] = box_area(a0, b0);
    link[m] = __float_as_int(b1.z);
    src[m] = 2 * f + 1;
    area[m] = box_area(a1, b1);
    ++m;
  }
  int out[4];
  for (int k = 0; k < 4; ++k) {
    out[k] = link[k];
    if (k < m && link[k] >= 0) {
      const uint32_t q2 = atomicAdd(alloc, 1u);  // 4-wide node index
      if (q2 >= cap4) {                          // never: a 4-wide node consumes >= 1 binary node
        out[k] = kEmptyLink;
        continue;
      }
      const uint32_t p = atomicAdd(nout, 1u);    // next level's queue slot
      out[k] = (int)q2;
      out_pairs[2 * p] = link[k];
      out_pairs[2 * p + 1] = (int)q2;
    }
  }
  nodes4[q].link = make_int4(out[0], out[1], out[2], out[3]);
  nodes4[q].src = make_int4(src[0], src[1], src[2], src[3]);
}

// One depth of the collapse: the queue of this depth holds *nin_p (binary
// node, 4-wide node) pairs (written by the previous depth's launch); each
// pair is collapsed by collapse_one, which allocates the internal members
// at the next depth (alloc) and queues them (*nout).  Grid-stride, so the
// host launches one fixed grid per depth without reading the length back.
__global__ void k_collapse(const Node* __restrict__ nodes, const int32_t* __restrict__ in_pairs,
                           const uint32_t* __restrict__ nin_p, int32_t* __restrict__ out_pairs, uint32_t* nout,
                           uint32_t* alloc, Node4* __restrict__ nodes4, int64_t cap4) {
  const uint32_t nin = *nin_p;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nin; i += gridDim.x * blockDim.x)
    collapse_one(nodes, in_pairs, i, out_pairs, nout, alloc, nodes4, cap4);
}

// At build: copy each member's box from its binary slot (whole 32-B sector
// reads, 112-B node writes).
__global__ void __launch_bounds__(256) k_fill4(const Node* __restrict__ nodes, Node4* __restrict__ nodes4, int64_t n4) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= n4) return;
  const int4 src = nodes4[q].src;
  const int sv[4] = {src.x, src.y, src.z, src.w};
  float lx[4], ly[4], lz[4], hx[4], hy[4], hz[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    // unused slot: the inverted infinite box, which no ray enters
    const float inf = __int_as_float(0x7f800000);
    float4 a = make_float4(inf, inf, inf, -inf), b = make_float4(-inf, -inf, 0, 0);
    if (sv[c] >= 0) {
      const float4* s = (sv[c] & 1) ? &nodes[sv[c] >> 1].c : &nodes[sv[c] >> 1].a;
      a = __ldcg(s);
      b = __ldcg(s + 1);
    }
    lx[c] = a.x; ly[c] = a.y; lz[c] = a.z; hx[c] = a.w; hy[c] = b.x; hz[c] = b.y;
  }
  Node4* n = nodes4 + q;
  n->lox = make_float4(lx[0], lx[1], lx[2], lx[3]);
  n->loy = make_float4(ly[0], ly[1], ly[2], ly[3]);
  n->loz = make_float4(lz[0], lz[1], lz[2], lz[3]);
  n->hix = make_float4(hx[0], hx[1], hx[2], hx[3]);
  n->hiy = make_float4(hy[0], hy[1], hy[2], hy[3]);
  n->hiz = make_float4(hz[0], hz[1], hz[2], hz[3]);
}

// ----------------------------------------------------------------------------
// Two-level mode (§IV-B-3: a bottom level per mesh, a top level over the
// instances rebuilt every frame).  The LBVH above is built over the rest
// pose with body-prefixed keys, so each body's triangles are one sorted
// range and one subtree; the 4-wide collapse starts from every body's
// subtree root, which gives each body its own 4-wide bottom level.
// ----------------------------------------------------------------------------
// Sorted range [first, last] of every body (the key prefix above bit 3m).
__global__ void k_body_ranges(const uint64_t* __restrict__ keys, int64_t nt, int shift, int nbody,
                              int32_t* __restrict__ range, uint32_t* err) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nt) return;
  const uint64_t b = keys[i] >> shift;
  if (b >= (uint64_t)nbody) {  // never: the key prefix is a body id
    atomicOr(err, kErrCorrupt);
    return;
  }
  if (i == 0 || (keys[i - 1] >> shift) != b) range[2 * b] = (int32_t)i;
  if (i == nt - 1 || (keys[i + 1] >> shift) != b) range[2 * b + 1] = (int32_t)i;
}

// One block (nbody <= kMaxTlasBodies threads).  Body b with triangles gets
// the 4-wide node rank(b) (its rank among the bodies with triangles) as its
// bottom-level root.  Its subtree root in the Karras tree covers exactly
// [f, l]; a node is numbered by the end of its range that its parent's split
// falls on, so it is node l when the parent extends to the right
// (delta(l, l+1) > delta(f-1, f)) and node f otherwise, the tree's root if
// [f, l] is everything.  A body of one triangle becomes a 4-wide node with
// that leaf as its only member (its box copied from the leaf's slot);
// the others are queued for the collapse.
__global__ void __launch_bounds__(1024) k_body_roots(const uint64_t* __restrict__ keys, int64_t nt,
                                                     const int32_t* __restrict__ range, int nbody,
                                                     const int32_t* __restrict__ leaf_slot,
                                                     int32_t* __restrict__ blas_root, int32_t* __restrict__ pairs,
                                                     uint32_t* __restrict__ qlen, Node4* __restrict__ nodes4) {
  __shared__ int32_t scan_a[1024], scan_m[1024];
  const int b = threadIdx.x;
  int32_t f = -1, l = -1;
  if (b < nbody) {
    f = range[2 * b];
    l = range[2 * b + 1];
  }
  const bool has = f >= 0 && l >= f;
  const bool multi = has && l > f;
  scan_a[b] = has ? 1 : 0;
  scan_m[b] = multi ? 1 : 0;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {  // inclusive scans
    const int32_t a = b >= off ? scan_a[b - off] : 0, m = b >= off ? scan_m[b - off] : 0;
    __syncthreads();
    scan_a[b] += a;
    scan_m[b] += m;
    __syncthreads();
  }
  if (b == 0) {
    qlen[0] = (uint32_t)scan_m[1023];              // depth-0 collapse queue: the multi-triangle bodies
    qlen[kMaxDepth4] = (uint32_t)scan_a[1023];     // 4-wide nodes allocated so far: every root
    qlen[kMaxDepth4 + 1] = (uint32_t)scan_a[1023]; // number of bottom-level roots
  }
  if (b >= nbody) return;
  if (!has) {
    blas_root[b] = -1;
    return;
  }
  const int32_t q = scan_a[b] - 1;
  blas_root[b] = q;
  if (!multi) {  // one triangle at sorted position f
    const int32_t slot = nt > 1 ? leaf_slot[f] : 0;
    const float inf = __int_as_float(0x7f800000);
    Node4* n = nodes4 + q;
    n->lox = make_float4(inf, inf, inf, inf);
    n->loy = n->lox;
    n->loz = n->lox;
    n->hix = make_float4(-inf, -inf, -inf, -inf);
    n->hiy = n->hix;
    n->hiz = n->hix;
    n->link = make_int4(~f, kEmptyLink, kEmptyLink, kEmptyLink);
    n->src = make_int4(slot, -1, -1, -1);
    return;
  }
  int32_t root;
  if (f == 0 && l == nt - 1) {
    root = 0;
  } else {
    // (both positions checked: f - 1 is -1 for the first body)
    auto delta = [&](int64_t i, int64_t j) -> int {
      if (i < 0 || i >= nt || j < 0 || j >= nt) return -1;
      const uint64_t x = keys[i], y = keys[j];
      if (x != y) return __clzll((long long)(x ^ y));
      return 64 + __clz((int)((uint32_t)i ^ (uint32_t)j));
    };
    root = delta(l, l + 1) > delta(f - 1, f) ? l : f;
  }
  const int32_t k = scan_m[b] - 1;
  pairs[2 * k] = root;
  pairs[2 * k + 1] = q;
}

// Rest box of every body: the union of its bottom-level root's members.
__global__ void k_body_boxes(const Node4* __restrict__ nodes4, int64_t n4, const int32_t* __restrict__ blas_root,
                             int nbody, float4* __restrict__ body_box) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbody) return;
  const int32_t q = blas_root[b];
  const float inf = __int_as_float(0x7f800000);
  float3 lo = f3(inf, inf, inf), hi = f3(-inf, -inf, -inf);
  if (q >= 0 && q < n4) {
    const Node4& n = nodes4[q];
    const int l[4] = {n.link.x, n.link.y, n.link.z, n.link.w};
    const float LX[4] = {n.lox.x, n.lox.y, n.lox.z, n.lox.w}, LY[4] = {n.loy.x, n.loy.y, n.loy.z, n.loy.w};
    const float LZ[4] = {n.loz.x, n.loz.y, n.loz.z, n.loz.w}, HX[4] = {n.hix.x, n.hix.y, n.hix.z, n.hix.w};
    const float HY[4] = {n.hiy.x, n.hiy.y, n.hiy.z, n.hiy.w}, HZ[4] = {n.hiz.x, n.hiz.y, n.hiz.z, n.hiz.w};
    for (int k = 0; k < 4; ++k) {
      if (l[k] == kEmptyLink) continue;
      lo = f3(fminf(lo.x, LX[k]), fminf(lo.y, LY[k]), fminf(lo.z, LZ[k]));
      hi = f3(fmaxf(hi.x, HX[k]), fmaxf(hi.y, HY[k]), fmaxf(hi.z, HZ[k]));
    }
  }
  body_box[2 * b] = make_float4(lo.x, lo.y, lo.z, 0.0f);
  body_box[2 * b + 1] = make_float4(hi.x, hi.y, hi.z, 0.0f);
}

// Top-level entries (each two-level build): a body whose parts lie far
// apart has a rest box that covers mostly empty space, so the top level is
// built over subtrees of the bodies' bottom levels instead.  Thread b cuts
// body b's bottom level breadth first from its root: on each level, in
// order, a node whose members are all inner 4-wide nodes is replaced by its
// members while the body's entries stay within its share (kMaxTlasBodies /
// bodies with triangles, at most kEntriesPerBody); every triangle of the
// body lies under exactly one entry.  Entries are written in body order (at
// the scan of the counts) as (node, body) with their rest boxes (the node's
// slot in its parent, or the body's rest box for a root); the slots past the
// last hold (-1, -1).  One block of kMaxTlasBodies threads.
// (shares capped at 2, 4, 8 entries per body measured slower on the
// 7.3M-triangle scene, 65 bodies: the full share of 15 is used there)
constexpr int kEntriesPerBody = 64;
__global__ void __launch_bounds__(1024) k_top_entries(const Node4* __restrict__ nodes4, int64_t n4,
                                                      const int32_t* __restrict__ blas_root,
                                                      const float4* __restrict__ body_box, int nbody,
                                                      int32_t* __restrict__ inst, float4* __restrict__ inst_box,
                                                      uint32_t* err) {
  __shared__ int32_t scan[kMaxTlasBodies];
  const int b = threadIdx.x;
  const int32_t root = b < nbody ? blas_root[b] : -1;
  const bool has = root >= 0 && root < n4;
  if (b < nbody && root >= n4) atomicOr(err, kErrCorrupt);
  auto block_scan = [&](int32_t v) {  // inclusive, over the block
    scan[b] = v;
    __syncthreads();
    for (int off = 1; off < kMaxTlasBodies; off <<= 1) {
      const int32_t a = b >= off ? scan[b - off] : 0;
      __syncthreads();
      scan[b] += a;
      __syncthreads();
    }
    const int32_t r = scan[b], total = scan[kMaxTlasBodies - 1];
    __syncthreads();
    return make_int2(r, total);
  };
  const int nbodies = block_scan(has ? 1 : 0).y;
  const int share = nbodies > 0 ? max(1, min(kEntriesPerBody, kMaxTlasBodies / nbodies)) : 1;
  // entries of the current level: node, and where its rest box is (parent
  // node * 4 + slot; -1: the body's root)
  int32_t ent[kEntriesPerBody], from[kEntriesPerBody], nxt[kEntriesPerBody], nfrom[kEntriesPerBody];
  int n = 0;
  if (has) {
    ent[0] = root;
    from[0] = -1;
    n = 1;
  }
  for (int level = 0; level < 64 && n > 0; ++level) {
    // invariant: m + (n - k) <= share before entry k, so m never passes share
    int m = 0;
    bool split = false;
    for (int k = 0; k < n; ++k) {
      const int32_t v = ent[k];
      const int4 lk = nodes4[v].link;
      const int l[4] = {lk.x, lk.y, lk.z, lk.w};
      int kids = 0;
      bool inner = true;
      for (int c = 0; c < 4; ++c) {
        if (l[c] == kEmptyLink) continue;
        if (l[c] < 0 || l[c] >= n4) inner = false;  // a triangle (a link past the nodes: corrupt)
        else ++kids;
        if (l[c] >= n4) atomicOr(err, kErrCorrupt);
      }
      if (inner && kids > 0 && m + kids + (n - k - 1) <= share) {
        for (int c = 0; c < 4; ++c) {
          if (l[c] == kEmptyLink) continue;
          nxt[m] = l[c];
          nfrom[m] = 4 * v + c;
          ++m;
        }
        split = true;
      } else {
        nxt[m] = v;
        nfrom[m] = from[k];
        ++m;
      }
    }
    for (int k = 0; k < m; ++k) {
      ent[k] = nxt[k];
      from[k] = nfrom[k];
    }
    n = m;
    if (!split) break;
  }
  const int2 sc = block_scan(n);
  const int base = sc.x - n;
  for (int k = 0; k < n; ++k) {
    const int i = base + k;  // < kMaxTlasBodies: the shares add up to at most that
    if (i >= kMaxTlasBodies) {
      atomicOr(err, kErrCorrupt);
      break;
    }
    float4 lo, hi;
    if (from[k] < 0) {
      lo = body_box[2 * b];
      hi = body_box[2 * b + 1];
    } else {
      const float* f = &nodes4[from[k] >> 2].lox.x;  // lox loy loz hix hiy hiz, 4 slots each
      const int c = from[k] & 3;
      lo = make_float4(f[c], f[4 + c], f[8 + c], 0.0f);
      hi = make_float4(f[12 + c], f[16 + c], f[20 + c], 0.0f);
    }
    inst[2 * i] = ent[k];
    inst[2 * i + 1] = b;
    inst_box[2 * i] = lo;
    inst_box[2 * i + 1] = hi;
  }
  for (int i = sc.y + b; i < kMaxTlasBodies; i += blockDim.x) {
    inst[2 * i] = -1;
    inst[2 * i + 1] = -1;
  }
}

// ----------------------------------------------------------------------------
// Top level of one frame (one block of 1024 threads, one per top-level
// entry).
//   1. world box of every body with triangles and of every entry: the 8
//      corners of its rest box through its (body's) matrix,
//      x' = fma(m0,x, fma(m1,y, fma(m2,z, m3))) per row; the union of the
//      bodies' boxes gives the frame's shadow-ray lift eps = 1e-4 |hi - lo|;
//      span = largest |coordinate| of that union and of the bodies' rest boxes
//   2. the entries' boxes widened by 2^-10 (1 + span) on every side (the
//      body-frame ray's rounding against the world box test), keyed by the
//      30-bit Morton code of their centres (10 bits per axis) above the entry
//      index,
//      sorted (bitonic), Karras topology, node boxes by range union
//   3. collapse into 4-wide nodes (thread 0, breadth first, opening the
//      member of largest surface area), leaf links ~entry
// Also copies the matrices into the frame buffer (xfb).
// ----------------------------------------------------------------------------
struct TlasSmem {
  float lo[3][kMaxTlasBodies], hi[3][kMaxTlasBodies];    // widened instance boxes
  float nlo[3][kMaxTlasBodies], nhi[3][kMaxTlasBodies];  // binary node boxes
  unsigned long long key[kMaxTlasBodies];
  int32_t body[kMaxTlasBodies];
  int32_t child[2][kMaxTlasBodies];
  int32_t rng[2][kMaxTlasBodies];
  int32_t queue[3][kMaxTlasBodies];  // collapse queue: binary node, 4-wide node, depth
  int32_t scan[kMaxTlasBodies];
  uint32_t red[8];
};

__device__ __forceinline__ uint32_t spread10(uint32_t x) {
  x &= 0x3ffu;
  x = (x | (x << 16)) & 0x030000ffu;
  x = (x | (x << 8)) & 0x0300f00fu;
  x = (x | (x << 4)) & 0x030c30c3u;
  x = (x | (x << 2)) & 0x09249249u;
  return x;
}

__global__ void __launch_bounds__(1024) k_tlas(const float* __restrict__ xf, int nbody,
                                               const int32_t* __restrict__ blas_root,
                                               const float4* __restrict__ body_box,
                                               const int32_t* __restrict__ inst,
                                               const float4* __restrict__ inst_box, Node4* __restrict__ tlas,
                                               TlasInfo* __restrict__ info, float* __restrict__ xfb,
                                               uint32_t* err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TlasSmem& S = *reinterpret_cast<TlasSmem*>(smem_raw);
  const int tid = threadIdx.x;
  for (int i = tid; i < 12 * nbody; i += blockDim.x) xfb[i] = xf[i];
  if (tid < 8) S.red[tid] = tid < 3 ? 0xffffffffu : 0u;  // [0..2] min lo, [3..5] max hi, [6] span, [7] unused
  // world box of a rest box: its 8 corners through the matrix m
  auto world_box = [](const float* m, float4 rl, float4 rh, float3& lo, float3& hi) {
    for (int c = 0; c < 8; ++c) {
      const float x = (c & 1) ? rh.x : rl.x, y = (c & 2) ? rh.y : rl.y, z = (c & 4) ? rh.z : rl.z;
      const float3 p = f3(fmaf(m[0], x, fmaf(m[1], y, fmaf(m[2], z, m[3]))),
                          fmaf(m[4], x, fmaf(m[5], y, fmaf(m[6], z, m[7]))),
                          fmaf(m[8], x, fmaf(m[9], y, fmaf(m[10], z, m[11]))));
      lo = c ? f3(fminf(lo.x, p.x), fminf(lo.y, p.y), fminf(lo.z, p.z)) : p;
      hi = c ? f3(fmaxf(hi.x, p.x), fmaxf(hi.y, p.y), fmaxf(hi.z, p.z)) : p;
    }
  };
  // the frame's union, lift and span come from the bodies' boxes (the
  // instances of the method); the top level's leaves are the entries
  const bool bhas = tid < nbody && blas_root[tid] >= 0;
  float3 blo = f3(0, 0, 0), bhi = f3(0, 0, 0);
  float rspan = 0.0f;
  if (bhas) {
    const float4 rl = body_box[2 * tid], rh = body_box[2 * tid + 1];
    rspan = fmaxf(fmaxf(fmaxf(fabsf(rl.x), fabsf(rh.x)), fmaxf(fabsf(rl.y), fabsf(rh.y))),
                  fmaxf(fabsf(rl.z), fabsf(rh.z)));
    world_box(xf + 12 * tid, rl, rh, blo, bhi);
  }
  const int32_t eb = tid < kMaxTlasBodies ? inst[2 * tid + 1] : -1;  // the entry's body
  const bool has = tid < kMaxTlasBodies && inst[2 * tid] >= 0 && eb >= 0 && eb < nbody;
  float3 wlo = f3(0, 0, 0), whi = f3(0, 0, 0);
  if (has) world_box(xf + 12 * eb, inst_box[2 * tid], inst_box[2 * tid + 1], wlo, whi);
  // compaction: rank among the entries in use (the entries come first)
  S.scan[tid] = has ? 1 : 0;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    const int32_t a = tid >= off ? S.scan[tid - off] : 0;
    __syncthreads();
    S.scan[tid] += a;
    __syncthreads();
  }
  const int ninst = S.scan[1023];
  if (bhas) {
    atomicMin(&S.red[0], f2ord(blo.x));
    atomicMin(&S.red[1], f2ord(blo.y));
    atomicMin(&S.red[2], f2ord(blo.z));
    atomicMax(&S.red[3], f2ord(bhi.x));
    atomicMax(&S.red[4], f2ord(bhi.y));
    atomicMax(&S.red[5], f2ord(bhi.z));
    atomicMax(&S.red[6], __float_as_uint(rspan));  // non-negative: bits order as values
  }
  __syncthreads();
  const float3 ulo = f3(ord2f(S.red[0]), ord2f(S.red[1]), ord2f(S.red[2]));
  const float3 uhi = f3(ord2f(S.red[3]), ord2f(S.red[4]), ord2f(S.red[5]));
  const float span = fmaxf(__uint_as_float(S.red[6]),
                           fmaxf(fmaxf(fmaxf(fabsf(ulo.x), fabsf(uhi.x)), fmaxf(fabsf(ulo.y), fabsf(uhi.y))),
                                 fmaxf(fabsf(ulo.z), fabsf(uhi.z))));
  if (tid == 0) {
    TlasInfo ti;
    const float3 ext = sub3(uhi, ulo);
    ti.eps = ninst > 0 ? 1e-4f * sqrtf(dot3(ext, ext)) : 0.0f;
    ti.span = ninst > 0 ? span : 0.0f;
    ti.n = 0;
    ti.err = 0;
    *info = ti;
  }
  if (ninst == 0) return;
  const float margin = (1.0f + span) * (1.0f / 1024.0f);
  const int i = S.scan[tid] - 1;
  if (has) {
    S.lo[0][i] = wlo.x - margin;
    S.lo[1][i] = wlo.y - margin;
    S.lo[2][i] = wlo.z - margin;
    S.hi[0][i] = whi.x + margin;
    S.hi[1][i] = whi.y + margin;
    S.hi[2][i] = whi.z + margin;
    S.body[i] = tid;
  }
  __syncthreads();
  // keys: Morton code of the widened box centre over the union box
  int n2 = 1;
  while (n2 < ninst) n2 <<= 1;
  if (tid < n2) {
    unsigned long long k = ~0ull;
    if (tid < ninst) {
      uint32_t q[3];
      const float L[3] = {ulo.x, ulo.y, ulo.z}, H[3] = {uhi.x, uhi.y, uhi.z};
      for (int a = 0; a < 3; ++a) {
        const float c = 0.5f * (S.lo[a][tid] + S.hi[a][tid]);
        const float ext = H[a] - L[a];
        const float f = ext > 0.0f ? (c - L[a]) * (1024.0f / ext) : 0.0f;
        q[a] = f > 0.0f ? (f >= 1023.0f ? 1023u : (uint32_t)f) : 0u;
      }
      const uint32_t code = (spread10(q[0]) << 2) | (spread10(q[1]) << 1) | spread10(q[2]);
      k = ((unsigned long long)code << 10) | (unsigned long long)tid;
    }
    S.key[tid] = k;
  }
  __syncthreads();
  for (int kk = 2; kk <= n2; kk <<= 1) {  // bitonic sort, ascending
    for (int j = kk >> 1; j > 0; j >>= 1) {
      if (tid < n2) {
        const int x = tid ^ j;
        if (x > tid) {
          const unsigned long long a = S.key[tid], b = S.key[x];
          const bool up = (tid & kk) == 0;
          if ((a > b) == up) {
            S.key[tid] = b;
            S.key[x] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  // Karras topology over the sorted keys (unique: the index is in the low bits)
  const int n = ninst;
  auto kdel = [&](int a, int b) -> int {
    if (b < 0 || b >= n) return -1;
    return __clzll((long long)(S.key[a] ^ S.key[b]));
  };
  if (tid < n - 1) {
    const int d = (kdel(tid, tid + 1) - kdel(tid, tid - 1)) >= 0 ? 1 : -1;
    const int dmin = kdel(tid, tid - d);
    int lmax = 2;
    while (kdel(tid, tid + lmax * d) > dmin) lmax <<= 1;
    int l = 0;
    for (int t = lmax >> 1; t >= 1; t >>= 1)
      if (kdel(tid, tid + (l + t) * d) > dmin) l += t;
    const int j = tid + l * d;
    const int dnode = kdel(tid, j);
    int sp = 0, t = l;
    do {
      t = (t + 1) >> 1;
      if (kdel(tid, tid + (sp + t) * d) > dnode) sp += t;
    } while (t > 1);
    const int gamma = tid + sp * d + (d < 0 ? -1 : 0);
    const int lo = min(tid, j), hi = max(tid, j);
    // child codes: internal node index, or n - 1 + sorted position for a leaf
    S.child[0][tid] = lo == gamma ? n - 1 + gamma : gamma;
    S.child[1][tid] = hi == gamma + 1 ? n - 1 + gamma + 1 : gamma + 1;
    S.rng[0][tid] = lo;
    S.rng[1][tid] = hi;
  }
  __syncthreads();
  if (tid < n - 1) {  // node box = union of the instances of its range
    float bl[3] = {__int_as_float(0x7f800000), __int_as_float(0x7f800000), __int_as_float(0x7f800000)};
    float bh[3] = {-bl[0], -bl[0], -bl[0]};
    for (int p = S.rng[0][tid]; p <= S.rng[1][tid]; ++p) {
      const int ii = (int)(S.key[p] & 1023ull);
      for (int a = 0; a < 3; ++a) {
        bl[a] = fminf(bl[a], S.lo[a][ii]);
        bh[a] = fmaxf(bh[a], S.hi[a][ii]);
      }
    }
    for (int a = 0; a < 3; ++a) {
      S.nlo[a][tid] = bl[a];
      S.nhi[a][tid] = bh[a];
    }
  }
  __syncthreads();
  if (tid != 0) return;
  // collapse (serial, breadth first): member code c < n-1 is a binary node,
  // c >= n-1 the instance at sorted position c - (n-1)
  auto box_of = [&](int c, float* bl, float* bh) {
    if (c < n - 1) {
      for (int a = 0; a < 3; ++a) { bl[a] = S.nlo[a][c]; bh[a] = S.nhi[a][c]; }
    } else {
      const int ii = (int)(S.key[c - (n - 1)] & 1023ull);
      for (int a = 0; a < 3; ++a) { bl[a] = S.lo[a][ii]; bh[a] = S.hi[a][ii]; }
    }
  };
  auto area = [&](int c) {
    float bl[3], bh[3];
    box_of(c, bl, bh);
    const float dx = bh[0] - bl[0], dy = bh[1] - bl[1], dz = bh[2] - bl[2];
    return dx * dy + dy * dz + dz * dx;
  };
  const float inf = __int_as_float(0x7f800000);
  int nn = 1, head = 0, tail = 0, maxdep = 1;
  if (n == 1) {
    S.queue[0][0] = -1;  // a single instance: one node holding it
  } else {
    S.queue[0][0] = 0;
  }
  S.queue[1][0] = 0;
  S.queue[2][0] = 1;
  tail = 1;
  while (head < tail) {
    const int x = S.queue[0][head], q = S.queue[1][head], dep = S.queue[2][head];
    ++head;
    int mem[4] = {0, 0, 0, 0}, cnt;
    if (x < 0) {
      mem[0] = n - 1;  // code of the single leaf (sorted position 0)
      cnt = 1;
    } else {
      mem[0] = S.child[0][x];
      mem[1] = S.child[1][x];
      cnt = 2;
      while (cnt < 4) {
        int best = -1;
        float ba = -1.0f;
        for (int k = 0; k < cnt; ++k)
          if (mem[k] < n - 1) {
            const float a = area(mem[k]);
            if (a > ba) { ba = a; best = k; }
          }
        if (best < 0) break;
        const int c = mem[best];
        mem[best] = S.child[0][c];
        mem[cnt++] = S.child[1][c];
      }
    }
    float lx[4], ly[4], lz[4], hx[4], hy[4], hz[4];
    int link[4];
    for (int k = 0; k < 4; ++k) {
      if (k >= cnt) {
        lx[k] = ly[k] = lz[k] = inf;
        hx[k] = hy[k] = hz[k] = -inf;
        link[k] = kEmptyLink;
        continue;
      }
      float bl[3], bh[3];
      box_of(mem[k], bl, bh);
      lx[k] = bl[0]; ly[k] = bl[1]; lz[k] = bl[2];
      hx[k] = bh[0]; hy[k] = bh[1]; hz[k] = bh[2];
      if (mem[k] < n - 1) {
        link[k] = nn;
        S.queue[0][tail] = mem[k];
        S.queue[1][tail] = nn;
        S.queue[2][tail] = dep + 1;
        ++tail;
        ++nn;
        maxdep = max(maxdep, dep + 1);
      } else {
        link[k] = ~S.body[(int)(S.key[mem[k] - (n - 1)] & 1023ull)];
      }
    }
    Node4* o = tlas + q;
    o->lox = make_float4(lx[0], lx[1], lx[2], lx[3]);
    o->loy = make_float4(ly[0], ly[1], ly[2], ly[3]);
    o->loz = make_float4(lz[0], lz[1], lz[2], lz[3]);
    o->hix = make_float4(hx[0], hx[1], hx[2], hx[3]);
    o->hiy = make_float4(hy[0], hy[1], hy[2], hy[3]);
    o->hiz = make_float4(hz[0], hz[1], hz[2], hz[3]);
    o->link = make_int4(link[0], link[1], link[2], link[3]);
    o->src = make_int4(-1, -1, -1, -1);
  }
  if (maxdep > kTlasMaxDepth4) {  // the traversal stack is sized for kTlasMaxDepth4 top-level depths
    info->err = 1;
    atomicOr(err, kErrStack);
    return;
  }
  info->n = nn;
}

// ----------------------------------------------------------------------------
// Per-frame refit of the 4-wide tree, by treelets.  At build the tree is cut
// into treelets -- the largest subtrees of at most kTlNodes 4-wide nodes (a
// treelet root has at most kTlNodes nodes in its subtree, its parent more)
// -- and the top nodes above them.  A treelet's leaves are one contiguous
// range of sorted triangles (a subtree of the radix tree covers a key
// range), so each frame
//   1. k_refit_leaves writes every triangle's 48-B record and its box
//      (`stage`, 24 B per leaf, coalesced);
//   2. k_refit_tl, one warp per treelet, reads its leaves' boxes (one
//      range) and writes its nodes deepest first, each node's six child-box
//      vectors whole (96 B), from the leaf boxes and the unions of its
//      internal children in shared memory; the treelet root's union goes to
//      nunion;
//   3. the top nodes, deepest depth first, from nunion and `stage`.
// Each node is written once, whole, and no node's boxes are read back.  Min/max are
// exact, so every box equals the min/max over its triangles' vertices bit
// for bit.
// ----------------------------------------------------------------------------
constexpr int kTlNodes = 32;                 // nodes per treelet, at most (= one warp)
constexpr int kTlLeaves = 3 * kTlNodes + 1;  // leaves of a 4-wide subtree of kTlNodes nodes, at most
constexpr int kTlWarps = 4;                  // treelets per block
// a treelet's boxes in shared memory, 6 floats per slot: its leaves
// [0, kTlLeaves), its nodes' unions [kTlLeaves, kTlLeaves + kTlNodes), and
// one slot holding the inverted infinite box (an unused child)
constexpr int kTlSlotEmpty = kTlLeaves + kTlNodes;
constexpr int kTlSlots = kTlSlotEmpty + 1;
// build counters: [0] treelets, [1] orphan leaves, [2] top nodes, [3] error
// bits, [4] leaves covered by treelets
constexpr int kTlCounters = 8;

// Triangle at sorted position p (index record id): world vertices -> its
// 48-B record; box.
__device__ __forceinline__ void leaf_record_id(const float4* __restrict__ rest, const uint16_t* __restrict__ vb,
                                               const float* __restrict__ xf, uint4 id,
                                               const uint32_t* __restrict__ smat, float4* __restrict__ tris,
                                               int64_t p, float3& lo, float3& hi) {
  const float3 w0 = xform(xf + 12 * vb[id.x], rest[id.x]);
  const float3 w1 = xform(xf + 12 * vb[id.y], rest[id.y]);
  const float3 w2 = xform(xf + 12 * vb[id.z], rest[id.z]);
  const float3 e1 = sub3(w1, w0), e2 = sub3(w2, w0);
  tris[3 * p] = make_float4(w0.x, w0.y, w0.z, __uint_as_float(id.w));
  tris[3 * p + 1] = make_float4(e1.x, e1.y, e1.z, __uint_as_float(smat[p]));
  tris[3 * p + 2] = make_float4(e2.x, e2.y, e2.z, 0.0f);
  lo = fmin3(w0, fmin3(w1, w2));
  hi = fmax3(w0, fmax3(w1, w2));
}

__device__ __forceinline__ void leaf_record(const float4* __restrict__ rest, const uint16_t* __restrict__ vb,
                                            const float* __restrict__ xf, const uint4* __restrict__ sidx,
                                            const uint32_t* __restrict__ smat, float4* __restrict__ tris, int64_t p,
                                            float3& lo, float3& hi) {
  leaf_record_id(rest, vb, xf, sidx[p], smat, tris, p, lo, hi);
}

// Writes node q's child boxes (b[6][4]: lox, loy, loz, hix, hiy, hiz per
// child slot) whole and returns their union in u[6].
__device__ __forceinline__ void write_node(Node4* __restrict__ nodes4, int64_t q, const float b[6][4], float u[6]) {
  float4* n = &nodes4[q].lox;
#pragma unroll
  for (int k = 0; k < 6; ++k) n[k] = make_float4(b[k][0], b[k][1], b[k][2], b[k][3]);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    u[k] = fminf(fminf(b[k][0], b[k][1]), fminf(b[k][2], b[k][3]));
    u[k + 3] = fmaxf(fmaxf(b[k + 3][0], b[k + 3][1]), fmaxf(b[k + 3][2], b[k + 3][3]));
  }
}

// Leaves: one thread per triangle writes its 48-B record and its box (6
// floats at lbox + 6p).  Short 128-thread blocks: they find room beside a
// render's blocks when the refit overlaps the previous frame's render.
__global__ void __launch_bounds__(128) k_refit_leaves(const float4* __restrict__ rest, const uint16_t* __restrict__ vb,
                                                      const float* __restrict__ xf, const uint4* __restrict__ sidx,
                                                      const uint32_t* __restrict__ smat, int64_t nt,
                                                      float4* __restrict__ tris, float* __restrict__ lbox,
                                                      float* __restrict__ xfb, int nxf) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p < nxf) xfb[p] = xf[p];  // the frame buffer's copy of the body matrices
  if (p >= nt) return;
  float3 lo, hi;
  leaf_record(rest, vb, xf, sidx, smat, tris, p, lo, hi);
  float2* o = reinterpret_cast<float2*>(lbox + 6 * p);
  o[0] = make_float2(lo.x, lo.y);
  o[1] = make_float2(lo.z, hi.x);
  o[2] = make_float2(hi.y, hi.z);
}

// Treelet nodes: one warp per treelet loads its leaves' boxes (one
// contiguous range of lbox) into shared memory, then writes its nodes
// deepest first, one lane per node: the node's six child-box vectors whole
// (96 B) from the leaf boxes and the unions of its internal children, and
// its own union in shared memory for its parent (a warp barrier between
// depths); the treelet root's union also goes to nunion.  Four treelets per
// 128-thread block, no block barrier: the blocks are as short-lived as
// those of the leaf pass, so they fit beside a render's blocks.
__global__ void __launch_bounds__(32 * kTlWarps) k_refit_tl(Node4* __restrict__ nodes4,
                                                            const int4* __restrict__ info,
                                                            const int2* __restrict__ tl_node,
                                                            const int4* __restrict__ refs,
                                                            const float* __restrict__ lbox,
                                                            float* __restrict__ nunion, int ntl) {
  __shared__ float2 boxes[kTlWarps][kTlSlots][3];  // each warp's treelet: lo.xy, lo.z hi.x, hi.yz per slot
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = blockIdx.x * kTlWarps + w;
  if (t >= ntl) return;  // the whole warp
  float2(*bx)[3] = boxes[w];
  const int4 in = info[t];
  const int off = in.x, nn = in.y & 0xffff, maxrd = in.y >> 16, l0 = in.z, l1 = in.w;
  const float inf = __int_as_float(0x7f800000);
  if (lane == 0) {
    bx[kTlSlotEmpty][0] = make_float2(inf, inf);
    bx[kTlSlotEmpty][1] = make_float2(inf, -inf);
    bx[kTlSlotEmpty][2] = make_float2(-inf, -inf);
  }
  const float2* src = reinterpret_cast<const float2*>(lbox + 6 * (int64_t)l0);
  for (int j = lane; j <= l1 - l0; j += 32) {  // a lane per leaf: 3 x 8 B
    bx[j][0] = src[3 * j];
    bx[j][1] = src[3 * j + 1];
    bx[j][2] = src[3 * j + 2];
  }
  int64_t q = -1;
  int rd = -1;
  int4 rf = make_int4(kTlSlotEmpty, kTlSlotEmpty, kTlSlotEmpty, kTlSlotEmpty);
  if (lane < nn) {
    const int2 e = tl_node[off + lane];
    q = e.x;
    rd = e.y;
    rf = refs[off + lane];
  }
  __syncwarp();
  for (int r = maxrd; r >= 0; --r) {
    if (rd == r) {
      const int c4[4] = {rf.x, rf.y, rf.z, rf.w};
      float b[6][4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const float2 x0 = bx[c4[c]][0], x1 = bx[c4[c]][1], x2 = bx[c4[c]][2];
        b[0][c] = x0.x; b[1][c] = x0.y; b[2][c] = x1.x;
        b[3][c] = x1.y; b[4][c] = x2.x; b[5][c] = x2.y;
      }
      float u[6];
      write_node(nodes4, q, b, u);
      bx[kTlLeaves + lane][0] = make_float2(u[0], u[1]);
      bx[kTlLeaves + lane][1] = make_float2(u[2], u[3]);
      bx[kTlLeaves + lane][2] = make_float2(u[4], u[5]);
      if (r == 0)
#pragma unroll
        for (int k = 0; k < 6; ++k) nunion[6 * q + k] = u[k];
    }
    __syncwarp();
  }
}

// A top node: its internal children's unions from nunion (treelet roots and
// deeper top nodes), its leaves' boxes from lbox.
__device__ __forceinline__ void refit_top_node(Node4* __restrict__ nodes4, int64_t q, int64_t n4, int64_t nt,
                                               float* __restrict__ nunion, const float* __restrict__ stage) {
  const int4 lk = nodes4[q].link;
  const int l[4] = {lk.x, lk.y, lk.z, lk.w};
  const float inf = __int_as_float(0x7f800000);
  float b[6][4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const float* src = nullptr;
    if (l[c] >= 0 && l[c] < n4) src = nunion + 6 * (int64_t)l[c];
    else if (l[c] < 0 && l[c] != kEmptyLink && ~(int64_t)l[c] < nt) src = stage + 6 * ~(int64_t)l[c];
#pragma unroll
    for (int k = 0; k < 6; ++k) b[k][c] = src ? __ldcg(src + k) : (k < 3 ? inf : -inf);
  }
  float u[6];
  write_node(nodes4, q, b, u);
#pragma unroll
  for (int k = 0; k < 6; ++k) nunion[6 * q + k] = u[k];
}

__global__ void __launch_bounds__(128) k_refit_top_level(Node4* nodes4, const int32_t* __restrict__ top, int64_t b,
                                                         int64_t e, int64_t n4, int64_t nt, float* nunion,
                                                         const float* __restrict__ stage) {
  const int64_t i = b + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < e) refit_top_node(nodes4, top[i], n4, nt, nunion, stage);
}

// groups g0 .. g1 of the top list (each one depth, deepest first) in order
__global__ void __launch_bounds__(1024) k_refit_top_small(Node4* nodes4, const int32_t* __restrict__ top,
                                                          const int64_t* __restrict__ grp, int g0, int g1, int64_t n4,
                                                          int64_t nt, float* nunion, const float* __restrict__ stage) {
  for (int g = g0; g <= g1; ++g) {
    for (int64_t i = grp[g] + threadIdx.x; i < grp[g + 1]; i += blockDim.x)
      refit_top_node(nodes4, top[i], n4, nt, nunion, stage);
    __syncthreads();
  }
}

// ---- treelet build (once per build, single-level trees) ----------------------
// subtree node and leaf counts, one depth (deepest first)
__global__ void k_tl_size(const Node4* __restrict__ nodes4, int64_t begin, int64_t end, int64_t n4,
                          int32_t* __restrict__ size, int32_t* __restrict__ nleaf) {
  const int64_t q = begin + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= end) return;
  const int4 lk = nodes4[q].link;
  const int l[4] = {lk.x, lk.y, lk.z, lk.w};
  int32_t sz = 1, nl = 0;
  for (int c = 0; c < 4; ++c) {
    if (l[c] >= 0 && l[c] < n4) {
      sz += size[l[c]];
      nl += nleaf[l[c]];
    } else if (l[c] < 0 && l[c] != kEmptyLink) {
      nl += 1;
    }
  }
  size[q] = sz;
  nleaf[q] = nl;
}

__global__ void k_tl_root(const int32_t* __restrict__ size, int32_t* tid, int32_t* depth, int32_t* top, int32_t* ctr) {
  if (size[0] <= kTlNodes) {
    tid[0] = 0;
    depth[0] = 0;
    ctr[0] = 1;
  } else {
    tid[0] = -1;
    top[0] = 0;
    ctr[2] = 1;
  }
}

// treelet membership, one depth (shallowest first): a child of a top node
// starts a treelet if its subtree is small enough, else it is a top node;
// a child of a treelet node joins that treelet; leaves extend their
// treelet's leaf range or are orphans (children of top nodes, counted)
__global__ void k_tl_assign(const Node4* __restrict__ nodes4, int64_t begin, int64_t end, int d, int64_t n4,
                            int64_t nt, const int32_t* __restrict__ size, int32_t* tid, int32_t* depth, int32_t* lo,
                            int32_t* hi, int32_t* cnt, int32_t* nl, int32_t* top, int32_t* ctr) {
  const int64_t q = begin + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= end) return;
  const int t = tid[q];
  if (t >= 0) atomicAdd(&cnt[t], 1);
  const int4 lk = nodes4[q].link;
  const int l[4] = {lk.x, lk.y, lk.z, lk.w};
  for (int c = 0; c < 4; ++c) {
    if (l[c] >= 0 && l[c] < n4) {
      int tc = t;
      if (t < 0) {
        if (size[l[c]] <= kTlNodes) {
          tc = atomicAdd(&ctr[0], 1);
          depth[tc] = d + 1;
        } else {
          top[atomicAdd(&ctr[2], 1)] = l[c];
        }
      }
      tid[l[c]] = tc;
    } else if (l[c] != kEmptyLink) {  // a leaf (an internal link >= n4 never occurs)
      const int64_t p = ~(int64_t)l[c];
      if (l[c] >= 0 || p >= nt) {  // never for a complete collapse
        atomicOr(&ctr[3], 1);
        continue;
      }
      if (t >= 0) {
        atomicMin(&lo[t], (int32_t)p);
        atomicMax(&hi[t], (int32_t)p);
        atomicAdd(&nl[t], 1);
      } else {
        atomicAdd(&ctr[1], 1);  // an orphan: its box is read by the top pass
      }
    }
  }
}

// exclusive scan of n int32 values: block sums, then each block's scan from
// the sum of the earlier blocks
__global__ void __launch_bounds__(1024) k_scan_sums(const int32_t* __restrict__ in, int64_t n,
                                                    int32_t* __restrict__ bsum) {
  __shared__ int32_t ws[32];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int64_t i = blockIdx.x * 1024ll + tid;
  int32_t v = i < n ? in[i] : 0;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) ws[w] = v;
  __syncthreads();
  if (w == 0) {
    int32_t y = ws[lane];
    for (int o = 16; o > 0; o >>= 1) y += __shfl_xor_sync(0xffffffffu, y, o);
    if (lane == 0) bsum[blockIdx.x] = y;
  }
}

__global__ void __launch_bounds__(1024) k_scan_apply(const int32_t* __restrict__ in, int64_t n,
                                                     const int32_t* __restrict__ bsum, int32_t* __restrict__ out) {
  __shared__ int32_t ws[32];
  __shared__ int32_t base;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if (w == 0) {
    int32_t y = 0;
    for (int k = lane; k < (int)blockIdx.x; k += 32) y += bsum[k];
    for (int o = 16; o > 0; o >>= 1) y += __shfl_xor_sync(0xffffffffu, y, o);
    if (lane == 0) base = y;
  }
  const int64_t i = blockIdx.x * 1024ll + tid;
  const int32_t v = i < n ? in[i] : 0;
  int32_t x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[w] = x;
  __syncthreads();
  if (w == 0) {
    int32_t y = ws[lane];
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t z = __shfl_up_sync(0xffffffffu, y, o);
      if (lane >= o) y += z;
    }
    ws[lane] = y;
  }
  __syncthreads();
  if (i < n) out[i] = base + (w ? ws[w - 1] : 0) + x - v;
}

// list slot of every treelet node (its treelet's nodes contiguous, in any order)
__global__ void k_tl_scatter(int64_t n4, const int32_t* __restrict__ tid, const int32_t* __restrict__ off,
                             int32_t* cur, int2* __restrict__ tl_node, int32_t* __restrict__ local) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= n4) return;
  const int t = tid[q];
  if (t < 0) return;
  const int32_t k = atomicAdd(&cur[t], 1);
  tl_node[off[t] + k] = make_int2((int)q, 0);
  local[q] = k;
}

// per list slot: depth below the treelet root, and its children as
// shared-memory slots of the treelet kernel (leaf - first leaf, kTlLeaves +
// list slot of an internal child, kTlSlotEmpty)
__global__ void k_tl_refs(const Node4* __restrict__ nodes4, int64_t nlist, int64_t n4, int64_t nt,
                          int2* __restrict__ tl_node, const int32_t* __restrict__ tid, const int32_t* __restrict__ local,
                          const int32_t* __restrict__ lo, const int32_t* __restrict__ depth,
                          const int64_t* __restrict__ lvl4, int D, int4* __restrict__ refs, int32_t* maxrd,
                          int32_t* ctr) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nlist) return;
  const int q = tl_node[i].x;
  if (q < 0 || q >= n4) {  // never: every slot is written once by k_tl_scatter
    atomicOr(&ctr[3], 32);
    return;
  }
  const int t = tid[q];
  int dq = 0;
  for (int k = 1; k < D; ++k) dq += lvl4[k] <= q;
  const int r = dq - depth[t];
  tl_node[i].y = r;
  atomicMax(&maxrd[t], r);
  const int4 lk = nodes4[q].link;
  const int l[4] = {lk.x, lk.y, lk.z, lk.w};
  int o[4];
  for (int c = 0; c < 4; ++c) {
    o[c] = kTlSlotEmpty;
    if (l[c] >= 0 && l[c] < n4) {
      if (tid[l[c]] != t || local[l[c]] >= kTlNodes) atomicOr(&ctr[3], 4);
      else o[c] = kTlLeaves + local[l[c]];
    } else if (l[c] < 0 && l[c] != kEmptyLink) {
      const int64_t j = ~(int64_t)l[c] - lo[t];
      if (j < 0 || j >= kTlLeaves || ~(int64_t)l[c] >= nt) atomicOr(&ctr[3], 8);
      else o[c] = (int)j;
    }
  }
  refs[i] = make_int4(o[0], o[1], o[2], o[3]);
}

// top nodes: a flag per node, then (after an exclusive scan of the flags)
// the list in descending node order = deepest depth first
__global__ void k_tl_topflag(int64_t n4, const int32_t* __restrict__ tid, int32_t* __restrict__ flag) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q < n4) flag[q] = tid[q] < 0 ? 1 : 0;
}

__global__ void k_tl_topscatter(int64_t n4, int64_t ntop, const int32_t* __restrict__ flag,
                                const int32_t* __restrict__ pos, int32_t* __restrict__ top) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q < n4 && flag[q] && pos[q] < ntop) top[ntop - 1 - pos[q]] = (int32_t)q;  // (pos < ntop: always)
}

// pos at the first node of each depth (the top nodes above that depth)
__global__ void k_tl_topbounds(const int32_t* __restrict__ pos, const int64_t* __restrict__ lvl4, int D,
                               int32_t* __restrict__ out) {
  const int d = threadIdx.x;
  if (d < D) out[d] = pos[lvl4[d]];
}

// per treelet: (list offset, nodes | max depth << 16, first leaf, last
// leaf); checks that the leaves form one range of at most kTlLeaves
__global__ void k_tl_info(int ntl, int64_t nt, const int32_t* __restrict__ off, const int32_t* __restrict__ cnt,
                          const int32_t* __restrict__ maxrd, const int32_t* __restrict__ lo,
                          const int32_t* __restrict__ hi, const int32_t* __restrict__ nl, int4* __restrict__ info,
                          int32_t* ctr) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntl) return;
  const int n = hi[t] - lo[t] + 1;
  const bool ok = cnt[t] >= 1 && cnt[t] <= kTlNodes && maxrd[t] >= 0 && maxrd[t] < 0x7fff && n >= 1 &&
                  n <= kTlLeaves && (n == nl[t] || nt == 1);
  if (!ok) atomicOr(&ctr[3], 16);
  info[t] = make_int4(off[t], cnt[t] | (maxrd[t] << 16), lo[t], hi[t]);
  atomicAdd(&ctr[4], n);
}

inline int grid_for(int64_t n, int threads) { return (int)((n + threads - 1) / threads); }

}  // namespace

int lbvh_validate(fire_scene_s* s, cudaStream_t st, uint32_t* bad_host) {
  uint32_t* bad = s->ctrl + 8;
  if (int e = cuda_check(cudaMemsetAsync(bad, 0, 4, st), "memset")) return e;
  int64_t n = std::max(s->nv, s->nt);
  if (n > 0) {
    int g = (int)std::min<int64_t>(grid_for(n, 256), 4 * 148 * 8);
    k_validate<<<g, 256, 0, st>>>(s->rest, s->nv, s->idx, s->tmat, s->nt, s->vbody, s->nmat, s->nbody, bad);
    if (int e = cuda_check(cudaGetLastError(), "k_validate")) return e;
  }
  if (int e = cuda_check(cudaMemcpyAsync(bad_host, bad, 4, cudaMemcpyDeviceToHost, st), "copy")) return e;
  if (int e = cuda_check(cudaStreamSynchronize(st), "sync")) return e;
  return cuda_check(cudaMemsetAsync(bad, 0, 4, st), "memset");
}

namespace {
__global__ void k_count_mixed(const uint32_t* __restrict__ idx, const uint16_t* __restrict__ vb, int64_t nt,
                              uint32_t* bad) {
  uint32_t n = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nt; i += (int64_t)gridDim.x * blockDim.x) {
    const uint16_t b = vb[idx[3 * i]];
    n += vb[idx[3 * i + 1]] != b || vb[idx[3 * i + 2]] != b;
  }
  if (n) atomicAdd(bad, n);
}
}  // namespace

int lbvh_count_mixed(fire_scene_s* s, cudaStream_t st, uint32_t* bad_host) {
  uint32_t* bad = s->ctrl + 15;
  if (int e = cuda_check(cudaMemsetAsync(bad, 0, 4, st), "memset")) return e;
  if (s->nt > 0) {
    const int g = (int)std::min<int64_t>(grid_for(s->nt, 256), 4 * 148 * 8);
    k_count_mixed<<<g, 256, 0, st>>>(s->idx, s->vbody, s->nt, bad);
    if (int e = cuda_check(cudaGetLastError(), "k_count_mixed")) return e;
  }
  if (int e = cuda_check(cudaMemcpyAsync(bad_host, bad, 4, cudaMemcpyDeviceToHost, st), "copy")) return e;
  return cuda_check(cudaStreamSynchronize(st), "sync");
}

int lbvh_build(fire_scene_s* s, cudaStream_t st) {
  const int64_t T = s->nt;
  if (T == 0) { s->built = true; s->height = 0; return FIRE_OK; }
  s->built = false;  // until this build has completed
  // bounds live in ctrl[9..14]: lo = +inf ordered, hi = -inf ordered
  uint32_t init[6];
  for (int k = 0; k < 3; ++k) { init[k] = 0xffffffffu; init[3 + k] = 0u; }
  if (int e = cuda_check(cudaMemcpyAsync(s->ctrl + 9, init, sizeof(init), cudaMemcpyHostToDevice, st), "copy")) return e;
  uint32_t* bounds = s->ctrl + 9;
  // two-level mode: the bottom levels are built over the rest pose
  const float* xf_geom = s->two_level ? s->xf_ident : s->xf;
  prof_begin(s, kStageBuild, st);
  k_centroids<<<(int)std::min<int64_t>(grid_for(T, 256), (int64_t)sm_count() * 8), 256, 0, st>>>(
      s->rest, s->idx, s->vbody, xf_geom, T, s->cen, bounds);
  int prefix_bits = 0;
  while (s->nbody > 1 && (1 << prefix_bits) < s->nbody) ++prefix_bits;
  const int mbits = std::min(21, (63 - prefix_bits) / 3);
  const int coarse_bits = s->two_level ? 0 : std::min(kCoarseBits, mbits);
  k_morton<<<grid_for(T, 256), 256, 0, st>>>(s->cen, T, bounds, s->idx, s->vbody, prefix_bits, mbits, coarse_bits,
                                             s->keys, s->order, s->keys_orig);
  // sort (keys, order) with ping-pong through (keys_alt, vals_alt); 7 passes
  const int ntiles = (int)((T + kSortTile - 1) / kSortTile);
  uint32_t* totals = s->hist + (int64_t)kSortBins * ntiles;
  uint64_t* ka = s->keys; uint32_t* va = s->order;
  uint64_t* kb = s->keys_alt; uint32_t* vb = s->vals_alt;
  for (int p = 0; p < kSortPasses; ++p) {
    int shift = p * kSortBits;
    k_sort_upsweep<<<ntiles, kSortThreads, 0, st>>>(ka, T, shift, s->hist, ntiles);
    k_sort_scan<<<kSortBins, 1024, 0, st>>>(s->hist, ntiles, totals);
    k_sort_downsweep<<<ntiles, kSortThreads, 0, st>>>(ka, va, kb, vb, T, shift, s->hist, ntiles, totals);
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  // odd pass count: results are in the alt buffers; swap ownership
  if (ka != s->keys) { std::swap(s->keys, s->keys_alt); std::swap(s->order, s->vals_alt); }
  if (T > 1) {
    if (int e = cuda_check(cudaMemsetAsync(s->leaf_slot, 0xff, 4 * T, st), "memset")) return e;
    if (int e = cuda_check(cudaMemsetAsync(s->node_slot, 0xff, 4 * (T - 1), st), "memset")) return e;
    if (int e = cuda_check(cudaMemsetAsync(s->nodes, 0xff, 64 * (T - 1), st), "memset")) return e;
    k_karras<<<grid_for(T - 1, 256), 256, 0, st>>>(s->keys, T, s->nodes, s->leaf_slot, s->node_slot);
  }
  k_gather_sorted<<<grid_for(T, 256), 256, 0, st>>>(s->order, s->idx, s->tmat, T, s->sidx, s->smat, s->rank);
  if (T > 1)
    if (int e = cuda_check(cudaMemsetAsync(s->counters, 0, 4 * (T - 1), st), "memset")) return e;
  const int nxf = 12 * s->nbody;
  k_refit_build<<<grid_for(std::max<int64_t>(T, nxf), 256), 256, 0, st>>>(
      s->rest, s->vbody, xf_geom, s->sidx, s->smat, T, s->tris, s->nodes, s->leaf_slot, s->node_slot, s->counters,
      s->xf_buf[s->cur], nxf, s->two_level ? 1 : 0);
  prof_end(s, kStageBuild, st, 2 + 3 * kSortPasses + (T > 1 ? 1 : 0) + 2);
  if (int e = cuda_check(cudaGetLastError(), "build kernels")) return e;
  Node n0;
  if (int e = cuda_check(cudaMemcpyAsync(&n0, &s->nodes[0], sizeof(Node), cudaMemcpyDeviceToHost, st), "copy")) return e;
  if (int e = cuda_check(cudaStreamSynchronize(st), "sync")) return e;
  int h0, h1;
  memcpy(&h0, &n0.b.w, 4);
  memcpy(&h1, &n0.d.w, 4);
  s->height = T > 1 ? 1 + std::max(h0, h1) : 1;
  // 4-wide traversal tree: collapse depth by depth from the binary root; the
  // nodes of depth L get the contiguous indices [lvl4[L], lvl4[L+1]).  One
  // launch per depth with the queue lengths kept on the device (qlen[d] =
  // nodes at depth d); a 4-wide depth consumes at least one binary level,
  // so `height` launches suffice, and the lengths are read back once.
  {
    // queue halves hold one pair per binary internal node (T - 1); the
    // 4-wide nodes number at most T (two-level: a root per body, and every
    // further node consumes a binary node of its body)
    const int64_t capq = std::max<int64_t>(T - 1, 1);
    const int64_t cap4 = std::max<int64_t>(T, 1);
    int32_t* qa = s->q4;
    int32_t* qb = s->q4 + 2 * capq;
    uint32_t* qlen = reinterpret_cast<uint32_t*>(s->lvl_aux + 8 * kMaxDepth4);  // [kMaxDepth4]
    uint32_t* alloc = qlen + kMaxDepth4;                                         // 4-wide nodes allocated
    const int32_t root[2] = {0, 0};
    const int L = std::max(1, std::min(s->height, kMaxDepth4 - 1));
    // h[d]: 4-wide nodes at depth d; h[kMaxDepth4]: nodes allocated;
    // h[kMaxDepth4 + 1]: depth-0 nodes (the roots)
    std::vector<uint32_t> h(kMaxDepth4 + 2, 0u);
    if (!s->two_level) {
      h[0] = 1u;               // depth 0: the root
      h[kMaxDepth4] = 1u;      // the root is allocated
      h[kMaxDepth4 + 1] = 1u;
      if (int e = cuda_check(cudaMemcpyAsync(qa, root, sizeof(root), cudaMemcpyHostToDevice, st), "copy")) return e;
    }
    if (int e = cuda_check(cudaMemcpyAsync(qlen, h.data(), 4 * h.size(), cudaMemcpyHostToDevice, st), "copy"))
      return e;
    if (s->two_level) {
      // every body's subtree root starts a bottom level (key prefix above bit 3m)
      int prefix_bits = 0;
      while (s->nbody > 1 && (1 << prefix_bits) < s->nbody) ++prefix_bits;
      const int shift = 3 * std::min(21, (63 - prefix_bits) / 3);
      if (s->nbody > kMaxTlasBodies) return set_error(FIRE_ERR_INVALID_ARG, "two-level mode: too many bodies");
      if (int e = cuda_check(cudaMemsetAsync(s->body_range, 0xff, 8 * (size_t)s->nbody, st), "memset")) return e;
      k_body_ranges<<<grid_for(T, 256), 256, 0, st>>>(s->keys, T, prefix_bits > 0 ? shift : 63, s->nbody,
                                                       s->body_range, s->ctrl + 8);
      k_body_roots<<<1, 1024, 0, st>>>(s->keys, T, s->body_range, s->nbody, s->leaf_slot, s->blas_root, qa, qlen,
                                       s->nodes4);
    }
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(grid_for(capq, 256), (int64_t)sm_count() * 8));
    for (int d = 0; d < L; ++d) {
      k_collapse<<<grid, 256, 0, st>>>(s->nodes, qa, qlen + d, qb, qlen + d + 1, alloc, s->nodes4, cap4);
      std::swap(qa, qb);
    }
    if (int e = cuda_check(cudaGetLastError(), "collapse")) return e;
    if (int e = cuda_check(cudaMemcpyAsync(h.data(), qlen, 4 * h.size(), cudaMemcpyDeviceToHost, st), "copy"))
      return e;
    if (int e = cuda_check(cudaStreamSynchronize(st), "collapse")) return e;
    if (h[L] != 0u) return set_error(FIRE_ERR_CUDA, "4-wide collapse deeper than supported");
    h[0] = h[kMaxDepth4 + 1];  // depth 0 also holds the one-triangle bottom levels (not queued)
    s->lvl4.assign(1, 0);
    for (int d = 0; d < L && h[d] > 0; ++d) s->lvl4.push_back(std::min<int64_t>(s->lvl4.back() + h[d], cap4));
    s->n4 = s->lvl4.back();
    s->height4 = (int)s->lvl4.size() - 1;
    if (int e = cuda_check(cudaMemcpyAsync(s->lvl_aux, s->lvl4.data(), 8 * s->lvl4.size(), cudaMemcpyHostToDevice, st),
                           "copy"))
      return e;
    k_fill4<<<grid_for(s->n4, 256), 256, 0, st>>>(s->nodes, s->nodes4, s->n4);
    if (s->two_level) {
      k_body_boxes<<<grid_for(s->nbody, 256), 256, 0, st>>>(s->nodes4, s->n4, s->blas_root, s->nbody, s->body_box);
      k_top_entries<<<1, kMaxTlasBodies, 0, st>>>(s->nodes4, s->n4, s->blas_root, s->body_box, s->nbody, s->inst,
                                                  s->inst_box, s->ctrl + 8);
    }
    if (int e = cuda_check(cudaGetLastError(), "4-wide tree")) return e;
    if (int e = cuda_check(cudaStreamSynchronize(st), "sync")) return e;  // lvl4 host vector copied
  }
  if (int e = treelet_build(s, st)) return e;
  s->built = true;
  return FIRE_OK;
}

int tlas_build(fire_scene_s* s, cudaStream_t st) {
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [] {
    attr = cudaFuncSetAttribute(k_tlas, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TlasSmem));
  });
  if (int e = cuda_check(attr, "top-level shared memory")) return e;
  if (s->nbody > kMaxTlasBodies) return set_error(FIRE_ERR_INVALID_ARG, "two-level mode: too many bodies");
  k_tlas<<<1, 1024, sizeof(TlasSmem), st>>>(s->xf, s->nbody, s->blas_root, s->body_box, s->inst, s->inst_box,
                                            s->tlas_buf[s->cur],
                                            s->tinfo_buf[s->cur], s->xf_buf[s->cur], s->ctrl + 8);
  return cuda_check(cudaGetLastError(), "k_tlas");
}

int lbvh_refit(fire_scene_s* s, cudaStream_t st) {
  const int64_t T = s->nt;
  if (T == 0) return FIRE_OK;
  prof_begin(s, kStageRefit, st);
  const int nxf = 12 * s->nbody;
  k_refit_leaves<<<grid_for(std::max<int64_t>(T, nxf), 128), 128, 0, st>>>(s->rest, s->vbody, s->xf, s->sidx, s->smat, T, s->tris, s->stage,
                                              s->xf_buf[s->cur], nxf);
  if (s->ntl > 0)
    k_refit_tl<<<(unsigned)((s->ntl + kTlWarps - 1) / kTlWarps), 32 * kTlWarps, 0, st>>>(
        s->nodes4, s->tl_info, s->tl_node, s->tl_refs, s->stage, s->nunion, s->ntl);
  // top nodes, deepest depth first: a depth of more than 1024 top nodes gets
  // its own launch, runs of smaller ones go to one block
  const std::vector<int64_t>& grp = s->tl_grp_host;
  const int G = (int)grp.size() - 1;
  int launches = s->ntl > 0 ? 2 : 1;
  for (int g = 0; g < G;) {
    const int64_t n = grp[g + 1] - grp[g];
    ++launches;
    if (n > 1024) {
      k_refit_top_level<<<grid_for(n, 128), 128, 0, st>>>(s->nodes4, s->tl_top, grp[g], grp[g + 1], s->n4, T,
                                                           s->nunion, s->stage);
      ++g;
      continue;
    }
    int g1 = g;
    while (g1 + 1 < G && grp[g1 + 2] - grp[g1 + 1] <= 1024) ++g1;
    k_refit_top_small<<<1, 1024, 0, st>>>(s->nodes4, s->tl_top, s->tl_grp, g, g1, s->n4, T, s->nunion, s->stage);
    g = g1 + 1;
  }
  prof_end(s, kStageRefit, st, launches);
  return cuda_check(cudaGetLastError(), "refit kernels");
}

// Treelets of a single-level tree (after the collapse; see the refit above).
int treelet_build(fire_scene_s* s, cudaStream_t st) {
  s->ntl = 0;
  s->norphan = 0;
  s->tl_grp_host.assign(1, 0);
  if (s->two_level || s->n4 == 0) return FIRE_OK;
  const int64_t T = s->nt, n4 = s->n4;
  int32_t* w = s->tl_scratch;
  int32_t *size = w, *nleaf = w + T, *tid = w + 2 * T, *local = w + 3 * T, *lo = w + 4 * T, *hi = w + 5 * T;
  int32_t *cnt = w + 6 * T, *cur = w + 7 * T, *depth = w + 8 * T, *maxrd = w + 9 * T, *nl = w + 10 * T;
  int32_t* off = w + 11 * T;
  int32_t* bsum = w + 12 * T;
  int32_t* ctr = bsum + (T + 1023) / 1024 + 1;
  if (int e = cuda_check(cudaMemsetAsync(lo, 0x7f, 4 * T, st), "memset")) return e;  // 0x7f7f7f7f > any leaf
  if (int e = cuda_check(cudaMemsetAsync(hi, 0xff, 4 * T, st), "memset")) return e;  // -1
  if (int e = cuda_check(cudaMemsetAsync(cnt, 0, 8 * T, st), "memset")) return e;    // cnt, cur
  if (int e = cuda_check(cudaMemsetAsync(maxrd, 0, 8 * T, st), "memset")) return e;  // maxrd, nl
  if (int e = cuda_check(cudaMemsetAsync(ctr, 0, 4 * kTlCounters, st), "memset")) return e;
  const int D = (int)s->lvl4.size() - 1;
  for (int d = D - 1; d >= 0; --d) {
    const int64_t n = s->lvl4[d + 1] - s->lvl4[d];
    k_tl_size<<<grid_for(n, 256), 256, 0, st>>>(s->nodes4, s->lvl4[d], s->lvl4[d + 1], n4, size, nleaf);
  }
  k_tl_root<<<1, 1, 0, st>>>(size, tid, depth, s->tl_top, ctr);
  for (int d = 0; d < D; ++d) {
    const int64_t n = s->lvl4[d + 1] - s->lvl4[d];
    k_tl_assign<<<grid_for(n, 256), 256, 0, st>>>(s->nodes4, s->lvl4[d], s->lvl4[d + 1], d, n4, T, size, tid, depth,
                                                  lo, hi, cnt, nl, s->tl_top, ctr);
  }
  int32_t h[kTlCounters];
  if (int e = cuda_check(cudaMemcpyAsync(h, ctr, sizeof(h), cudaMemcpyDeviceToHost, st), "copy")) return e;
  if (int e = cuda_check(cudaStreamSynchronize(st), "treelets")) return e;
  if (h[3] != 0 || h[0] < 1) return set_error(FIRE_ERR_CUDA, "treelet partition of the 4-wide tree failed");
  const int ntl = h[0];
  const int64_t norph = h[1], ntop = h[2], nlist = n4 - ntop;
  const int64_t nb = (ntl + 1023) / 1024;
  k_scan_sums<<<(unsigned)nb, 1024, 0, st>>>(cnt, ntl, bsum);
  k_scan_apply<<<(unsigned)nb, 1024, 0, st>>>(cnt, ntl, bsum, off);
  k_tl_scatter<<<grid_for(n4, 256), 256, 0, st>>>(n4, tid, off, cur, s->tl_node, local);
  if (nlist > 0)
    k_tl_refs<<<grid_for(nlist, 256), 256, 0, st>>>(s->nodes4, nlist, n4, T, s->tl_node, tid, local, lo, depth,
                                                    reinterpret_cast<const int64_t*>(s->lvl_aux), D, s->tl_refs,
                                                    maxrd, ctr);
  k_tl_info<<<grid_for(ntl, 256), 256, 0, st>>>(ntl, T, off, cnt, maxrd, lo, hi, nl, s->tl_info, ctr);
  // top list, deepest depth first (descending node order), and where each
  // depth starts in it
  int32_t* flag = nleaf;  // free after the sizes
  int32_t* pos = size;    // free after the assignment
  int32_t* bounds = ctr + kTlCounters;  // [D]
  const int64_t nb4 = (n4 + 1023) / 1024;
  k_tl_topflag<<<grid_for(n4, 256), 256, 0, st>>>(n4, tid, flag);
  k_scan_sums<<<(unsigned)nb4, 1024, 0, st>>>(flag, n4, bsum);
  k_scan_apply<<<(unsigned)nb4, 1024, 0, st>>>(flag, n4, bsum, pos);
  k_tl_topscatter<<<grid_for(n4, 256), 256, 0, st>>>(n4, ntop, flag, pos, s->tl_top);
  k_tl_topbounds<<<1, kMaxDepth4, 0, st>>>(pos, reinterpret_cast<const int64_t*>(s->lvl_aux), D, bounds);
  std::vector<int32_t> P((size_t)D + 1);
  if (int e = cuda_check(cudaMemcpyAsync(h, ctr, sizeof(h), cudaMemcpyDeviceToHost, st), "copy")) return e;
  if (int e = cuda_check(cudaMemcpyAsync(P.data(), bounds, 4 * (size_t)D, cudaMemcpyDeviceToHost, st), "copy"))
    return e;
  if (int e = cuda_check(cudaGetLastError(), "treelet kernels")) return e;
  if (int e = cuda_check(cudaStreamSynchronize(st), "treelets")) return e;
  if (h[3] != 0 || h[4] + norph != T)
    return set_error(FIRE_ERR_CUDA, "treelet partition of the 4-wide tree failed");
  P[D] = (int32_t)ntop;
  // depth d's top nodes sit at [ntop - P[d+1], ntop - P[d]) of the list
  std::vector<int64_t> grp(1, 0);
  for (int d = D - 1; d >= 0; --d)
    if (P[d + 1] > P[d]) grp.push_back(ntop - P[d]);
  if (grp.back() != ntop) return set_error(FIRE_ERR_CUDA, "treelet top list inconsistent");
  if (int e = cuda_check(cudaMemcpyAsync(s->tl_grp, grp.data(), 8 * grp.size(), cudaMemcpyHostToDevice, st), "copy"))
    return e;
  s->ntl = ntl;
  s->norphan = norph;
  s->tl_grp_host = grp;
  return FIRE_OK;
}

}  // namespace fire
