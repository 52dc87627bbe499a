// Device functions of the visibility and shading path, shared by the
// single-frame, batched and differentiable kernels.
//   camera ray     -- §IV-A-1 view transform restated as a pinhole ray
//   nearest hit    -- replaces the rasterised main pass + depth test (§IV-A-1)
//   any hit        -- §IV-B-3 shadow ray query to each light
//   brdf           -- §IV-B-1 Cook-Torrance (GGX D, Schlick F, Schlick-GGX G) + Lambert
#pragma once

#include "fire_internal.cuh"

namespace fire {

constexpr float kPi = 3.14159265358979323846f;
constexpr float kInvPi = 0.318309886183790671538f;
// Relative slack of the box tests (covers the FP32 rounding of the slab
// distances, a few 2^-24, and of the triangle test's t); boxes are only ever
// accepted more often, never less, so the nearest hit is unchanged.
constexpr float kBoxSlack = 1.0f + 1.0f / 65536.0f;
constexpr uint32_t kFull = 0xffffffffu;

__host__ __device__ __forceinline__ float inf_f() { return bits_as_float(0x7f800000u); }

// ---------------------------------------------------------------------------
// Camera: sample k of pixel (x, y):
//   fx = x + (0.5 + ox), ndx = (2 fx)/W - 1, sx = ndx * sxs   (same for y with
//   ndy = 1 - (2 fy)/H, sy = ndy * sys); d = normalize(fma(sx, r, fma(sy, u, f)))
// 4 spp: rotated grid (-1/8,-3/8), (3/8,-1/8), (-3/8,1/8), (1/8,3/8).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void spp_offset(int spp, int k, float& ox, float& oy) {
  ox = 0.0f;
  oy = 0.0f;
  if (spp == 4) {
    ox = (k == 0) ? -0.125f : (k == 1) ? 0.375f : (k == 2) ? -0.375f : 0.125f;
    oy = (k == 0) ? -0.375f : (k == 1) ? -0.125f : (k == 2) ? 0.125f : 0.375f;
  }
}

__device__ __forceinline__ float3 cam_dir(const CamParams& c, int x, int y, int k) {
  float ox, oy;
  spp_offset(c.spp, k, ox, oy);
  float fx = (float)x + (0.5f + ox);
  float fy = (float)y + (0.5f + oy);
  float ndx = (2.0f * fx) / (float)c.W - 1.0f;
  float ndy = 1.0f - (2.0f * fy) / (float)c.H;
  float sx = ndx * c.sxs, sy = ndy * c.sys;
  float3 dir = f3(fmaf(sx, c.rx, fmaf(sy, c.ux, c.fx)), fmaf(sx, c.ry, fmaf(sy, c.uy, c.fy)),
                  fmaf(sx, c.rz, fmaf(sy, c.uz, c.fz)));
  return normalize3(dir);
}

// Reciprocal direction for the slab test; components below 1e-30 in
// magnitude become +-1e30 so that no 0 * inf appears.
__host__ __device__ __forceinline__ float rcp_rn(float d) {
#ifdef __CUDA_ARCH__
  return __frcp_rn(d);
#else
  return 1.0f / d;  // IEEE division: the correctly rounded reciprocal, as __frcp_rn
#endif
}
__host__ __device__ __forceinline__ float safe_rcp(float d) {
  return fabsf(d) < 1e-30f ? (d >= 0.0f ? 1e30f : -1e30f) : rcp_rn(d);
}

// Conservative slab test of the box [lo, hi] against [0, tmax]; returns the
// entry distance in tnear.
__device__ __forceinline__ bool slab(float3 o, float3 inv, float lox, float loy, float loz, float hix,
                                     float hiy, float hiz, float tmax, float& tnear) {
  float tx0 = (lox - o.x) * inv.x, tx1 = (hix - o.x) * inv.x;
  float ty0 = (loy - o.y) * inv.y, ty1 = (hiy - o.y) * inv.y;
  float tz0 = (loz - o.z) * inv.z, tz1 = (hiz - o.z) * inv.z;
  float tn = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fmaxf(fminf(tz0, tz1), 0.0f));
  float tf = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fminf(fmaxf(tz0, tz1), tmax));
  tnear = tn;
  return tn <= tf * kBoxSlack;
}

// ---------------------------------------------------------------------------
// Ray/triangle test (Moller-Trumbore) in the fixed FP32 order:
//   p = d x e2, det = e1.p, inv = 1/det, s = o - v0, u = (s.p) inv,
//   q = s x e1, v = (d.q) inv, t = (e2.q) inv; inside iff det != 0, u >= 0,
//   u <= 1, v >= 0, fl(u + v) <= 1.  Every term is computed and the decision
//   taken once at the end (a det of 0 gives an infinite inv and u, v that
//   fail the tests): in the traversal's leaf loop, which runs with few lanes,
//   early exits only split those lanes further (shadow pass 0.929 -> 0.920
//   ms against returning at det == 0 and at u outside [0, 1]).
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ bool mt_t(float3 o, float3 d, float4 A, float4 B, float4 C, float& t) {
  float3 v0 = xyz(A), e1 = xyz(B), e2 = xyz(C);
  float3 p = cross3(d, e2);
  float det = dot3(e1, p);
  float inv = rcp_rn(det);
  float3 s = sub3(o, v0);
  float u = dot3(s, p) * inv;
  float3 q = cross3(s, e1);
  float v = dot3(d, q) * inv;
  t = dot3(e2, q) * inv;
  return det != 0.0f && u >= 0.0f && u <= 1.0f && v >= 0.0f && (u + v) <= 1.0f;
}

// Memory policy of the traversal code, which is written once for the device
// and the host: DeviceLoads (read-only-path __ldg loads, atomicOr on the
// sticky error word) in the kernels; the host emulation passes a policy that
// checks every load.  (The host side of these members exists only because
// the traversal is a host-and-device template; host code uses its own.)
struct DeviceLoads {
#ifdef __CUDA_ARCH__
  __host__ __device__ static float4 f4(const float4* p) { return __ldg(p); }
  __host__ __device__ static int4 i4(const int4* p) { return __ldg(p); }
  __host__ __device__ static float f1(const float* p) { return __ldg(p); }
  __host__ __device__ static int i1(const int32_t* p) { return __ldg(p); }
  __host__ __device__ static void fail(uint32_t* e, uint32_t bits) { atomicOr(e, bits); }
#else
  __host__ __device__ static float4 f4(const float4* p) { return *p; }
  __host__ __device__ static int4 i4(const int4* p) { return *p; }
  __host__ __device__ static float f1(const float* p) { return *p; }
  __host__ __device__ static int i1(const int32_t* p) { return *p; }
  __host__ __device__ static void fail(uint32_t* e, uint32_t bits) { *e |= bits; }
#endif
};

// Index of the lowest set bit of a non-zero mask.
__host__ __device__ __forceinline__ int lowest_slot(unsigned m) {
#ifdef __CUDA_ARCH__
  return __ffs(m) - 1;
#else
  return __builtin_ctz(m);
#endif
}

struct TraceCtx {
  const Node4* __restrict__ nodes4;  // 4-wide traversal tree
  int64_t n4;
  float span;        // largest |coordinate| of the scene box (box-test slack)
  const float4* __restrict__ tris;
  int64_t nt;
  int64_t cap;       // node-visit cap per ray (>= 1)
  uint32_t* err;     // sticky error word
};

constexpr int kDone = 0x7fffffff;  // stack sentinel: nothing left to visit

// Leaf = one triangle at sorted position ~code.  Nearest mode updates the
// (t, original index) minimum; any mode returns true on a hit in (0, tmax)
// that is not triangle `skip`.
template <class M, bool ANY>
__host__ __device__ __forceinline__ bool leaf_test(const TraceCtx& c, int code, float3 o, float3 d, float tmax,
                                                   int skip, int& prim, int& pos, float& tb) {
  int p = ~code;
  if ((uint64_t)p >= (uint64_t)c.nt) p = 0;  // never for a built tree (keeps loads in bounds)
  const float4* tr = c.tris + 3 * (int64_t)p;
  float4 A = M::f4(tr), B = M::f4(tr + 1), C = M::f4(tr + 2);
  int orig = float_as_bits(A.w);
  float t;
  if (ANY) return orig != skip && mt_t(o, d, A, B, C, t) && t > 0.0f && t < tmax;
  if (mt_t(o, d, A, B, C, t) && t > 0.0f && t < inf_f() && (t < tb || (t == tb && orig < prim))) {
    tb = t;
    prim = orig;
    pos = p;
  }
  return false;
}

// Three-input min / max (one instruction each on sm_100-class GPUs; two
// calls on the host).
__host__ __device__ __forceinline__ float fmax3f(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  float r;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
#else
  return fmaxf(fmaxf(a, b), c);
#endif
}
__host__ __device__ __forceinline__ float fmin3f(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  float r;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
#else
  return fminf(fminf(a, b), c);
#endif
}

// Per-ray data of the 4-wide box test: for each axis the member (0..5 =
// lox, loy, loz, hix, hiy, hiz) holding the near plane and the far plane,
// picked once from the sign of the direction, so a child's entry and exit
// distances need no per-axis min/max.
// Each plane distance is one FMA, t = fma(plane, inv, c), with the per-ray
// constants c = -o*inv -+ s.  The slack s_a = 2^-19 (M + |o_a|) |inv_a| (M =
// largest |coordinate| of the scene box) exceeds the FMA form's rounding
// error, |plane*inv| u + |o*inv| u + |t| u <= 3u (M + |o_a|)|inv_a|, by a
// factor of 10 and also covers the triangle test's own rounding, so entry
// distances are only ever lowered and exit distances raised: a box holding a
// hit the triangle test would accept is never culled.
struct RaySetup {
  float3 inv;
  float cnx, cny, cnz, cfx, cfy, cfz;
  int nx, ny, nz, fx, fy, fz;
};

__host__ __device__ __forceinline__ RaySetup ray_setup(float3 o, float3 d, float span) {
  RaySetup r;
  r.inv = f3(safe_rcp(d.x), safe_rcp(d.y), safe_rcp(d.z));
  const float k = 1.0f / 524288.0f;  // 2^-19
  const float sx = k * (span + fabsf(o.x)) * fabsf(r.inv.x);
  const float sy = k * (span + fabsf(o.y)) * fabsf(r.inv.y);
  const float sz = k * (span + fabsf(o.z)) * fabsf(r.inv.z);
  const float ox = -o.x * r.inv.x, oy = -o.y * r.inv.y, oz = -o.z * r.inv.z;
  r.cnx = ox - sx;
  r.cny = oy - sy;
  r.cnz = oz - sz;
  r.cfx = ox + sx;
  r.cfy = oy + sy;
  r.cfz = oz + sz;
  r.nx = r.inv.x >= 0.0f ? 0 : 3;
  r.ny = r.inv.y >= 0.0f ? 1 : 4;
  r.nz = r.inv.z >= 0.0f ? 2 : 5;
  r.fx = 3 - r.nx;
  r.fy = 5 - r.ny;
  r.fz = 7 - r.nz;
  return r;
}

// Entry/exit test of one child against [0, tmax] (entry tn, exit tf), and
// the child's key in the node step's ordering (smallest first):
//   nearest hit: tn + tf, twice the middle of the ray's span inside the box
//     -- small near boxes before large ones that merely start nearer;
//   any hit: -tf, the child whose span reaches farthest along the ray
//     first: an occluder lies between the surface and the light, and the
//     boxes reaching toward the light hold it more often than those that
//     merely start farther.
// (7.3M-triangle frame, against the entry distance -- nearest first, any hit
// farthest first: primary 1.015 -> 0.998 ms, shadow 1.06 -> 0.965 ms; the
// exit alone for the nearest hit 1.07 ms; for any hit the middle 0.985, the
// exit before clamping to tmax 0.983, the span's length 1.42 ms.)  Unused
// slots hold the inverted infinite box (lo = +inf, hi = -inf): entry +inf,
// exit -inf, never hit.  The order changes the work, never the result.
template <bool ANY>
__host__ __device__ __forceinline__ bool slab4(const RaySetup& r, float nx, float ny, float nz, float fx, float fy, float fz,
                                      float tmax, float& key) {
  float tnx = fmaf(nx, r.inv.x, r.cnx), tny = fmaf(ny, r.inv.y, r.cny), tnz = fmaf(nz, r.inv.z, r.cnz);
  float tfx = fmaf(fx, r.inv.x, r.cfx), tfy = fmaf(fy, r.inv.y, r.cfy), tfz = fmaf(fz, r.inv.z, r.cfz);
  float tn = fmax3f(tnx, tny, fmaxf(tnz, 0.0f));
  float tf = fmin3f(tfx, tfy, fminf(tfz, tmax));
  key = ANY ? -tf : tn + tf;
  return tn <= tf;
}

__host__ __device__ __forceinline__ void cswap(float& ka, int& va, float& kb, int& vb) {
  const bool s = kb < ka;
  const float tk = s ? kb : ka;
  kb = s ? ka : kb;
  ka = tk;
  const int tv = s ? vb : va;
  vb = s ? va : vb;
  va = tv;
}

// Stack traversal of the 4-wide tree (collapsed from the Karras binary
// tree), children in slab4's order.  One node fetch (7 x 16 B) tests all
// four child boxes; hit internal children are ordered by their keys with a
// 5-comparator network, the first becomes the next node and the rest are
// pushed, last first; then the node's leaf children (one triangle each) are
// tested in the same step, so the nearest-hit bound tightens before the next
// node's boxes are tested.  (Postponing leaves until the whole warp holds
// one -- the while-while form of Aila and Laine -- measured 2x slower with
// one triangle per leaf: the delayed bound lets rays wander into far
// subtrees.)
//   ANY:  any hit in (0, tmax) other than `skip`; returns true on a hit.
//   else: nearest hit in (0, inf) by (t, original index) -- independent of
//         the visiting order; prim = original index (-1 = miss), pos = sorted
//         position, tb = t.
template <class M, int STACK, bool ANY>
__host__ __device__ __forceinline__ bool traverse(const TraceCtx& c, float3 o, float3 d, float tmax, int skip,
                                                  int& prim, int& pos, float& tb) {
  prim = -1;
  pos = -1;
  tb = ANY ? tmax : inf_f();
  if (c.nt == 0) return false;
  const uint32_t n4 = (uint32_t)c.n4;
  const RaySetup r = ray_setup(o, d, c.span);
  int stack[STACK];
  stack[0] = kDone;
  int sp = 1;
  int cur = 0;  // 4-wide node, or kDone
  int budget = (int)(c.cap < (int64_t)0x7fffffff ? c.cap : (int64_t)0x7fffffff);
  while (cur != kDone) {
    if (--budget < 0) {
      M::fail(c.err, kErrTimeout);
      return false;
    }
    if ((uint32_t)cur >= n4) {  // never for a built tree
      M::fail(c.err, kErrCorrupt);
      return false;
    }
    const float4* m = &c.nodes4[cur].lox;  // lox loy loz hix hiy hiz link
    const float4 nx = M::f4(m + r.nx), ny = M::f4(m + r.ny), nz = M::f4(m + r.nz);
    const float4 fx = M::f4(m + r.fx), fy = M::f4(m + r.fy), fz = M::f4(m + r.fz);
    const int4 lk = M::i4(reinterpret_cast<const int4*>(m + 6));
    float k0, k1, k2, k3;
    int v0 = lk.x, v1 = lk.y, v2 = lk.z, v3 = lk.w;
    bool h0 = slab4<ANY>(r, nx.x, ny.x, nz.x, fx.x, fy.x, fz.x, tb, k0);
    bool h1 = slab4<ANY>(r, nx.y, ny.y, nz.y, fx.y, fy.y, fz.y, tb, k1);
    bool h2 = slab4<ANY>(r, nx.z, ny.z, nz.z, fx.z, fy.z, fz.z, tb, k2);
    bool h3 = slab4<ANY>(r, nx.w, ny.w, nz.w, fx.w, fy.w, fz.w, tb, k3);
    // hit leaves as a bit mask, tested by one loop: a warp's lanes test their
    // k-th leaf together instead of one masked test per child slot
    unsigned lm = (unsigned)(h0 && v0 < 0) | ((unsigned)(h1 && v1 < 0) << 1) | ((unsigned)(h2 && v2 < 0) << 2) |
                  ((unsigned)(h3 && v3 < 0) << 3);
    h0 = h0 && !(lm & 1u);
    h1 = h1 && !(lm & 2u);
    h2 = h2 && !(lm & 4u);
    h3 = h3 && !(lm & 8u);
    // the next node first (pop, the one entered child, or the first of the
    // ordered children with the rest pushed), then this node's leaves: the
    // lanes' different branches end before the leaf loop, and the leaf codes
    // come from the link vector (the ordering permutes v0..v3).  The visiting
    // order is the same either way; measured against leaves first: primary
    // 0.995 -> 0.946 ms, shadow 0.96 -> 0.93 ms (7.3M-triangle frame).
    int next;
    const int cnt = (int)h0 + (int)h1 + (int)h2 + (int)h3;
    if (cnt == 0) {
      next = stack[--sp];
    } else if (cnt == 1) {
      next = h0 ? v0 : h1 ? v1 : h2 ? v2 : v3;
#ifdef __CUDA_ARCH__
    } else if (!__any_sync(__activemask(), cnt > 2)) {
      // every lane here entered exactly two children: one compare-exchange
      // orders them as the network would (the same strict compare), at a
      // vote's cost (shadow pass 0.922 -> 0.912 ms on the 7.3M-triangle
      // frame); the host walk keeps the network
      const bool a01 = h0 && h1, a02 = h0 && h2, a12 = h1 && h2;
      int va = h0 ? v0 : h1 ? v1 : v2;
      float ka = h0 ? k0 : h1 ? k1 : k2;
      int vb = h3 ? v3 : (a01 ? v1 : (a02 || a12) ? v2 : v3);
      float kb = h3 ? k3 : (a01 ? k1 : (a02 || a12) ? k2 : k3);
      cswap(ka, va, kb, vb);
      if (sp + 1 <= STACK) stack[sp++] = vb;
      else M::fail(c.err, kErrStack);
      next = va;
#endif
    } else {
      // ordered by slab4's key: on the 7.3M-triangle frame 57-61 % of the
      // shadow rays are occluded, mostly by bodies between the surface and
      // the light rather than by the surface's own neighbourhood, and an
      // order toward the light reaches them sooner (farthest entry first
      // measured 1.41 -> 1.37 ms against nearest entry first, which was 9 %
      // faster than the unsorted order)
      k0 = h0 ? k0 : inf_f();
      k1 = h1 ? k1 : inf_f();
      k2 = h2 ? k2 : inf_f();
      k3 = h3 ? k3 : inf_f();
      cswap(k0, v0, k1, v1);
      cswap(k2, v2, k3, v3);
      cswap(k0, v0, k2, v2);
      cswap(k1, v1, k3, v3);
      cswap(k1, v1, k2, v2);
      if (sp + cnt - 1 <= STACK) {
        if (cnt == 4) stack[sp++] = v3;
        if (cnt >= 3) stack[sp++] = v2;
        stack[sp++] = v1;
      } else {
        M::fail(c.err, kErrStack);
      }
      next = v0;
    }
    while (lm) {
      const int slot = lowest_slot(lm);
      lm &= lm - 1;
      const int code = slot == 0 ? lk.x : slot == 1 ? lk.y : slot == 2 ? lk.z : lk.w;
      if (leaf_test<M, ANY>(c, code, o, d, tmax, skip, prim, pos, tb)) return true;
    }
    cur = next;
  }
  return false;
}

template <int STACK>
__device__ __forceinline__ void trace_nearest(const TraceCtx& c, float3 o, float3 d, int& prim, int& pos,
                                              float& tb) {
  traverse<DeviceLoads, STACK, false>(c, o, d, 0.0f, -1, prim, pos, tb);
}

template <int STACK>
__device__ __forceinline__ bool trace_any(const TraceCtx& c, float3 o, float3 d, float tmax, int skip) {
  int prim, pos;
  float tb;
  return traverse<DeviceLoads, STACK, true>(c, o, d, tmax, skip, prim, pos, tb);
}

// ---------------------------------------------------------------------------
// Smooth shading normal (§IV-A-1: the main pass shades with the meshes'
// per-vertex normals).  For the hit of the ray (o, d) on the triangle at
// sorted position pos (record A = v0, B = e1, C = e2):
//   (u, v)  barycentrics from the same FP32 triangle-test steps that found
//           the hit, so they are the traversal's own values
//   n_r     = fma(v, n2, fma(u, n1, w0 n0)) per component, w0 = (1 - u) - v,
//           from the rest normals of the triangle's three vertices
//   n_w     = R n_r, R = rotation of the vertex's body in the frame's matrices
//   n_s     = normalize(n_w), negated if n_s . n_g < 0 (n_g: the geometric
//           normal already facing the ray); a zero n_w keeps n_g
// The shadow-ray origin stays lifted along n_g (hit_frame).
// ---------------------------------------------------------------------------
struct SmoothCtx {
  const float4* vnrm;  // [nv] rest normals, or nullptr (flat)
  const float* bxf;    // [nbody*12] body matrices of the frame
  const uint4* sidx;   // [nt] sorted index records (i0, i1, i2, orig)
  const uint16_t* vbody;
};

__device__ __forceinline__ float3 shading_normal(const SmoothCtx& c, int pos, float4 A, float4 B, float4 C,
                                                 float3 o, float3 d, float3 ng) {
  const float3 v0 = xyz(A), e1 = xyz(B), e2 = xyz(C);
  const float3 p = cross3(d, e2);
  const float inv = __frcp_rn(dot3(e1, p));
  const float3 s = sub3(o, v0);
  const float u = dot3(s, p) * inv;
  const float3 q = cross3(s, e1);
  const float v = dot3(d, q) * inv;
  const uint4 id = __ldg(c.sidx + pos);
  const float4 n0 = __ldg(c.vnrm + id.x), n1 = __ldg(c.vnrm + id.y), n2 = __ldg(c.vnrm + id.z);
  const float w0 = (1.0f - u) - v;
  const float3 nr = f3(fmaf(v, n2.x, fmaf(u, n1.x, w0 * n0.x)), fmaf(v, n2.y, fmaf(u, n1.y, w0 * n0.y)),
                       fmaf(v, n2.z, fmaf(u, n1.z, w0 * n0.z)));
  const float* m = c.bxf + 12 * (uint32_t)__ldg(c.vbody + id.x);
  const float3 nw = f3(fmaf(__ldg(m + 0), nr.x, fmaf(__ldg(m + 1), nr.y, __ldg(m + 2) * nr.z)),
                       fmaf(__ldg(m + 4), nr.x, fmaf(__ldg(m + 5), nr.y, __ldg(m + 6) * nr.z)),
                       fmaf(__ldg(m + 8), nr.x, fmaf(__ldg(m + 9), nr.y, __ldg(m + 10) * nr.z)));
  if (!(dot3(nw, nw) > 0.0f)) return ng;
  const float3 ns = normalize3(nw);
  return dot3(ns, ng) < 0.0f ? neg3(ns) : ns;
}

// Scene box = union of the 4-wide root's child boxes (the same exact min/max
// as the binary root's box).
template <class M = DeviceLoads>
__host__ __device__ __forceinline__ void root_box(const Node4* nodes4, float3& lo, float3& hi) {
  const Node4* r = nodes4;
  const int4 lk = M::i4(&r->link);
  const float4 lx = M::f4(&r->lox), ly = M::f4(&r->loy), lz = M::f4(&r->loz);
  const float4 hx = M::f4(&r->hix), hy = M::f4(&r->hiy), hz = M::f4(&r->hiz);
  const int l[4] = {lk.x, lk.y, lk.z, lk.w};
  const float LX[4] = {lx.x, lx.y, lx.z, lx.w}, LY[4] = {ly.x, ly.y, ly.z, ly.w}, LZ[4] = {lz.x, lz.y, lz.z, lz.w};
  const float HX[4] = {hx.x, hx.y, hx.z, hx.w}, HY[4] = {hy.x, hy.y, hy.z, hy.w}, HZ[4] = {hz.x, hz.y, hz.z, hz.w};
  lo = f3(inf_f(), inf_f(), inf_f());
  hi = f3(-inf_f(), -inf_f(), -inf_f());
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (l[k] == kEmptyLink) continue;
    lo = f3(fminf(lo.x, LX[k]), fminf(lo.y, LY[k]), fminf(lo.z, LZ[k]));
    hi = f3(fmaxf(hi.x, HX[k]), fmaxf(hi.y, HY[k]), fmaxf(hi.z, HZ[k]));
  }
}

// Shadow-ray lift: eps = 1e-4 * |hi - lo| of the scene box.
__device__ __forceinline__ float scene_eps(const Node4* nodes4, int64_t nt) {
  if (nt == 0) return 0.0f;
  float3 lo, hi;
  root_box(nodes4, lo, hi);
  float3 ext = sub3(hi, lo);
  return 1e-4f * sqrtf(dot3(ext, ext));
}

// Largest |coordinate| of the scene box (scale of the box-test slack).
template <class M = DeviceLoads>
__host__ __device__ __forceinline__ float scene_span(const Node4* nodes4, int64_t nt) {
  if (nt == 0) return 0.0f;
  float3 lo, hi;
  root_box<M>(nodes4, lo, hi);
  return fmax3f(fmaxf(fabsf(lo.x), fabsf(hi.x)), fmaxf(fabsf(lo.y), fabsf(hi.y)), fmaxf(fabsf(lo.z), fabsf(hi.z)));
}

// ---------------------------------------------------------------------------
// §IV-B-1 BRDF, per channel, FP32 in this order:
//   h = normalize(l + v); nl, nv, nh, vh = max(dot, 0)
//   a = r*r; a2 = a*a; dd = fma(nh*nh, a2 - 1, 1); D = a2 / ((pi*dd)*dd)
//   k = ((r+1)*(r+1))*0.125; gl = fma(nl, 1-k, k); gv = fma(nv, 1-k, k)
//   vis = 0.25 / (gl*gv); Dv = D*vis; w = 1 - vh; w5 = ((w*w)*(w*w))*w
//   F0 = fma(m, albedo - 0.04, 0.04); F = fma(1 - F0, w5, F0)
//   f = ((1 - F)*(1 - m))*albedo*(1/pi) + Dv*F
// ---------------------------------------------------------------------------
__device__ __forceinline__ float3 brdf(float3 n, float3 v, float3 l, float alb_r, float alb_g, float alb_b,
                                       float r, float m) {
  float3 h = normalize3(add3(l, v));
  float nl = fmaxf(dot3(n, l), 0.0f);
  float nv = fmaxf(dot3(n, v), 0.0f);
  float nh = fmaxf(dot3(n, h), 0.0f);
  float vh = fmaxf(dot3(v, h), 0.0f);
  float a = r * r;
  float a2 = a * a;
  float dd = fmaf(nh * nh, a2 - 1.0f, 1.0f);
  float D = a2 / ((kPi * dd) * dd);
  float rp1 = r + 1.0f;
  float k = (rp1 * rp1) * 0.125f;
  float omk = 1.0f - k;
  float gl = fmaf(nl, omk, k);
  float gv = fmaf(nv, omk, k);
  float vis = 0.25f / (gl * gv);
  float Dv = D * vis;
  float w = 1.0f - vh;
  float w2 = w * w;
  float w5 = (w2 * w2) * w;
  float omm = 1.0f - m;
  float alb[3] = {alb_r, alb_g, alb_b};
  float f[3];
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) {
    float F0 = fmaf(m, alb[ch] - 0.04f, 0.04f);
    float F = fmaf(1.0f - F0, w5, F0);
    float spec = Dv * F;
    float kd = (1.0f - F) * omm;
    float diff = (kd * alb[ch]) * kInvPi;
    f[ch] = diff + spec;
  }
  return f3(f[0], f[1], f[2]);
}

// Light j seen from po: unit vector l, irradiance factor E (I / d^2 point,
// I directional), shadow-ray range tmax.
__device__ __forceinline__ void light_vec(const LightParams& L, int j, float I, float3 po, float3& l,
                                          float& E, float& tmax) {
  if (L.type[j] == 0) {
    float3 lv = sub3(f3(L.x[j], L.y[j], L.z[j]), po);
    float d2 = dot3(lv, lv);
    float dist = sqrtf(d2);
    l = f3(lv.x / dist, lv.y / dist, lv.z / dist);
    E = I / d2;
    tmax = dist;
  } else {
    l = f3(L.x[j], L.y[j], L.z[j]);
    E = I;
    tmax = inf_f();
  }
}

// Hit frame: n = normalize(e1 x e2) turned to face the ray, p = fma(t, d, o),
// po = fma(eps, n, p).
__device__ __forceinline__ void hit_frame(float4 B, float4 C, float3 o, float3 d, float t, float eps, float3& n,
                                          float3& po) {
  n = normalize3(cross3(xyz(B), xyz(C)));
  if (dot3(n, d) > 0.0f) n = neg3(n);
  float3 p = f3(fmaf(t, d.x, o.x), fmaf(t, d.y, o.y), fmaf(t, d.z, o.z));
  po = f3(fmaf(eps, n.x, p.x), fmaf(eps, n.y, p.y), fmaf(eps, n.z, p.z));
}

// Work mapping: one warp = one task of 32 samples; spp 4 -> a 4 x 2 pixel
// block x 4 samples (lanes 4q..4q+3 hold pixel q; the compact block keeps a
// warp's rays closer than 8 pixels of a row: primary 1.09 -> 1.04 ms, shadow
// 1.37 -> 1.34 ms on the 7.3M-triangle frame), spp 1 -> an 8 x 4 pixel block.
// The batch's autotuner may pick another task width (a power of two: 2, 4 or
// 8 pixels at 4 spp, 4, 8, 16 or 32 at 1 spp); lanes 4q..4q+3 always hold
// pixel q's four samples.
struct TaskGrid {
  int tiles_x, tiles_y, row_begin, rows_per_task, W, row_end, spp, lw;  // lw = log2(task width)
};

__host__ __device__ __forceinline__ TaskGrid make_grid_w(int W, int row_begin, int row_end, int spp, int lw) {
  TaskGrid g;
  g.W = W;
  g.spp = spp;
  g.row_begin = row_begin;
  g.row_end = row_end;
  g.lw = lw;
  const int px = spp == 4 ? 8 : 32;  // pixels per task
  const int tw = 1 << lw;
  g.rows_per_task = px / tw;
  g.tiles_x = (W + tw - 1) / tw;
  g.tiles_y = (row_end - row_begin + g.rows_per_task - 1) / g.rows_per_task;
  return g;
}

__host__ __device__ __forceinline__ TaskGrid make_grid(int W, int row_begin, int row_end, int spp) {
  return make_grid_w(W, row_begin, row_end, spp, spp == 4 ? 2 : 3);  // 4 x 2 or 8 x 4 pixels
}

__device__ __forceinline__ bool task_sample(const TaskGrid& g, int task, int lane, int& x, int& y, int& k) {
  const int tx = task % g.tiles_x, ty = task / g.tiles_x;
  const int q = g.spp == 4 ? lane >> 2 : lane;  // pixel of the task
  x = (tx << g.lw) + (q & ((1 << g.lw) - 1));
  y = g.row_begin + ty * g.rows_per_task + (q >> g.lw);
  k = g.spp == 4 ? lane & 3 : 0;
  return x < g.W && y < g.row_end;
}

}  // namespace fire
