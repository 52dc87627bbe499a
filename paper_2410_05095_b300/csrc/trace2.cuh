// Traversal of the two-level acceleration structure (§IV-B-3: a bottom level
// per mesh built once, a top level over the instances rebuilt every frame),
// and the hit frame of its triangles.
//
// The top level is searched with the world ray.  Reaching an entry (leaf
// link ~entry: a subtree of body b's bottom level) turns the ray into the
// body's frame,
//   o' = R^T (o - t_b),  d' = R^T d  (rows of R^T: the columns of the 3x4
//   matrix, fmaf(m0, q.x, fmaf(m4, q.y, m8 q.z)) etc.),
// pushes an exit marker and searches the entry's subtree (rest-pose
// triangle records) with it; popping the marker restores the world ray.
// Hits rank by (t of the body-frame ray, original index), and a shadow ray's
// hits count for t in (0, t_max) of the body-frame ray, the world t_max.
//
// The code is written once for the device and for the host: `M` is the
// memory policy (DeviceLoads: __ldg and atomicOr; the host emulation passes a
// policy whose every load checks that the address lies inside one of the
// arrays handed to it and is aligned for its width).  Every index is also
// checked against its array's length here, on both sides, before an address
// is formed: a failed check sets kErrCorrupt and ends the ray.
#pragma once

#include "trace_device.cuh"

namespace fire {

struct Trace2View {
  const Node4* tlas;      // top level of the frame buffer
  int64_t ntlas;
  const Node4* blas;      // bottom levels (all bodies)
  int64_t nblas;
  const float4* tris;     // rest-pose triangle records
  int64_t nt;
  const int32_t* inst;    // [2*ninst] top-level entries: (bottom-level node, body); node -1: unused
  int ninst;
  const float* xf;        // [nbody*12] the frame's body matrices (16-B aligned)
  int nbody;
  float span;             // box-test slack scale (TlasInfo::span)
  int64_t cap;            // node-visit cap per ray
  uint32_t* err;          // sticky error word
};

// o' = R^T (o - t), d' = R^T d for the row-major 3x4 matrix m.
__host__ __device__ __forceinline__ void object_ray(const float m[12], float3 o, float3 d, float3& oo, float3& dd) {
  const float3 q = sub3(o, f3(m[3], m[7], m[11]));
  oo = f3(fmaf(m[0], q.x, fmaf(m[4], q.y, m[8] * q.z)), fmaf(m[1], q.x, fmaf(m[5], q.y, m[9] * q.z)),
          fmaf(m[2], q.x, fmaf(m[6], q.y, m[10] * q.z)));
  dd = f3(fmaf(m[0], d.x, fmaf(m[4], d.y, m[8] * d.z)), fmaf(m[1], d.x, fmaf(m[5], d.y, m[9] * d.z)),
          fmaf(m[2], d.x, fmaf(m[6], d.y, m[10] * d.z)));
}

// Leaf of a bottom level: one rest-pose triangle at sorted position ~code,
// tested with the body-frame ray (the single-level leaf test's arithmetic).
template <class M, bool ANY>
__host__ __device__ __forceinline__ bool leaf_test2(const Trace2View& c, int code, float3 o, float3 d, float tmax,
                                                    int skip, int& prim, int& pos, float& tb) {
  const uint32_t p = ~(uint32_t)code;  // (a triangle link is negative: p < 2^31)
  if ((int64_t)p >= c.nt) {
    M::fail(c.err, kErrCorrupt);
    return false;
  }
  const float4* tr = c.tris + 3 * (size_t)p;
  const float4 A = M::f4(tr), B = M::f4(tr + 1), C = M::f4(tr + 2);
  const int orig = float_as_bits(A.w);
  float t;
  if (ANY) return orig != skip && mt_t(o, d, A, B, C, t) && t > 0.0f && t < tmax;
  if (mt_t(o, d, A, B, C, t) && t > 0.0f && t < inf_f() && (t < tb || (t == tb && orig < prim))) {
    tb = t;
    prim = orig;
    pos = (int)p;
  }
  return false;
}

// Stack traversal of the top level and the bottom levels it reaches (the
// single-level traversal's node step: sign-selected planes, FMA slabs,
// leaves tested at once, entered children ordered by slab4's key -- the
// middle of the span nearest first, any hit the farthest exit first).  In
// the top level every entered member, node or instance, is ordered and
// pushed; an instance is entered when it is popped.
//   ANY:  any hit in (0, tmax) other than triangle `skip`; true on a hit.
//   else: nearest hit by (t, original index): prim (-1 = miss), pos =
//         sorted position, tb = t.
template <class M, int STACK, bool ANY>
__host__ __device__ __forceinline__ bool traverse2(const Trace2View& c, float3 o, float3 d, float tmax, int skip,
                                                   int& prim, int& pos, float& tb) {
  static_assert(STACK >= 4, "stack too small");
  prim = -1;
  pos = -1;
  tb = ANY ? tmax : inf_f();
  if (c.nt == 0 || c.ntlas <= 0) return false;
  RaySetup r = ray_setup(o, d, c.span);
  float3 ro = o, rd = d;  // ray of the level being searched
  bool in_body = false;
  // nearest hit: the body whose frame ro, rd and r are in (-1: the world
  // ray), so that entering another entry of the body just left reuses its
  // ray (primary pass 1.443 -> 1.398 ms on the 7.3M-triangle frame); any
  // hit restores the world ray on every exit (the kept ray measured 1.35 ->
  // 1.39 ms there)
  int ray_body = -1;
  int stack[STACK];
  stack[0] = kDone;
  int sp = 1;
  int cur = 0;  // top-level root
  int budget = (int)(c.cap < (int64_t)0x7fffffff ? c.cap : (int64_t)0x7fffffff);
  while (cur != kDone) {
    if (--budget < 0) {
      M::fail(c.err, kErrTimeout);
      return false;
    }
    if (cur == kExitInstance) {  // leave the subtree
      in_body = false;
      if (ANY) {  // back to the world ray (nearest hit: when the top level needs it)
        ro = o;
        rd = d;
        r = ray_setup(o, d, c.span);
      }
      cur = stack[--sp];
      continue;
    }
    if (!in_body && cur < 0) {  // enter top-level entry ~cur: a subtree of body b's bottom level
      const int e = ~cur;
      if (e < 0 || e >= c.ninst) {
        M::fail(c.err, kErrCorrupt);
        return false;
      }
      const int root = M::i1(c.inst + 2 * e), b = M::i1(c.inst + 2 * e + 1);
      if (root < 0) {  // an unused entry (never entered: it has no box)
        cur = stack[--sp];
        continue;
      }
      if (root >= c.nblas || b < 0 || b >= c.nbody) {
        M::fail(c.err, kErrCorrupt);
        return false;
      }
      if (sp >= STACK) {  // no room for the exit marker: the instance is skipped
        M::fail(c.err, kErrStack);
        cur = stack[--sp];
        continue;
      }
      if (ANY || b != ray_body) {
        // the body's matrix: three 16-B rows (48 B per body from a 16-B aligned base)
        const float4* mx = reinterpret_cast<const float4*>(c.xf) + 3 * (int64_t)b;
        const float4 m0 = M::f4(mx), m1 = M::f4(mx + 1), m2 = M::f4(mx + 2);
        const float m[12] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w, m2.x, m2.y, m2.z, m2.w};
        object_ray(m, o, d, ro, rd);
        r = ray_setup(ro, rd, c.span);
        ray_body = b;
      }
      stack[sp++] = kExitInstance;
      in_body = true;
      cur = root;
      continue;
    }
    if (!ANY && !in_body && ray_body >= 0) {  // a top-level node: back to the world ray
      ro = o;
      rd = d;
      r = ray_setup(o, d, c.span);
      ray_body = -1;
    }
    const Node4* base = in_body ? c.blas : c.tlas;
    const uint32_t nn = (uint32_t)(in_body ? c.nblas : c.ntlas);  // (node counts < 2^31)
    if ((uint32_t)cur >= nn) {
      M::fail(c.err, kErrCorrupt);
      return false;
    }
    const float4* m = &base[cur].lox;  // lox loy loz hix hiy hiz link
    const float4 nx = M::f4(m + r.nx), ny = M::f4(m + r.ny), nz = M::f4(m + r.nz);
    const float4 fx = M::f4(m + r.fx), fy = M::f4(m + r.fy), fz = M::f4(m + r.fz);
    const int4 lk = M::i4(reinterpret_cast<const int4*>(m + 6));
    float k0, k1, k2, k3;
    int v0 = lk.x, v1 = lk.y, v2 = lk.z, v3 = lk.w;
    bool h0 = slab4<ANY>(r, nx.x, ny.x, nz.x, fx.x, fy.x, fz.x, tb, k0);
    bool h1 = slab4<ANY>(r, nx.y, ny.y, nz.y, fx.y, fy.y, fz.y, tb, k1);
    bool h2 = slab4<ANY>(r, nx.z, ny.z, nz.z, fx.z, fy.z, fz.z, tb, k2);
    bool h3 = slab4<ANY>(r, nx.w, ny.w, nz.w, fx.w, fy.w, fz.w, tb, k3);
    unsigned lm = 0;  // triangle leaves of a bottom-level node
    if (in_body) {
      lm = (unsigned)(h0 && v0 < 0) | ((unsigned)(h1 && v1 < 0) << 1) | ((unsigned)(h2 && v2 < 0) << 2) |
           ((unsigned)(h3 && v3 < 0) << 3);
      h0 = h0 && !(lm & 1u);
      h1 = h1 && !(lm & 2u);
      h2 = h2 && !(lm & 4u);
      h3 = h3 && !(lm & 8u);
    } else {
      // an unused slot holds the inverted infinite box and is never entered;
      // a link of kEmptyLink that passes anyway would be a corrupt node
      if ((h0 && v0 == kEmptyLink) || (h1 && v1 == kEmptyLink) || (h2 && v2 == kEmptyLink) ||
          (h3 && v3 == kEmptyLink)) {
        M::fail(c.err, kErrCorrupt);
        return false;
      }
    }
    // the next entry first, then this node's leaves (the single-level
    // traversal's step order; leaf codes from the link vector)
    int next;
    const int cnt = (int)h0 + (int)h1 + (int)h2 + (int)h3;
    if (cnt == 0) {
      next = stack[--sp];
    } else if (cnt == 1) {
      next = h0 ? v0 : h1 ? v1 : h2 ? v2 : v3;
#ifdef __CUDA_ARCH__
    } else if (!__any_sync(__activemask(), cnt > 2)) {  // two children: one compare-exchange
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
      if (leaf_test2<M, ANY>(c, code, ro, rd, tmax, skip, prim, pos, tb)) return true;
    }
    cur = next;
  }
  return false;
}

// Hit frame of a two-level hit: the rest-pose normal e1 x e2 turned by the
// rows of the body's rotation, n = normalize(R (e1 x e2)), facing the ray;
// p = fma(t, d, o) on the world ray, po = fma(eps, n, p).
__host__ __device__ __forceinline__ void hit_frame2(float4 B, float4 C, const float m[12], float3 o, float3 d,
                                                    float t, float eps, float3& n, float3& po) {
  const float3 cr = cross3(xyz(B), xyz(C));
  n = normalize3(f3(fmaf(m[0], cr.x, fmaf(m[1], cr.y, m[2] * cr.z)), fmaf(m[4], cr.x, fmaf(m[5], cr.y, m[6] * cr.z)),
                    fmaf(m[8], cr.x, fmaf(m[9], cr.y, m[10] * cr.z))));
  if (dot3(n, d) > 0.0f) n = neg3(n);
  const float3 p = f3(fmaf(t, d.x, o.x), fmaf(t, d.y, o.y), fmaf(t, d.z, o.z));
  po = f3(fmaf(eps, n.x, p.x), fmaf(eps, n.y, p.y), fmaf(eps, n.z, p.z));
}

}  // namespace fire
