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

__device__ __forceinline__ float inf_f() { return __int_as_float(0x7f800000); }

// ---------------------------------------------------------------------------
// Camera: sample k of pixel (x, y):
//   fx = x + (0.5 + ox), ndx = (2 fx)/W - 1, sx = ndx * sxs   (same for y with
//   ndy = 1 - (2 fy)/H, sy = ndy * sys); d = normalize(fma(sx, r, fma(sy, u, f)))
// 4 spp: rotated grid (-1/8,-3/8), (3/8,-1/8), (-3/8,1/8), (1/8,3/8).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float3 cam_dir(const CamParams& c, int x, int y, int k) {
  float ox = 0.0f, oy = 0.0f;
  if (c.spp == 4) {
    ox = (k == 0) ? -0.125f : (k == 1) ? 0.375f : (k == 2) ? -0.375f : 0.125f;
    oy = (k == 0) ? -0.375f : (k == 1) ? -0.125f : (k == 2) ? 0.125f : 0.375f;
  }
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
__device__ __forceinline__ float safe_rcp(float d) {
  return fabsf(d) < 1e-30f ? (d >= 0.0f ? 1e30f : -1e30f) : __frcp_rn(d);
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
//   p = d x e2, det = e1.p (reject 0), inv = 1/det, s = o - v0, u = (s.p) inv,
//   q = s x e1, v = (d.q) inv, t = (e2.q) inv; inside iff u >= 0, v >= 0,
//   fl(u + v) <= 1.  (u > 1 is rejected early: with v >= 0 it implies
//   fl(u + v) > 1, so the decision is the same.)
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool mt_t(float3 o, float3 d, float4 A, float4 B, float4 C, float& t) {
  float3 v0 = xyz(A), e1 = xyz(B), e2 = xyz(C);
  float3 p = cross3(d, e2);
  float det = dot3(e1, p);
  if (det == 0.0f) return false;
  float inv = __frcp_rn(det);
  float3 s = sub3(o, v0);
  float u = dot3(s, p) * inv;
  if (!(u >= 0.0f && u <= 1.0f)) return false;
  float3 q = cross3(s, e1);
  float v = dot3(d, q) * inv;
  if (!(v >= 0.0f && (u + v) <= 1.0f)) return false;
  t = dot3(e2, q) * inv;
  return true;
}

struct TraceCtx {
  const Node* __restrict__ nodes;
  const float4* __restrict__ tris;
  int64_t nt;
  int64_t cap;       // node-visit cap per ray (>= 1)
  uint32_t* err;     // sticky error word
};

constexpr int kDone = 0x7fffffff;  // stack sentinel: nothing left to visit

// Leaf = one triangle at sorted position ~code.  Nearest mode updates the
// (t, original index) minimum; any mode returns true on a hit in (0, tmax)
// that is not triangle `skip`.
template <bool ANY>
__device__ __forceinline__ bool leaf_test(const TraceCtx& c, int code, float3 o, float3 d, float tmax, int skip,
                                          int& prim, int& pos, float& tb) {
  int p = ~code;
  if ((uint64_t)p >= (uint64_t)c.nt) p = 0;  // never for a built tree (keeps loads in bounds)
  const float4* tr = c.tris + 3 * (int64_t)p;
  float4 A = __ldg(tr), B = __ldg(tr + 1), C = __ldg(tr + 2);
  int orig = __float_as_int(A.w);
  float t;
  if (ANY) return orig != skip && mt_t(o, d, A, B, C, t) && t > 0.0f && t < tmax;
  if (mt_t(o, d, A, B, C, t) && t > 0.0f && t < inf_f() && (t < tb || (t == tb && orig < prim))) {
    tb = t;
    prim = orig;
    pos = p;
  }
  return false;
}

// Stack traversal of the binary LBVH, nearest child first.  A leaf child
// (one triangle) is tested as soon as its box is hit, so the nearest-hit
// bound tightens early; only internal children go on the stack.
// (Postponing leaves until the whole warp holds one -- the while-while form
// of Aila and Laine -- measured 2x slower here: with one triangle per leaf the
// delayed bound lets rays wander into far subtrees.)
//   ANY:  any hit in (0, tmax) other than `skip`; returns true on a hit.
//   else: nearest hit in (0, inf) by (t, original index) -- independent of
//         the visiting order; prim = original index (-1 = miss), pos = sorted
//         position, tb = t.
template <int STACK, bool ANY>
__device__ __forceinline__ bool traverse(const TraceCtx& c, float3 o, float3 d, float tmax, int skip, int& prim,
                                         int& pos, float& tb) {
  prim = -1;
  pos = -1;
  tb = ANY ? tmax : inf_f();
  if (c.nt == 0) return false;
  const uint32_t nnodes = (uint32_t)(c.nt > 1 ? c.nt - 1 : 1);
  const float3 inv = f3(safe_rcp(d.x), safe_rcp(d.y), safe_rcp(d.z));
  int stack[STACK];
  stack[0] = kDone;
  int sp = 1;
  int cur = 0;  // internal node, or kDone
  int64_t budget = c.cap;
  while (cur != kDone) {
    if (--budget < 0) {
      atomicOr(c.err, kErrTimeout);
      return false;
    }
    if ((uint32_t)cur >= nnodes) {  // never for a built tree
      atomicOr(c.err, kErrCorrupt);
      return false;
    }
    const Node* n = c.nodes + cur;
    float4 a = __ldg(&n->a), b = __ldg(&n->b), cc = __ldg(&n->c), dq = __ldg(&n->d);
    const int2 dd = make_int2(__float_as_int(b.z), __float_as_int(dq.z));  // child links
    float tn0, tn1;
    bool h0 = slab(o, inv, a.x, a.y, a.z, a.w, b.x, b.y, tb, tn0);
    bool h1 = slab(o, inv, cc.x, cc.y, cc.z, cc.w, dq.x, dq.y, tb, tn1);
    if (h0 && dd.x < 0) {
      if (leaf_test<ANY>(c, dd.x, o, d, tmax, skip, prim, pos, tb)) return true;
      h0 = false;
    }
    if (h1 && dd.y < 0) {
      if (leaf_test<ANY>(c, dd.y, o, d, tmax, skip, prim, pos, tb)) return true;
      h1 = false;
    }
    if (h0 && h1) {
      bool first0 = tn0 <= tn1;
      if (sp < STACK) stack[sp++] = first0 ? dd.y : dd.x;
      else atomicOr(c.err, kErrStack);
      cur = first0 ? dd.x : dd.y;
    } else if (h0) {
      cur = dd.x;
    } else if (h1) {
      cur = dd.y;
    } else {
      cur = stack[--sp];
    }
  }
  return false;
}

template <int STACK>
__device__ __forceinline__ void trace_nearest(const TraceCtx& c, float3 o, float3 d, int& prim, int& pos,
                                              float& tb) {
  traverse<STACK, false>(c, o, d, 0.0f, -1, prim, pos, tb);
}

template <int STACK>
__device__ __forceinline__ bool trace_any(const TraceCtx& c, float3 o, float3 d, float tmax, int skip) {
  int prim, pos;
  float tb;
  return traverse<STACK, true>(c, o, d, tmax, skip, prim, pos, tb);
}

// Shadow-ray lift: eps = 1e-4 * |hi - lo| of the scene box (union of the
// root's two child boxes).
__device__ __forceinline__ float scene_eps(const Node* nodes, int64_t nt) {
  if (nt == 0) return 0.0f;
  float4 a = __ldg(&nodes[0].a), b = __ldg(&nodes[0].b), c = __ldg(&nodes[0].c), d = __ldg(&nodes[0].d);
  float3 lo = f3(fminf(a.x, c.x), fminf(a.y, c.y), fminf(a.z, c.z));
  float3 hi = f3(fmaxf(a.w, c.w), fmaxf(b.x, d.x), fmaxf(b.y, d.y));
  float3 ext = sub3(hi, lo);
  return 1e-4f * sqrtf(dot3(ext, ext));
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

// Work mapping: one warp = one task of 32 samples; spp 4 -> 8 pixels of a row
// x 4 samples (lanes 4q..4q+3 hold pixel q), spp 1 -> an 8 x 4 pixel block.
struct TaskGrid {
  int tiles_x, tiles_y, row_begin, rows_per_task, W, row_end, spp;
};

__host__ __device__ __forceinline__ TaskGrid make_grid(int W, int row_begin, int row_end, int spp) {
  TaskGrid g;
  g.W = W;
  g.spp = spp;
  g.row_begin = row_begin;
  g.row_end = row_end;
  g.rows_per_task = spp == 4 ? 1 : 4;
  g.tiles_x = (W + 7) / 8;
  g.tiles_y = (row_end - row_begin + g.rows_per_task - 1) / g.rows_per_task;
  return g;
}

__device__ __forceinline__ bool task_sample(const TaskGrid& g, int task, int lane, int& x, int& y, int& k) {
  int tx = task % g.tiles_x, ty = task / g.tiles_x;
  if (g.spp == 4) {
    x = tx * 8 + (lane >> 2);
    y = g.row_begin + ty;
    k = lane & 3;
  } else {
    x = tx * 8 + (lane & 7);
    y = g.row_begin + ty * 4 + (lane >> 3);
    k = 0;
  }
  return x < g.W && y < g.row_end;
}

}  // namespace fire
