// CPU oracle for the renderer hot path -- TEST INFRASTRUCTURE ONLY.
//
// Plain single-threaded C++17, compiled with -O2 -ffp-contract=off so that no
// multiply-add is fused unless written as std::fmaf.  Only tests/, the smoke
// check and the benchmark's CPU-baseline leg load it.  It shares no code,
// header or constant with the CUDA library; both restate the same definitions
// (listed per function below) independently.
//
// Precision: the plain method is FP32 (every workload of this build is FP32),
// and integer decisions taken from floats (Morton codes, nearest-hit argmin,
// shadow visibility) are taken in FP32 on both sides.  The operation order of
// each FP32 expression is fixed here and documented; the gradient checks use
// the FP64 twin at the end of the file.
//
// Parity unpinned: tree quality (node visits per ray) is reported, not pinned.
#include "fire_oracle.h"

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <numeric>
#include <vector>

namespace {

// float(pi) and float(1/pi), nearest floats.
const float kPiF = 3.14159265358979323846f;
const float kInvPiF = 0.318309886183790671538f;
const double kPiD = 3.14159265358979323846;
const float kInfF = std::numeric_limits<float>::infinity();

struct V3 { float x, y, z; };
static inline V3 mk(float x, float y, float z) { V3 r = {x, y, z}; return r; }
static inline V3 sub3(V3 a, V3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
static inline V3 add3(V3 a, V3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
static inline V3 neg3(V3 a) { return mk(-a.x, -a.y, -a.z); }
// dot(a,b) = fma(ax,bx, fma(ay,by, az*bz))
static inline float dot3(V3 a, V3 b) { return std::fmaf(a.x, b.x, std::fmaf(a.y, b.y, a.z * b.z)); }
// cross(a,b).x = fma(ay,bz, -(az*by)), cyclic
static inline V3 cross3(V3 a, V3 b) {
  return mk(std::fmaf(a.y, b.z, -(a.z * b.y)), std::fmaf(a.z, b.x, -(a.x * b.z)),
            std::fmaf(a.x, b.y, -(a.y * b.x)));
}
// normalize(v) = v / sqrt(dot(v,v)), three correctly rounded divisions
static inline V3 normalize3(V3 v) {
  float len = std::sqrt(dot3(v, v));
  return mk(v.x / len, v.y / len, v.z / len);
}

struct D3 { double x, y, z; };
static inline D3 dk(double x, double y, double z) { D3 r = {x, y, z}; return r; }
static inline D3 dsub(D3 a, D3 b) { return dk(a.x - b.x, a.y - b.y, a.z - b.z); }
static inline double ddot(D3 a, D3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static inline D3 dcross(D3 a, D3 b) {
  return dk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
static inline D3 dnorm(D3 v) { double l = std::sqrt(ddot(v, v)); return dk(v.x / l, v.y / l, v.z / l); }
static inline D3 tod(V3 v) { return dk(v.x, v.y, v.z); }

struct Box { float lo[3], hi[3]; };

}  // namespace

struct orc_scene {
  int64_t nv = 0, nt = 0;
  int32_t nmat = 0, nbody = 0;
  std::vector<float> rest;        // [nv*4]
  std::vector<uint32_t> idx;      // [nt*3]
  std::vector<uint32_t> tri_mat;  // [nt]
  std::vector<uint16_t> vbody;    // [nv]
  std::vector<orc_material> mats;
  // per-frame state
  std::vector<V3> world;          // [nv]
  bool built = false;
  std::vector<uint64_t> morton;   // by original triangle
  std::vector<uint32_t> order;    // sorted position -> original triangle
  std::vector<int32_t> child;     // [(nt-1)*2] Karras codes
  std::vector<int32_t> parent;    // [2nt-1]
  std::vector<Box> box;           // [2nt-1] by Karras code
  float cb[6] = {0, 0, 0, 0, 0, 0};  // centroid bounds
  Box scene_box;
  // two-level mode (see the two-level section below)
  bool two_level = false;
  std::vector<float> xf;              // [nbody*12] transforms of the last update
  struct BNode { Box box; int32_t left = -1, right = -1, first = 0, count = 0; };
  struct Body { std::vector<BNode> nodes; std::vector<int32_t> tris; Box rest_box; };
  std::vector<Body> bodies;           // rest-space BVH per body
  std::vector<Box> inst_box;          // world box per body (empty bodies: unused)
  Box inst_union;
  // smooth shading: rest-pose vertex normals [nv*4] (xyz; empty = flat)
  std::vector<float> vnrm;
};

namespace {

// ---------------------------------------------------------------------------
// §IV-C / §IV-B-3 step (4): per-body rigid transform of the rest vertices.
// x' = fma(m0,x, fma(m1,y, fma(m2,z, m3))) per row of the 3x4 matrix.
// ---------------------------------------------------------------------------
void transform(orc_scene& S, const float* xf) {
  S.world.resize(S.nv);
  for (int64_t i = 0; i < S.nv; ++i) {
    const float* m = xf + 12 * (int64_t)S.vbody[i];
    float x = S.rest[4 * i], y = S.rest[4 * i + 1], z = S.rest[4 * i + 2];
    S.world[i] = mk(std::fmaf(m[0], x, std::fmaf(m[1], y, std::fmaf(m[2], z, m[3]))),
                    std::fmaf(m[4], x, std::fmaf(m[5], y, std::fmaf(m[6], z, m[7]))),
                    std::fmaf(m[8], x, std::fmaf(m[9], y, std::fmaf(m[10], z, m[11]))));
  }
}

inline void tri_verts(const orc_scene& S, int64_t t, V3& a, V3& b, V3& c) {
  a = S.world[S.idx[3 * t]];
  b = S.world[S.idx[3 * t + 1]];
  c = S.world[S.idx[3 * t + 2]];
}

Box tri_box(const orc_scene& S, int64_t t) {
  V3 a, b, c;
  tri_verts(S, t, a, b, c);
  Box r;
  const float A[3] = {a.x, a.y, a.z}, B[3] = {b.x, b.y, b.z}, C[3] = {c.x, c.y, c.z};
  for (int k = 0; k < 3; ++k) {
    r.lo[k] = std::min(A[k], std::min(B[k], C[k]));
    r.hi[k] = std::max(A[k], std::max(B[k], C[k]));
  }
  return r;
}

Box box_union(const Box& a, const Box& b) {
  Box r;
  for (int k = 0; k < 3; ++k) {
    r.lo[k] = std::min(a.lo[k], b.lo[k]);
    r.hi[k] = std::max(a.hi[k], b.hi[k]);
  }
  return r;
}

// ---------------------------------------------------------------------------
// Morton code of a centroid with m bits per axis:
//   q_a = min(floor((c_a - lo_a) * s_a), 2^m - 1), s_a = 2^m / (hi_a - lo_a)
//   (0 if hi_a == lo_a); bit k of q_x -> bit 3k+2, of q_y -> 3k+1, of q_z -> 3k.
// Written as a plain per-bit loop.
// Body field (scenes of several rigid bodies, §IV-C: each body moves as a
// whole), with B = bits of (nbody - 1), m = min(21, (63 - B) / 3) and the
// body of the triangle's first vertex:
//   key = coarse << (B + 3(m-c)) | body << 3(m-c) | fine
// where coarse = the code's top 3c bits (the top c bits of each q_a) and fine
// = its low 3(m-c) bits.  Inside each coarse cell (1/2^c of the bounds per
// axis) a body's triangles are consecutive in the sorted order and form one
// subtree, so only the nodes of the coarse levels mix bodies, like the
// paper's per-mesh bottom levels under a top level (§IV-B-3).  c = 4 for the
// single-level tree; c = 0 (the body above everything: one subtree per body)
// for the bottom levels of the two-level mode.  One body: B = 0, m = 21, and
// the key is the plain Morton code.
// ---------------------------------------------------------------------------
uint32_t quantise(float c, float lo, float s, uint32_t qmax) {
  float f = (c - lo) * s;
  if (!(f > 0.0f)) return 0u;
  if (f >= (float)qmax) return qmax;
  return (uint32_t)f;
}

uint64_t interleave(uint32_t qx, uint32_t qy, uint32_t qz, int m) {
  uint64_t code = 0;
  for (int k = 0; k < m; ++k) {
    code |= (uint64_t)((qx >> k) & 1u) << (3 * k + 2);
    code |= (uint64_t)((qy >> k) & 1u) << (3 * k + 1);
    code |= (uint64_t)((qz >> k) & 1u) << (3 * k);
  }
  return code;
}

// Bits of the body field and Morton bits per axis for a scene of nbody bodies.
void key_layout(int32_t nbody, int& B, int& m) {
  B = 0;
  while (nbody > 1 && (1 << B) < nbody) ++B;
  m = std::min(21, (63 - B) / 3);
}

constexpr int kCoarseBits = 4;  // c of the single-level tree

uint64_t body_key(uint64_t code, uint64_t body, int B, int m, int c) {
  const int fine = 3 * (m - c);
  const uint64_t low = fine > 0 ? code & ((1ull << fine) - 1) : 0;
  return ((code >> fine) << (B + fine)) | (body << fine) | low;
}

int clz64(uint64_t x) { int n = 0; for (int b = 63; b >= 0 && !((x >> b) & 1u); --b) ++n; return n; }
int clz32(uint32_t x) { int n = 0; for (int b = 31; b >= 0 && !((x >> b) & 1u); --b) ++n; return n; }

// Length of the common prefix of sorted keys i and j, keys augmented with
// their position when equal (Karras 2012).
int delta(const std::vector<uint64_t>& k, int64_t i, int64_t j) {
  if (k[i] != k[j]) return clz64(k[i] ^ k[j]);
  return 64 + clz32((uint32_t)i ^ (uint32_t)j);
}

// Top-down construction of the same radix tree the parallel Karras build
// produces: a range [first, last] is split after the last position that
// still shares more than delta(first, last) prefix bits with `first`
// (binary search); the child covering [first, split] is numbered `split`,
// the one covering [split+1, last] is numbered `split+1`; one-element ranges
// are leaves (code T-1+position).
void build_range(orc_scene& S, const std::vector<uint64_t>& k, int32_t node, int64_t first,
                 int64_t last) {
  const int64_t T = S.nt;
  int common = delta(k, first, last);
  int64_t lo = first, hi = last - 1;  // invariant: answer in [lo, hi], delta(first, lo) > common or lo==first
  while (lo < hi) {
    int64_t mid = (lo + hi + 1) / 2;
    if (delta(k, first, mid) > common) lo = mid; else hi = mid - 1;
  }
  int64_t split = lo;
  int32_t left = (split == first) ? (int32_t)(T - 1 + split) : (int32_t)split;
  int32_t right = (split + 1 == last) ? (int32_t)(T - 1 + split + 1) : (int32_t)(split + 1);
  S.child[2 * node] = left;
  S.child[2 * node + 1] = right;
  S.parent[left] = node;
  S.parent[right] = node;
  if (split != first) build_range(S, k, (int32_t)split, first, split);
  if (split + 1 != last) build_range(S, k, (int32_t)(split + 1), split + 1, last);
}

Box refit_node(orc_scene& S, int32_t code) {
  const int64_t T = S.nt;
  if (code >= T - 1) {
    S.box[code] = tri_box(S, S.order[code - (T - 1)]);
  } else {
    Box a = refit_node(S, S.child[2 * code]);
    Box b = refit_node(S, S.child[2 * code + 1]);
    S.box[code] = box_union(a, b);
  }
  return S.box[code];
}

void build(orc_scene& S) {
  const int64_t T = S.nt;
  S.morton.assign(T, 0);
  S.order.resize(T);
  S.child.assign(T > 1 ? 2 * (T - 1) : 0, -1);
  S.parent.assign(T > 0 ? 2 * T - 1 : 0, -1);
  S.box.resize(T > 0 ? 2 * T - 1 : 0);
  if (T == 0) { S.built = true; return; }
  std::vector<float> cen(3 * T);
  float lo[3] = {kInfF, kInfF, kInfF}, hi[3] = {-kInfF, -kInfF, -kInfF};
  for (int64_t t = 0; t < T; ++t) {
    Box b = tri_box(S, t);
    for (int a = 0; a < 3; ++a) {
      float c = 0.5f * (b.lo[a] + b.hi[a]);
      cen[3 * t + a] = c;
      lo[a] = std::min(lo[a], c);
      hi[a] = std::max(hi[a], c);
    }
  }
  int B, m;
  key_layout(S.nbody, B, m);
  const float cells = (float)(1u << m);
  const uint32_t qmax = (1u << m) - 1u;
  float s[3];
  for (int a = 0; a < 3; ++a) {
    s[a] = (hi[a] > lo[a]) ? cells / (hi[a] - lo[a]) : 0.0f;
    S.cb[a] = lo[a];
    S.cb[3 + a] = hi[a];
  }
  for (int64_t t = 0; t < T; ++t) {
    const uint64_t body = B > 0 ? (uint64_t)S.vbody[S.idx[3 * t]] : 0u;
    const uint64_t code =
        interleave(quantise(cen[3 * t], lo[0], s[0], qmax), quantise(cen[3 * t + 1], lo[1], s[1], qmax),
                   quantise(cen[3 * t + 2], lo[2], s[2], qmax), m);
    S.morton[t] = B > 0 ? body_key(code, body, B, m, kCoarseBits) : code;
  }
  std::iota(S.order.begin(), S.order.end(), 0u);
  std::stable_sort(S.order.begin(), S.order.end(),
                   [&](uint32_t a, uint32_t b) { return S.morton[a] < S.morton[b]; });
  std::vector<uint64_t> k(T);
  for (int64_t i = 0; i < T; ++i) k[i] = S.morton[S.order[i]];
  if (T > 1) build_range(S, k, 0, 0, T - 1);
  S.built = true;
}

void refit_all(orc_scene& S) {
  const int64_t T = S.nt;
  if (T == 0) return;
  Box root = refit_node(S, 0);  // T == 1: code 0 is leaf 0
  S.scene_box = root;
}

// ---------------------------------------------------------------------------
// Ray/triangle test (Moller-Trumbore) with the fixed FP32 operation order.
// ---------------------------------------------------------------------------
bool mt_hit(V3 o, V3 d, V3 v0, V3 v1, V3 v2, float& t, float& u, float& v) {
  V3 e1 = sub3(v1, v0), e2 = sub3(v2, v0);
  V3 p = cross3(d, e2);
  float det = dot3(e1, p);
  if (det == 0.0f) return false;
  float inv = 1.0f / det;
  V3 s = sub3(o, v0);
  u = dot3(s, p) * inv;
  V3 q = cross3(s, e1);
  v = dot3(d, q) * inv;
  t = dot3(e2, q) * inv;
  return u >= 0.0f && v >= 0.0f && (u + v) <= 1.0f;
}

struct Hit {
  int32_t prim = -1;
  float t = kInfF, u = 0, v = 0;
  int32_t prim2 = -1;
  float t2 = kInfF;
};

// Lexicographic (t, original index) order: equal t -> smaller index wins.
// Only finite t reach here, so "no hit yet" (t = inf) always loses.
inline bool better(float t, int32_t i, float tb, int32_t ib) {
  return t < tb || (t == tb && i < ib);
}

void consider(Hit& h, int32_t tri, float t, float u, float v) {
  if (better(t, tri, h.t, h.prim)) {
    h.t2 = h.t; h.prim2 = h.prim;
    h.t = t; h.u = u; h.v = v; h.prim = tri;
  } else if (tri != h.prim && better(t, tri, h.t2, h.prim2)) {
    h.t2 = t; h.prim2 = tri;
  }
}

// Conservative box test in double: box inflated by an absolute margin and
// the ray interval by a relative one, so that it never rejects a box whose
// triangles the FP32 triangle test would accept (the traversal must equal
// brute force; a few extra visits do not matter here).
bool box_hit(const Box& b, V3 o, V3 d, double tmin, double tmax, double& tnear) {
  const double O[3] = {o.x, o.y, o.z}, Dd[3] = {d.x, d.y, d.z};
  double t0 = tmin, t1 = tmax * (1.0 + 1e-3) + 1e-6;
  for (int a = 0; a < 3; ++a) {
    double m = 1e-4 * (1.0 + std::fabs((double)b.lo[a]) + std::fabs((double)b.hi[a]));
    double lo = (double)b.lo[a] - m, hi = (double)b.hi[a] + m;
    if (Dd[a] == 0.0) {
      if (O[a] < lo || O[a] > hi) return false;
      continue;
    }
    double ta = (lo - O[a]) / Dd[a], tb = (hi - O[a]) / Dd[a];
    if (ta > tb) std::swap(ta, tb);
    t0 = std::max(t0, ta);
    t1 = std::min(t1, tb);
  }
  tnear = t0;
  return t0 <= t1;
}

// Karras code 0 is the root: internal node 0, or leaf 0 when T == 1.
int32_t root_code(const orc_scene&) { return 0; }
inline bool is_leaf(const orc_scene& S, int32_t code) { return code >= S.nt - 1; }

void trace_bvh(const orc_scene& S, V3 o, V3 d, float tmin, Hit& h, bool want2) {
  std::vector<int32_t> stack;
  stack.push_back(root_code(S));
  while (!stack.empty()) {
    int32_t code = stack.back();
    stack.pop_back();
    double bound = want2 ? (double)h.t2 : (double)h.t;
    double tn;
    if (!box_hit(S.box[code], o, d, tmin, bound, tn)) continue;
    if (is_leaf(S, code)) {
      int32_t tri = (int32_t)S.order[code - (S.nt - 1)];
      V3 a, b, c;
      tri_verts(S, tri, a, b, c);
      float t, u, v;
      if (mt_hit(o, d, a, b, c, t, u, v) && t > tmin && t < kInfF) consider(h, tri, t, u, v);
    } else {
      stack.push_back(S.child[2 * code + 1]);
      stack.push_back(S.child[2 * code]);
    }
  }
}

void trace_brute(const orc_scene& S, V3 o, V3 d, float tmin, Hit& h) {
  for (int64_t tri = 0; tri < S.nt; ++tri) {
    V3 a, b, c;
    tri_verts(S, tri, a, b, c);
    float t, u, v;
    if (mt_hit(o, d, a, b, c, t, u, v) && t > tmin && t < kInfF) consider(h, (int32_t)tri, t, u, v);
  }
}

// ---------------------------------------------------------------------------
// Two-level mode (§IV-B-3: one bottom-level structure per mesh in its own
// frame, built once; a top level over the instances rebuilt every frame).
// Here a body is an instance: its triangles stay in rest coordinates and a
// ray meets them in the body's frame.  For the body matrix M = [R | t]
// (rows m0..m11, rigid) the object-space ray is
//   q = o - t;  o'_c = fma(R_0c, q.x, fma(R_1c, q.y, R_2c * q.z)),
//   d'_c = the same with d               (R^T applied: columns of R)
// and the Moller-Trumbore test runs on the rest triangle with (o', d'); its
// t ranks hits across bodies with the usual (t, original index) order.  The
// hit normal is normalize(R cross(e1', e2')) (rows of R), turned to face the
// ray; the hit point is fma(t, d, o) of the world ray.  The shadow-ray
// epsilon uses the union of the bodies' world boxes, each the min/max of the
// 8 transformed corners of the body's rest box.  Each body's triangles must
// share the body of their vertices.  The per-body trees here are plain
// median splits (any conservative tree gives the brute-force result).
// ---------------------------------------------------------------------------
inline V3 rest_v(const orc_scene& S, uint32_t i) { return mk(S.rest[4 * i], S.rest[4 * i + 1], S.rest[4 * i + 2]); }

Box rest_tri_box(const orc_scene& S, int32_t t) {
  V3 a = rest_v(S, S.idx[3 * t]), b = rest_v(S, S.idx[3 * t + 1]), c = rest_v(S, S.idx[3 * t + 2]);
  Box r;
  const float A[3] = {a.x, a.y, a.z}, B[3] = {b.x, b.y, b.z}, C[3] = {c.x, c.y, c.z};
  for (int k = 0; k < 3; ++k) {
    r.lo[k] = std::min(A[k], std::min(B[k], C[k]));
    r.hi[k] = std::max(A[k], std::max(B[k], C[k]));
  }
  return r;
}

int32_t body_build(const orc_scene& S, orc_scene::Body& B, int32_t first, int32_t count) {
  orc_scene::BNode nd;
  nd.box = rest_tri_box(S, B.tris[first]);
  for (int32_t i = 1; i < count; ++i) nd.box = box_union(nd.box, rest_tri_box(S, B.tris[first + i]));
  const int32_t me = (int32_t)B.nodes.size();
  B.nodes.push_back(nd);
  if (count <= 4) {
    B.nodes[me].first = first;
    B.nodes[me].count = count;
    return me;
  }
  int axis = 0;
  float ext = -1.0f;
  for (int k = 0; k < 3; ++k)
    if (nd.box.hi[k] - nd.box.lo[k] > ext) { ext = nd.box.hi[k] - nd.box.lo[k]; axis = k; }
  auto cen = [&](int32_t t) { Box b = rest_tri_box(S, t); return b.lo[axis] + b.hi[axis]; };
  const int32_t half = count / 2;
  std::nth_element(B.tris.begin() + first, B.tris.begin() + first + half, B.tris.begin() + first + count,
                   [&](int32_t a, int32_t b) { return cen(a) < cen(b) || (cen(a) == cen(b) && a < b); });
  const int32_t l = body_build(S, B, first, half);
  const int32_t r = body_build(S, B, first + half, count - half);
  B.nodes[me].left = l;
  B.nodes[me].right = r;
  return me;
}

bool set_two_level(orc_scene& S) {
  for (int64_t t = 0; t < S.nt; ++t) {
    const uint16_t b = S.vbody[S.idx[3 * t]];
    if (S.vbody[S.idx[3 * t + 1]] != b || S.vbody[S.idx[3 * t + 2]] != b) return false;
  }
  S.bodies.assign(S.nbody, orc_scene::Body());
  for (int64_t t = 0; t < S.nt; ++t) S.bodies[S.vbody[S.idx[3 * t]]].tris.push_back((int32_t)t);
  for (auto& B : S.bodies) {
    if (B.tris.empty()) continue;
    body_build(S, B, 0, (int32_t)B.tris.size());
    B.rest_box = B.nodes[0].box;
  }
  S.two_level = true;
  return true;
}

V3 xf_point(const float* m, V3 p) {
  return mk(std::fmaf(m[0], p.x, std::fmaf(m[1], p.y, std::fmaf(m[2], p.z, m[3]))),
            std::fmaf(m[4], p.x, std::fmaf(m[5], p.y, std::fmaf(m[6], p.z, m[7]))),
            std::fmaf(m[8], p.x, std::fmaf(m[9], p.y, std::fmaf(m[10], p.z, m[11]))));
}

void instance_boxes(orc_scene& S) {
  S.inst_box.assign(S.nbody, Box());
  bool any = false;
  for (int b = 0; b < S.nbody; ++b) {
    const auto& B = S.bodies[b];
    if (B.tris.empty()) continue;
    const float* m = S.xf.data() + 12 * b;
    Box w;
    for (int c = 0; c < 8; ++c) {
      V3 p = xf_point(m, mk((c & 1) ? B.rest_box.hi[0] : B.rest_box.lo[0], (c & 2) ? B.rest_box.hi[1] : B.rest_box.lo[1],
                            (c & 4) ? B.rest_box.hi[2] : B.rest_box.lo[2]));
      const float P[3] = {p.x, p.y, p.z};
      for (int k = 0; k < 3; ++k) {
        w.lo[k] = c ? std::min(w.lo[k], P[k]) : P[k];
        w.hi[k] = c ? std::max(w.hi[k], P[k]) : P[k];
      }
    }
    S.inst_box[b] = w;
    S.inst_union = any ? box_union(S.inst_union, w) : w;
    any = true;
  }
}

void object_ray(const float* m, V3 o, V3 d, V3& oo, V3& dd) {
  V3 q = sub3(o, mk(m[3], m[7], m[11]));
  oo = mk(std::fmaf(m[0], q.x, std::fmaf(m[4], q.y, m[8] * q.z)),
          std::fmaf(m[1], q.x, std::fmaf(m[5], q.y, m[9] * q.z)),
          std::fmaf(m[2], q.x, std::fmaf(m[6], q.y, m[10] * q.z)));
  dd = mk(std::fmaf(m[0], d.x, std::fmaf(m[4], d.y, m[8] * d.z)),
          std::fmaf(m[1], d.x, std::fmaf(m[5], d.y, m[9] * d.z)),
          std::fmaf(m[2], d.x, std::fmaf(m[6], d.y, m[10] * d.z)));
}

// Nearest hit (any = false) or any hit in (0, tmax) other than `skip` in
// body b's frame; bvh = false tests every triangle of the body.
bool body_trace(const orc_scene& S, int b, V3 o, V3 d, float tmin, float tmax, int32_t skip, bool any,
                bool bvh, bool want2, Hit& h) {
  const auto& B = S.bodies[b];
  if (B.tris.empty()) return false;
  V3 oo, dd;
  object_ray(S.xf.data() + 12 * b, o, d, oo, dd);
  auto test = [&](int32_t tri) {
    if (tri == skip) return false;
    float t, u, v;
    V3 a = rest_v(S, S.idx[3 * tri]), bb = rest_v(S, S.idx[3 * tri + 1]), c = rest_v(S, S.idx[3 * tri + 2]);
    if (!(mt_hit(oo, dd, a, bb, c, t, u, v) && t > tmin && t < tmax)) return false;
    if (any) return true;
    consider(h, tri, t, u, v);
    return false;
  };
  if (!bvh) {
    for (int32_t tri : B.tris) if (test(tri)) return true;
    return false;
  }
  std::vector<int32_t> stack(1, 0);
  while (!stack.empty()) {
    const auto& nd = B.nodes[stack.back()];
    stack.pop_back();
    double bound = any ? (double)tmax : (want2 ? (double)h.t2 : (double)h.t);
    double tn;
    if (!box_hit(nd.box, oo, dd, tmin, bound, tn)) continue;
    if (nd.left < 0) {
      for (int32_t i = 0; i < nd.count; ++i) if (test(B.tris[nd.first + i])) return true;
    } else {
      stack.push_back(nd.right);
      stack.push_back(nd.left);
    }
  }
  return false;
}

Hit trace(const orc_scene& S, V3 o, V3 d, float tmin, bool bvh, bool want2) {
  Hit h;
  if (S.nt == 0) return h;
  if (S.two_level) {
    for (int b = 0; b < S.nbody; ++b) body_trace(S, b, o, d, tmin, kInfF, -1, false, bvh, want2, h);
    return h;
  }
  if (bvh) trace_bvh(S, o, d, tmin, h, want2); else trace_brute(S, o, d, tmin, h);
  return h;
}

// Any hit with 0 < t < tmax, skipping triangle `skip`.
bool occluded(const orc_scene& S, V3 o, V3 d, float tmax, int32_t skip, bool bvh) {
  if (S.nt == 0) return false;
  if (S.two_level) {
    Hit unused;
    for (int b = 0; b < S.nbody; ++b)
      if (body_trace(S, b, o, d, 0.0f, tmax, skip, true, bvh, false, unused)) return true;
    return false;
  }
  auto test = [&](int64_t tri) {
    if ((int32_t)tri == skip) return false;
    V3 a, b, c;
    tri_verts(S, tri, a, b, c);
    float t, u, v;
    return mt_hit(o, d, a, b, c, t, u, v) && t > 0.0f && t < tmax;
  };
  if (!bvh) {
    for (int64_t tri = 0; tri < S.nt; ++tri) if (test(tri)) return true;
    return false;
  }
  std::vector<int32_t> stack;
  stack.push_back(root_code(S));
  while (!stack.empty()) {
    int32_t code = stack.back();
    stack.pop_back();
    double tn;
    if (!box_hit(S.box[code], o, d, 0.0, (double)tmax, tn)) continue;
    if (is_leaf(S, code)) {
      if (test(S.order[code - (S.nt - 1)])) return true;
    } else {
      stack.push_back(S.child[2 * code + 1]);
      stack.push_back(S.child[2 * code]);
    }
  }
  return false;
}

// ---------------------------------------------------------------------------
// Camera (§IV-A-1 view transform restated as a pinhole ray generator):
// f = normalize(target - pos), r = normalize(cross(f, up)), u = cross(r, f);
// sy_scale = float(tan(vfov/2)) (double tan, rounded), sx_scale = sy_scale *
// (W / H); sample k of pixel (x, y) has offset (ox, oy) on the 4-sample
// rotated grid (or the pixel centre at 1 spp):
//   fx = x + (0.5 + ox);  ndx = (2 fx) / W - 1;  sx = ndx * sx_scale
//   fy = y + (0.5 + oy);  ndy = 1 - (2 fy) / H;  sy = ndy * sy_scale
//   d = normalize(fma(sx, r, fma(sy, u, f)))   (componentwise)
// ---------------------------------------------------------------------------
struct Cam { V3 o, f, r, u; float sxs, sys; int W, H, spp; };

const float kGrid4[4][2] = {{-0.125f, -0.375f}, {0.375f, -0.125f}, {-0.375f, 0.125f}, {0.125f, 0.375f}};

Cam make_cam(const orc_camera* c) {
  Cam k;
  V3 pos = mk(c->pos[0], c->pos[1], c->pos[2]);
  V3 tgt = mk(c->target[0], c->target[1], c->target[2]);
  V3 up = mk(c->up[0], c->up[1], c->up[2]);
  k.o = pos;
  k.f = normalize3(sub3(tgt, pos));
  k.r = normalize3(cross3(k.f, up));
  k.u = cross3(k.r, k.f);
  k.sys = (float)std::tan((double)c->vfov_deg * kPiD / 360.0);
  k.sxs = k.sys * ((float)c->width / (float)c->height);
  k.W = c->width; k.H = c->height; k.spp = c->spp;
  return k;
}

V3 cam_dir(const Cam& k, int x, int y, int s) {
  float ox = 0.0f, oy = 0.0f;
  if (k.spp == 4) { ox = kGrid4[s][0]; oy = kGrid4[s][1]; }
  float fx = (float)x + (0.5f + ox);
  float fy = (float)y + (0.5f + oy);
  float ndx = (2.0f * fx) / (float)k.W - 1.0f;
  float ndy = 1.0f - (2.0f * fy) / (float)k.H;
  float sx = ndx * k.sxs, sy = ndy * k.sys;
  V3 dir = mk(std::fmaf(sx, k.r.x, std::fmaf(sy, k.u.x, k.f.x)),
              std::fmaf(sx, k.r.y, std::fmaf(sy, k.u.y, k.f.y)),
              std::fmaf(sx, k.r.z, std::fmaf(sy, k.u.z, k.f.z)));
  return normalize3(dir);
}

// ---------------------------------------------------------------------------
// §IV-B-1: f = f_d + f_s,  f_s = D F G / (4 (n.l)(n.v)) with
//   D = a2 / (pi ((n.h)^2 (a2 - 1) + 1)^2),  a = r^2, a2 = a^2 (GGX, Walter 2007)
//   F = F0 + (1 - F0)(1 - v.h)^5                  (Schlick 1994)
//   G = G1(n.l) G1(n.v), G1(x) = x / (x (1-k) + k), k = (r+1)^2/8  (Karis 2013)
//   G / (4 nl nv) = 1 / (4 (nl(1-k)+k)(nv(1-k)+k))  (cancelled form)
//   F0 = 0.04 (1 - m) + albedo m,  f_d = (1 - F)(1 - m) albedo / pi (Lambert)
// FP32 operation order as written below.
// ---------------------------------------------------------------------------
void brdf32(V3 n, V3 v, V3 l, const orc_material& M, float f[3]) {
  V3 hu = add3(l, v);
  V3 h = normalize3(hu);
  float nl = std::max(dot3(n, l), 0.0f);
  float nv = std::max(dot3(n, v), 0.0f);
  float nh = std::max(dot3(n, h), 0.0f);
  float vh = std::max(dot3(v, h), 0.0f);
  float r = M.roughness, m = M.metallic;
  float a = r * r;
  float a2 = a * a;
  float dd = std::fmaf(nh * nh, a2 - 1.0f, 1.0f);
  float D = a2 / ((kPiF * dd) * dd);
  float rp1 = r + 1.0f;
  float k = (rp1 * rp1) * 0.125f;
  float omk = 1.0f - k;
  float gl = std::fmaf(nl, omk, k);
  float gv = std::fmaf(nv, omk, k);
  float vis = 0.25f / (gl * gv);
  float Dv = D * vis;
  float w = 1.0f - vh;
  float w2 = w * w;
  float w5 = (w2 * w2) * w;
  float omm = 1.0f - m;
  for (int c = 0; c < 3; ++c) {
    float alb = M.albedo[c];
    float F0 = std::fmaf(m, alb - 0.04f, 0.04f);
    float F = std::fmaf(1.0f - F0, w5, F0);
    float spec = Dv * F;
    float kd = (1.0f - F) * omm;
    float diff = (kd * alb) * kInvPiF;
    f[c] = diff + spec;
  }
}

struct SampleOut { int32_t prim; float t, t2; uint16_t vis; float rgb[3]; };

float scene_eps(const orc_scene& S) {
  if (S.nt == 0) return 0.0f;
  const Box& B = S.two_level ? S.inst_union : S.scene_box;
  V3 ext = mk(B.hi[0] - B.lo[0], B.hi[1] - B.lo[1], B.hi[2] - B.lo[2]);
  return 1e-4f * std::sqrt(dot3(ext, ext));
}

// Light vector of light j from point po (§IV-B-3: the shadow ray runs from the
// fragment's world position to the light's position; a directional light is
// at infinity).  E = I / d^2 for a point light, I for a directional one.
void light_vec(const orc_light& L, V3 po, V3& l, float& E, float& tmax) {
  if (L.type == 0) {
    V3 lv = sub3(mk(L.v[0], L.v[1], L.v[2]), po);
    float d2 = dot3(lv, lv);
    float dist = std::sqrt(d2);
    l = mk(lv.x / dist, lv.y / dist, lv.z / dist);
    E = L.intensity / d2;
    tmax = dist;
  } else {
    l = normalize3(mk(L.v[0], L.v[1], L.v[2]));
    E = L.intensity;
    tmax = kInfF;
  }
}

// Hit-point frame: p = fma(t, d, o); n = normalize(cross(e1, e2)) turned to
// face the ray; shadow origin po = fma(eps, n, p).
void hit_frame(const orc_scene& S, int32_t prim, V3 o, V3 d, float t, float eps, V3& n, V3& po) {
  V3 a, b, c;
  if (S.two_level) {
    a = rest_v(S, S.idx[3 * prim]);
    b = rest_v(S, S.idx[3 * prim + 1]);
    c = rest_v(S, S.idx[3 * prim + 2]);
    const float* m = S.xf.data() + 12 * S.vbody[S.idx[3 * prim]];
    V3 cr = cross3(sub3(b, a), sub3(c, a));
    n = normalize3(mk(std::fmaf(m[0], cr.x, std::fmaf(m[1], cr.y, m[2] * cr.z)),
                      std::fmaf(m[4], cr.x, std::fmaf(m[5], cr.y, m[6] * cr.z)),
                      std::fmaf(m[8], cr.x, std::fmaf(m[9], cr.y, m[10] * cr.z))));
  } else {
    tri_verts(S, prim, a, b, c);
    V3 e1 = sub3(b, a), e2 = sub3(c, a);
    n = normalize3(cross3(e1, e2));
  }
  if (dot3(n, d) > 0.0f) n = neg3(n);
  V3 p = mk(std::fmaf(t, d.x, o.x), std::fmaf(t, d.y, o.y), std::fmaf(t, d.z, o.z));
  po = mk(std::fmaf(eps, n.x, p.x), std::fmaf(eps, n.y, p.y), std::fmaf(eps, n.z, p.z));
}

// ---------------------------------------------------------------------------
// Smooth shading normal (§IV-A-1: the main pass shades with the meshes'
// per-vertex normal attribute, as glTF-like assets carry it).  For the hit
// of the ray (o, d) on triangle prim:
//   (u, v)  barycentrics from the ray/triangle test of the world-space
//           triangle (the same FP32 steps that found the hit), so the point
//           is (1-u-v) v0 + u v1 + v v2
//   n_r     = fma(v, n2, fma(u, n1, w0 n0)) per component, w0 = (1 - u) - v,
//           from the rest normals n0, n1, n2 of the triangle's vertices
//   n_w     = R n_r with the rows of the body's rotation R (normals of a
//           rigid body turn with it; no translation)
//   n_s     = normalize(n_w), then negated if n_s . n_g < 0, n_g being the
//           geometric normal already turned to face the ray; a zero n_w
//           keeps n_g
// n_s replaces n in n.l, n.v, n.h (shading and the cast test of the shadow
// rays); the shadow origin stays lifted along n_g.
// ---------------------------------------------------------------------------
V3 shading_normal(const orc_scene& S, int32_t prim, V3 o, V3 d, V3 ng) {
  if (S.vnrm.empty()) return ng;
  const uint32_t i[3] = {S.idx[3 * prim], S.idx[3 * prim + 1], S.idx[3 * prim + 2]};
  V3 a, b, c;
  tri_verts(S, prim, a, b, c);
  float t, u, v;
  mt_hit(o, d, a, b, c, t, u, v);
  V3 nn[3];
  for (int k = 0; k < 3; ++k) nn[k] = mk(S.vnrm[4 * i[k]], S.vnrm[4 * i[k] + 1], S.vnrm[4 * i[k] + 2]);
  const float w0 = (1.0f - u) - v;
  const V3 nr = mk(std::fmaf(v, nn[2].x, std::fmaf(u, nn[1].x, w0 * nn[0].x)),
                   std::fmaf(v, nn[2].y, std::fmaf(u, nn[1].y, w0 * nn[0].y)),
                   std::fmaf(v, nn[2].z, std::fmaf(u, nn[1].z, w0 * nn[0].z)));
  const float* m = S.xf.data() + 12 * S.vbody[i[0]];
  const V3 nw = mk(std::fmaf(m[0], nr.x, std::fmaf(m[1], nr.y, m[2] * nr.z)),
                   std::fmaf(m[4], nr.x, std::fmaf(m[5], nr.y, m[6] * nr.z)),
                   std::fmaf(m[8], nr.x, std::fmaf(m[9], nr.y, m[10] * nr.z)));
  if (!(dot3(nw, nw) > 0.0f)) return ng;
  V3 ns = normalize3(nw);
  if (dot3(ns, ng) < 0.0f) ns = neg3(ns);
  return ns;
}

SampleOut shade_sample(const orc_scene& S, const Cam& K, const orc_light* L, int nl, int x, int y,
                       int s, bool bvh, bool want2) {
  SampleOut out;
  out.vis = 0;
  out.rgb[0] = out.rgb[1] = out.rgb[2] = 0.0f;
  V3 o = K.o, d = cam_dir(K, x, y, s);
  Hit h = trace(S, o, d, 0.0f, bvh, want2);
  out.prim = h.prim;
  out.t = h.t;
  out.t2 = h.t2;
  if (h.prim < 0) return out;
  float eps = scene_eps(S);
  V3 n, po;
  hit_frame(S, h.prim, o, d, h.t, eps, n, po);
  n = shading_normal(S, h.prim, o, d, n);
  V3 v = neg3(d);
  const orc_material& M = S.mats[S.tri_mat[h.prim]];
  for (int j = 0; j < nl; ++j) {
    V3 l;
    float E, tmax;
    light_vec(L[j], po, l, E, tmax);
    float ndl = dot3(n, l);
    if (!(ndl > 0.0f)) continue;
    out.vis |= (uint16_t)(1u << (8 + j));
    if (occluded(S, po, l, tmax, h.prim, bvh)) continue;
    out.vis |= (uint16_t)(1u << j);
    float f[3];
    brdf32(n, v, l, M, f);
    float En = E * ndl;
    for (int c = 0; c < 3; ++c) out.rgb[c] = out.rgb[c] + f[c] * En;
  }
  return out;
}

// ---------------------------------------------------------------------------
// FP64 twin of the shading (fixed visibility), with its analytic gradient.
// ---------------------------------------------------------------------------
// The gradient checks hold the geometry fixed at the frame the renderer
// shades with: the FP32 hit frame and light vectors of the forward path
// (hit_frame, light_vec, h = normalize(l + v)) give n.l, n.v, n.h, v.h and
// the falloff g = 1/d^2 (1 for a directional light); everything that depends
// on the material parameters and intensities is then evaluated in FP64.
struct Cos64 { double nl, nv, nh, vh, g; bool lit; };
struct Geo64 { int nlights; Cos64 c[8]; };

bool geo64(const orc_scene& S, const Cam& K, const orc_light* L, int nl, int x, int y, int s,
           int32_t prim, float t, uint16_t vis, Geo64& G) {
  if (prim < 0) return false;
  V3 o = K.o, d = cam_dir(K, x, y, s);
  V3 n, po;
  hit_frame(S, prim, o, d, t, scene_eps(S), n, po);
  n = shading_normal(S, prim, o, d, n);
  V3 v = neg3(d);
  G.nlights = nl;
  for (int j = 0; j < nl; ++j) {
    V3 l;
    float E, tmax;
    light_vec(L[j], po, l, E, tmax);
    float d2 = 1.0f;
    if (L[j].type == 0) {
      V3 lv = sub3(mk(L[j].v[0], L[j].v[1], L[j].v[2]), po);
      d2 = dot3(lv, lv);
    }
    V3 h = normalize3(add3(l, v));
    Cos64& c = G.c[j];
    float ndl = dot3(n, l);
    c.lit = ((vis >> j) & 1u) && ndl > 0.0f;
    c.nl = std::max(ndl, 0.0f);
    c.nv = std::max(dot3(n, v), 0.0f);
    c.nh = std::max(dot3(n, h), 0.0f);
    c.vh = std::max(dot3(v, h), 0.0f);
    c.g = 1.0 / (double)d2;
  }
  return true;
}

// The same cosines from an FP64 hit frame recomputed from the FP32 inputs
// alone (the camera ray and the world triangle, widened): t by
// Moller-Trumbore in FP64, p = o + t d, n = normalize(e1 x e2) facing the
// ray, po = p + eps n, v = normalize(-d), the light vector, h, the cosines
// and 1/d^2 in FP64.  It owes nothing to the FP32 frame beyond those inputs,
// so it checks the reading that holds the geometry at that frame (flat
// normals, single-level scenes; visibility stays the forward's).
bool geo64_fresh(const orc_scene& S, const Cam& K, const orc_light* L, int nl, int x, int y, int s,
                 int32_t prim, uint16_t vis, Geo64& G) {
  if (prim < 0) return false;
  const D3 o = tod(K.o), d = tod(cam_dir(K, x, y, s));
  V3 a32, b32, c32;
  tri_verts(S, prim, a32, b32, c32);
  const D3 a = tod(a32), e1 = dsub(tod(b32), a), e2 = dsub(tod(c32), a);
  const D3 pv = dcross(d, e2);
  const double det = ddot(e1, pv);
  if (det == 0.0) return false;
  const D3 q = dcross(dsub(o, a), e1);
  const double t = ddot(e2, q) / det;
  const D3 p = dk(o.x + t * d.x, o.y + t * d.y, o.z + t * d.z);
  D3 n = dnorm(dcross(e1, e2));
  if (ddot(n, d) > 0.0) n = dk(-n.x, -n.y, -n.z);
  const double eps = scene_eps(S);
  const D3 po = dk(p.x + eps * n.x, p.y + eps * n.y, p.z + eps * n.z);
  const D3 v = dnorm(dk(-d.x, -d.y, -d.z));
  G.nlights = nl;
  for (int j = 0; j < nl; ++j) {
    D3 l;
    double g = 1.0;
    if (L[j].type == 0) {
      const D3 lv = dsub(dk(L[j].v[0], L[j].v[1], L[j].v[2]), po);
      const double d2 = ddot(lv, lv);
      l = dnorm(lv);
      g = 1.0 / d2;
    } else {
      l = dnorm(dk(L[j].v[0], L[j].v[1], L[j].v[2]));
    }
    const D3 h = dnorm(dk(l.x + v.x, l.y + v.y, l.z + v.z));
    Cos64& c = G.c[j];
    const double ndl = ddot(n, l);
    c.lit = ((vis >> j) & 1u) && ndl > 0.0;
    c.nl = std::max(ndl, 0.0);
    c.nv = std::max(ddot(n, v), 0.0);
    c.nh = std::max(ddot(n, h), 0.0);
    c.vh = std::max(ddot(v, h), 0.0);
    c.g = g;
  }
  return true;
}

// f_c and its derivatives d/d albedo_c, d/d rough, d/d metal (kmode 0), FP64,
// at fixed cosines.  dd is formed as (1-nh)(1+nh) + nh^2 a2 (no cancellation).
struct Brdf64 { double f[3], dalb[3], dr[3], dm[3]; };

Brdf64 brdf64(const Cos64& cs, const double* alb, double r, double m) {
  double nl = cs.nl, nv = cs.nv, nh = cs.nh, vh = cs.vh;
  double a = r * r, a2 = a * a;
  double s1 = (1.0 - nh) * (1.0 + nh);
  double dd = s1 + nh * nh * a2;
  double D = a2 / (kPiD * dd * dd);
  double dD_da2 = (s1 - a2 * nh * nh) / (kPiD * dd * dd * dd);
  double dD_dr = dD_da2 * 4.0 * r * r * r;
  double k = (r + 1.0) * (r + 1.0) / 8.0, dk_dr = (r + 1.0) / 4.0;
  double gl = nl * (1.0 - k) + k, gv = nv * (1.0 - k) + k;
  double vis = 1.0 / (4.0 * gl * gv);
  double dvis_dk = -vis * ((1.0 - nl) / gl + (1.0 - nv) / gv);
  double w = 1.0 - vh, w5 = w * w * w * w * w;
  Brdf64 B;
  for (int c = 0; c < 3; ++c) {
    double F0 = 0.04 * (1.0 - m) + alb[c] * m;
    double F = F0 + (1.0 - F0) * w5;
    double spec = D * vis * F;
    double diff = (1.0 - F) * (1.0 - m) * alb[c] / kPiD;
    B.f[c] = diff + spec;
    double dF_dF0 = 1.0 - w5;
    double dfdF = D * vis - (1.0 - m) * alb[c] / kPiD;
    B.dalb[c] = (1.0 - F) * (1.0 - m) / kPiD + dfdF * dF_dF0 * m;
    B.dm[c] = dfdF * dF_dF0 * (alb[c] - 0.04) - (1.0 - F) * alb[c] / kPiD;
    B.dr[c] = F * (dD_dr * vis + D * dvis_dk * dk_dr);
  }
  return B;
}

}  // namespace

// ===========================================================================
// C API
// ===========================================================================
extern "C" {

orc_scene* orc_scene_new(const float* verts4, int64_t nv, const uint32_t* idx, int64_t nt,
                         const uint32_t* tri_mat, const uint16_t* vert_body,
                         const orc_material* mats, int32_t nmat, int32_t nbody) {
  if (nv < 0 || nt < 0 || nmat < 1 || nbody < 1) return nullptr;
  for (int64_t i = 0; i < 3 * nt; ++i) if (idx[i] >= (uint64_t)nv) return nullptr;
  for (int64_t i = 0; i < nt; ++i) if (tri_mat[i] >= (uint32_t)nmat) return nullptr;
  for (int64_t i = 0; i < nv; ++i) if (vert_body[i] >= (uint32_t)nbody) return nullptr;
  orc_scene* S = new orc_scene;
  S->nv = nv; S->nt = nt; S->nmat = nmat; S->nbody = nbody;
  S->rest.assign(verts4, verts4 + 4 * nv);
  S->idx.assign(idx, idx + 3 * nt);
  S->tri_mat.assign(tri_mat, tri_mat + nt);
  S->vbody.assign(vert_body, vert_body + nv);
  S->mats.assign(mats, mats + nmat);
  return S;
}

void orc_scene_free(orc_scene* s) { delete s; }

int32_t orc_set_materials(orc_scene* s, const orc_material* mats, int32_t nmat) {
  if (nmat != s->nmat) return -1;
  s->mats.assign(mats, mats + nmat);
  return 0;
}

// sRGB-encoded colour to linear (IEC 61966-2-1 decode, §IV-A-1 colour
// inputs): c / 12.92 for c <= 0.04045, else ((c + 0.055) / 1.055)^2.4;
// evaluated in FP64 and rounded to FP32 once.
float orc_srgb_decode(float c) {
  const double x = c;
  return (float)(x <= 0.04045 ? x / 12.92 : std::pow((x + 0.055) / 1.055, 2.4));
}

int32_t orc_set_materials_srgb(orc_scene* s, const orc_material* mats, int32_t nmat) {
  if (nmat != s->nmat) return -1;
  s->mats.assign(mats, mats + nmat);
  for (auto& M : s->mats)
    for (int c = 0; c < 3; ++c) M.albedo[c] = orc_srgb_decode(M.albedo[c]);
  return 0;
}

int32_t orc_set_normals(orc_scene* s, const float* nrm4) {
  if (!nrm4) {
    s->vnrm.clear();
    return 0;
  }
  s->vnrm.assign(nrm4, nrm4 + 4 * s->nv);
  return 0;
}

void orc_shading_normal(const orc_scene* s, int32_t prim, const float* o, const float* d, float* n3) {
  const orc_scene& S = *s;
  V3 O = mk(o[0], o[1], o[2]), D = mk(d[0], d[1], d[2]), a, b, c;
  tri_verts(S, prim, a, b, c);
  V3 ng = normalize3(cross3(sub3(b, a), sub3(c, a)));
  if (dot3(ng, D) > 0.0f) ng = neg3(ng);
  V3 ns = shading_normal(S, prim, O, D, ng);
  n3[0] = ns.x; n3[1] = ns.y; n3[2] = ns.z;
}

int32_t orc_update(orc_scene* s, const float* xforms, int32_t rebuild) {
  transform(*s, xforms);
  if (rebuild || !s->built) build(*s);
  refit_all(*s);
  s->xf.assign(xforms, xforms + 12 * s->nbody);
  if (s->two_level) instance_boxes(*s);
  return 0;
}

int32_t orc_set_two_level(orc_scene* s, int32_t enable) {
  if (!enable) {
    s->two_level = false;
    return 0;
  }
  if (!set_two_level(*s)) return -1;
  if (!s->xf.empty()) instance_boxes(*s);
  return 0;
}

int32_t orc_get(const orc_scene* s, int32_t what, void* dst) {
  const int64_t T = s->nt;
  switch (what) {
    case 0: std::memcpy(dst, s->world.data(), sizeof(V3) * s->nv); return 0;
    case 1: std::memcpy(dst, s->morton.data(), 8 * T); return 0;
    case 2: std::memcpy(dst, s->order.data(), 4 * T); return 0;
    case 3: std::memcpy(dst, s->child.data(), 4 * s->child.size()); return 0;
    case 4: std::memcpy(dst, s->parent.data(), 4 * s->parent.size()); return 0;
    case 5: std::memcpy(dst, s->box.data(), sizeof(Box) * s->box.size()); return 0;
    case 6: std::memcpy(dst, s->cb, sizeof(float) * 6); return 0;
    case 7: std::memcpy(dst, &s->scene_box, sizeof(Box)); return 0;
  }
  return -1;
}

void orc_trace(const orc_scene* s, const float* o, const float* d, int64_t n, float tmin,
               int32_t use_bvh, int32_t* prim, float* t, float* u, float* v, float* t2) {
  for (int64_t i = 0; i < n; ++i) {
    Hit h = trace(*s, mk(o[3 * i], o[3 * i + 1], o[3 * i + 2]), mk(d[3 * i], d[3 * i + 1], d[3 * i + 2]),
                  tmin, use_bvh != 0, t2 != nullptr);
    prim[i] = h.prim;
    t[i] = h.t;
    if (u) u[i] = h.u;
    if (v) v[i] = h.v;
    if (t2) t2[i] = h.t2;
  }
}

void orc_occluded(const orc_scene* s, const float* o, const float* d, const float* tmax,
                  const int32_t* skip, int64_t n, int32_t use_bvh, uint8_t* out) {
  for (int64_t i = 0; i < n; ++i)
    out[i] = occluded(*s, mk(o[3 * i], o[3 * i + 1], o[3 * i + 2]), mk(d[3 * i], d[3 * i + 1], d[3 * i + 2]),
                      tmax[i], skip ? skip[i] : -1, use_bvh != 0) ? 1 : 0;
}

void orc_camera_ray(const orc_camera* c, int32_t x, int32_t y, int32_t k, float* o3, float* d3) {
  Cam K = make_cam(c);
  V3 d = cam_dir(K, x, y, k);
  o3[0] = K.o.x; o3[1] = K.o.y; o3[2] = K.o.z;
  d3[0] = d.x; d3[1] = d.y; d3[2] = d.z;
}

void orc_render_samples(const orc_scene* s, const orc_camera* c, const orc_light* L, int32_t nl,
                        const int64_t* ids, int64_t n, int32_t use_bvh,
                        int32_t* prim, float* t, float* t2, uint16_t* vis, float* rgb) {
  Cam K = make_cam(c);
  for (int64_t i = 0; i < n; ++i) {
    int64_t id = ids[i];
    int sidx = (int)(id % K.spp);
    int64_t pix = id / K.spp;
    int x = (int)(pix % K.W), y = (int)(pix / K.W);
    SampleOut so = shade_sample(*s, K, L, nl, x, y, sidx, use_bvh != 0, t2 != nullptr);
    if (prim) prim[i] = so.prim;
    if (t) t[i] = so.t;
    if (t2) t2[i] = so.t2;
    if (vis) vis[i] = so.vis;
    if (rgb) { rgb[3 * i] = so.rgb[0]; rgb[3 * i + 1] = so.rgb[1]; rgb[3 * i + 2] = so.rgb[2]; }
  }
}

// Box-filter resolve (§IV-B-2, multisample resolve): pixel = (sum over the
// samples in order k = 0..spp-1) / spp; alpha = hits / spp.
void orc_render_rows(const orc_scene* s, const orc_camera* c, const orc_light* L, int32_t nl,
                     int32_t row0, int32_t row1, int32_t use_bvh, float* rgba) {
  Cam K = make_cam(c);
  for (int y = row0; y < row1; ++y)
    for (int x = 0; x < K.W; ++x) {
      float acc[3] = {0.0f, 0.0f, 0.0f};
      int hits = 0;
      for (int k = 0; k < K.spp; ++k) {
        SampleOut so = shade_sample(*s, K, L, nl, x, y, k, use_bvh != 0, false);
        for (int ch = 0; ch < 3; ++ch) acc[ch] = acc[ch] + so.rgb[ch];
        hits += so.prim >= 0;
      }
      float* px = rgba + 4 * ((int64_t)y * K.W + x);
      for (int ch = 0; ch < 3; ++ch) px[ch] = acc[ch] / (float)K.spp;
      px[3] = (float)hits / (float)K.spp;
    }
}

void orc_brdf_f32(const float* n, const float* v, const float* l, const orc_material* m, float* f_rgb) {
  brdf32(mk(n[0], n[1], n[2]), mk(v[0], v[1], v[2]), mk(l[0], l[1], l[2]), *m, f_rgb);
}

double orc_ggx_d(double nh, double alpha) {
  double a2 = alpha * alpha;
  double dd = nh * nh * (a2 - 1.0) + 1.0;
  return a2 / (kPiD * dd * dd);
}

double orc_schlick_f(double vh, double f0) { return f0 + (1.0 - f0) * std::pow(1.0 - vh, 5.0); }

double orc_smith_g(double nl, double nv, double rough, int32_t kmode) {
  double k = kmode == 0 ? (rough + 1.0) * (rough + 1.0) / 8.0 : rough * rough / 2.0;
  return (nl / (nl * (1.0 - k) + k)) * (nv / (nv * (1.0 - k) + k));
}

void orc_brdf_f64(const double* n, const double* v, const double* l, const double* albedo,
                  double rough, double metal, int32_t kmode, double* fd_rgb, double* fs_rgb) {
  D3 N = dk(n[0], n[1], n[2]), V = dk(v[0], v[1], v[2]), L = dk(l[0], l[1], l[2]);
  D3 h = dnorm(dk(L.x + V.x, L.y + V.y, L.z + V.z));
  double nl = std::max(ddot(N, L), 0.0), nv = std::max(ddot(N, V), 0.0);
  double nh = std::max(ddot(N, h), 0.0), vh = std::max(ddot(V, h), 0.0);
  double D = orc_ggx_d(nh, rough * rough);
  double k = kmode == 0 ? (rough + 1.0) * (rough + 1.0) / 8.0 : rough * rough / 2.0;
  double visq = 1.0 / (4.0 * (nl * (1.0 - k) + k) * (nv * (1.0 - k) + k));
  for (int c = 0; c < 3; ++c) {
    double F0 = 0.04 * (1.0 - metal) + albedo[c] * metal;
    double F = orc_schlick_f(vh, F0);
    fs_rgb[c] = D * F * visq;
    fd_rgb[c] = (1.0 - F) * (1.0 - metal) * albedo[c] / kPiD;
  }
}

float orc_shadow_eps(const orc_scene* s) { return scene_eps(*s); }

static void shade_f64_rows(const orc_scene* s, const orc_camera* c, const orc_light* L, int32_t nl,
                           const int32_t* prim, const float* t, const uint16_t* vis,
                           const double* params, const double* inten, bool fresh, double* img) {
  Cam K = make_cam(c);
  for (int y = 0; y < K.H; ++y)
    for (int x = 0; x < K.W; ++x) {
      double acc[3] = {0, 0, 0};
      for (int k = 0; k < K.spp; ++k) {
        int64_t id = ((int64_t)y * K.W + x) * K.spp + k;
        Geo64 G;
        if (!(fresh ? geo64_fresh(*s, K, L, nl, x, y, k, prim[id], vis[id], G)
                    : geo64(*s, K, L, nl, x, y, k, prim[id], t[id], vis[id], G)))
          continue;
        const double* P = params + 5 * s->tri_mat[prim[id]];
        for (int j = 0; j < nl; ++j) {
          if (!G.c[j].lit) continue;
          Brdf64 B = brdf64(G.c[j], P, P[3], P[4]);
          for (int ch = 0; ch < 3; ++ch) acc[ch] += B.f[ch] * inten[j] * G.c[j].g * G.c[j].nl;
        }
      }
      for (int ch = 0; ch < 3; ++ch) img[3 * ((int64_t)y * K.W + x) + ch] = acc[ch] / K.spp;
    }
}

void orc_shade_f64(const orc_scene* s, const orc_camera* c, const orc_light* L, int32_t nl,
                   const int32_t* prim, const float* t, const uint16_t* vis,
                   const double* params, const double* inten, double* img) {
  shade_f64_rows(s, c, L, nl, prim, t, vis, params, inten, false, img);
}

int32_t orc_shade_f64_fresh(const orc_scene* s, const orc_camera* c, const orc_light* L, int32_t nl,
                            const int32_t* prim, const uint16_t* vis, const double* params,
                            const double* inten, double* img) {
  if (s->two_level || !s->vnrm.empty()) return -1;
  shade_f64_rows(s, c, L, nl, prim, nullptr, vis, params, inten, true, img);
  return 0;
}

void orc_grad_f64(const orc_scene* s, const orc_camera* c, const orc_light* L, int32_t nl,
                  const int32_t* prim, const float* t, const uint16_t* vis,
                  const double* params, const double* inten, const double* dimg,
                  double* dparams, double* dinten) {
  Cam K = make_cam(c);
  std::fill(dparams, dparams + 5 * s->nmat, 0.0);
  std::fill(dinten, dinten + nl, 0.0);
  for (int y = 0; y < K.H; ++y)
    for (int x = 0; x < K.W; ++x) {
      const double* gp = dimg + 3 * ((int64_t)y * K.W + x);
      for (int k = 0; k < K.spp; ++k) {
        int64_t id = ((int64_t)y * K.W + x) * K.spp + k;
        Geo64 G;
        if (!geo64(*s, K, L, nl, x, y, k, prim[id], t[id], vis[id], G)) continue;
        uint32_t mat = s->tri_mat[prim[id]];
        const double* P = params + 5 * mat;
        double* dP = dparams + 5 * mat;
        for (int j = 0; j < nl; ++j) {
          if (!G.c[j].lit) continue;
          Brdf64 B = brdf64(G.c[j], P, P[3], P[4]);
          double w = G.c[j].g * G.c[j].nl / K.spp;
          for (int ch = 0; ch < 3; ++ch) {
            double up = gp[ch] * w;  // dL/d f_c, per unit intensity
            dP[ch] += up * inten[j] * B.dalb[ch];
            dP[3] += up * inten[j] * B.dr[ch];
            dP[4] += up * inten[j] * B.dm[ch];
            dinten[j] += up * B.f[ch];
          }
        }
      }
    }
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Display output stage (§IV-A-1: Reinhard tone mapping, then gamma
// correction = the inverse of the sRGB-to-linear conversion; §IV-B-2: FXAA),
// applied to the resolved linear HDR image.  FP32, in this order:
//   c' = e * c; r = c' / (1 + c')                       (Reinhard, per channel)
//   s = r <= 0.0031308 ? 12.92 * r : 1.055 * r^(1/2.4) - 0.055   (sRGB, IEC 61966-2-1)
//   r^(1/2.4) = (r^(1/12))^5, r^(1/12) = m^(1/12) * 2^(-k/12) for r = m 2^-k,
//   m in [1, 2); m^(1/12) by three Newton steps on t^12 = m from the chord
//   1 + (m - 1)(2^(1/12) - 1); 2^(-k/12) and 2^(1/12) - 1 rounded from FP64
//   byte = floor(clamp(v, 0, 1) * 255 + 0.5)
// FXAA (Lottes' FXAA, its simple form), on the gamma-space image G with
// clamp-to-edge fetches and bilinear taps (pixel centres at +0.5):
//   luma = (0.299 r + 0.587 g) + 0.114 b
//   gradient (x right, y down) from the four diagonal neighbours;
//   edge direction d = (-(S - N), E - W) with N = lNW + lNE, S = lSW + lSE,
//   W = lNW + lSW, E = lNE + lSE;
//   d /= min(|d.x|, |d.y|) + max((lNW + lNE + lSW + lSE) * (0.25 / 8), 1/128),
//   clamped to [-8, 8] pixels;
//   A = (tap(p + d (1/3 - 1/2)) + tap(p + d (2/3 - 1/2))) / 2
//   B = A / 2 + (tap(p - d / 2) + tap(p + d / 2)) / 4
//   out = luma(B) outside [min, max] of the five lumas ? A : B
// Alpha (coverage) is quantised as is.
// ---------------------------------------------------------------------------
namespace {

struct DispConst {
  float tab[12];   // 2^(-k/12)
  float chord;     // 2^(1/12) - 1
};

DispConst disp_const() {
  DispConst c;
  for (int k = 0; k < 12; ++k) c.tab[k] = (float)std::pow(2.0, -k / 12.0);
  c.chord = (float)(std::pow(2.0, 1.0 / 12.0) - 1.0);
  return c;
}

float root12_pow5(const DispConst& C, float r) {  // r^(5/12), r in [2^-9, 1)
  int e = 0;
  float m = std::frexp(r, &e);  // r = m 2^e, m in [0.5, 1)
  m = m * 2.0f;                 // [1, 2)
  const int k = 1 - e;          // r = m 2^-k
  float t = 1.0f + (m - 1.0f) * C.chord;
  for (int i = 0; i < 3; ++i) {
    float t2 = t * t, t4 = t2 * t2, t8 = t4 * t4, t11 = (t8 * t2) * t;
    t = (11.0f * t + m / t11) / 12.0f;
  }
  const float u = t * C.tab[k];  // r^(1/12)
  const float u2 = u * u;
  return (u2 * u2) * u;
}

float srgb_encode(const DispConst& C, float r) {
  if (r <= 0.0031308f) return 12.92f * r;
  return 1.055f * root12_pow5(C, r) - 0.055f;
}

float tonemap(const DispConst& C, float c, float e) {
  const float cc = e * c;
  return srgb_encode(C, cc / (1.0f + cc));
}

uint8_t quant(float v) {
  const float w = std::min(std::max(v, 0.0f), 1.0f) * 255.0f + 0.5f;
  return (uint8_t)(int)std::floor(w);
}

float luma3(const float* c) { return (0.299f * c[0] + 0.587f * c[1]) + 0.114f * c[2]; }

struct Img {
  const float* g;  // [H*W*4] gamma-space rgb + coverage
  int W, H;
  const float* at(int i, int j) const {
    i = std::min(std::max(i, 0), W - 1);
    j = std::min(std::max(j, 0), H - 1);
    return g + 4 * ((int64_t)j * W + i);
  }
  void tap(float px, float py, float* out) const {
    const float u = px - 0.5f, v = py - 0.5f;
    const float fi = std::floor(u), fj = std::floor(v);
    const float fu = u - fi, fv = v - fj;
    const int i0 = (int)fi, j0 = (int)fj;
    const float *c00 = at(i0, j0), *c10 = at(i0 + 1, j0), *c01 = at(i0, j0 + 1), *c11 = at(i0 + 1, j0 + 1);
    for (int ch = 0; ch < 3; ++ch) {
      const float top = c00[ch] + (c10[ch] - c00[ch]) * fu;
      const float bot = c01[ch] + (c11[ch] - c01[ch]) * fu;
      out[ch] = top + (bot - top) * fv;
    }
  }
};

void fxaa_pixel(const Img& I, int x, int y, float* out) {
  const float lM = luma3(I.at(x, y)), lNW = luma3(I.at(x - 1, y - 1)), lNE = luma3(I.at(x + 1, y - 1)),
              lSW = luma3(I.at(x - 1, y + 1)), lSE = luma3(I.at(x + 1, y + 1));
  const float lmin = std::min(lM, std::min(std::min(lNW, lNE), std::min(lSW, lSE)));
  const float lmax = std::max(lM, std::max(std::max(lNW, lNE), std::max(lSW, lSE)));
  float dx = -((lSW + lSE) - (lNW + lNE));
  float dy = (lNE + lSE) - (lNW + lSW);
  const float reduce = std::max((((lNW + lNE) + lSW) + lSE) * (0.25f * 0.125f), 1.0f / 128.0f);
  const float rcp = 1.0f / (std::min(std::fabs(dx), std::fabs(dy)) + reduce);
  dx = std::min(std::max(dx * rcp, -8.0f), 8.0f);
  dy = std::min(std::max(dy * rcp, -8.0f), 8.0f);
  const float px = (float)x + 0.5f, py = (float)y + 0.5f;
  const float k1 = 1.0f / 3.0f - 0.5f, k2 = 2.0f / 3.0f - 0.5f;
  float a1[3], a2[3], b1[3], b2[3], A[3], B[3];
  I.tap(px + dx * k1, py + dy * k1, a1);
  I.tap(px + dx * k2, py + dy * k2, a2);
  I.tap(px + dx * -0.5f, py + dy * -0.5f, b1);
  I.tap(px + dx * 0.5f, py + dy * 0.5f, b2);
  for (int ch = 0; ch < 3; ++ch) {
    A[ch] = 0.5f * (a1[ch] + a2[ch]);
    B[ch] = A[ch] * 0.5f + 0.25f * (b1[ch] + b2[ch]);
  }
  const float lB = luma3(B);
  const float* pick = (lB < lmin || lB > lmax) ? A : B;
  for (int ch = 0; ch < 3; ++ch) out[ch] = pick[ch];
}

}  // namespace

extern "C" {

float orc_srgb_encode(float r) { return srgb_encode(disp_const(), r); }
float orc_root12_pow5(float r) { return root12_pow5(disp_const(), r); }

void orc_display(const float* hdr, int32_t W, int32_t H, float exposure, int32_t fxaa, float* gamma_out,
                 uint8_t* out) {
  const DispConst C = disp_const();
  std::vector<float> g(4 * (size_t)W * H);
  for (int64_t p = 0; p < (int64_t)W * H; ++p) {
    for (int ch = 0; ch < 3; ++ch) g[4 * p + ch] = tonemap(C, hdr[4 * p + ch], exposure);
    g[4 * p + 3] = hdr[4 * p + 3];
  }
  if (gamma_out) std::copy(g.begin(), g.end(), gamma_out);
  const Img I{g.data(), W, H};
  for (int y = 0; y < H; ++y)
    for (int x = 0; x < W; ++x) {
      const int64_t p = (int64_t)y * W + x;
      float c[3] = {g[4 * p], g[4 * p + 1], g[4 * p + 2]};
      if (fxaa) fxaa_pixel(I, x, y, c);
      for (int ch = 0; ch < 3; ++ch) out[4 * p + ch] = quant(c[ch]);
      out[4 * p + 3] = quant(g[4 * p + 3]);
    }
}

}  // extern "C"
