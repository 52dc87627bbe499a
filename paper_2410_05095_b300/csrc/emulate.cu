// Host emulation of the traversal (a check and a measurement aid, not a
// render path): the device structures of a built scene are copied to host
// memory and the traversal code the render kernels run (traverse for the
// single-level tree, traverse2 for the two-level structure, compiled here
// for the host) walks them for the caller's rays.  Every load goes through
// HostCheckedLoads, which verifies that the address lies inside one of the
// copied arrays and is aligned for its width (16 B for the vector loads, 4 B
// for scalars -- the device arrays themselves are 256-B aligned by
// cudaMalloc, which fire_scene checks); a violation is counted, the load
// returns zeros, and the call reports it.  The kernels' own index checks run
// here unchanged.
//
// The same loads give the traversal's work and demand: a node step is one
// fetch of a 4-wide node's link vector (the last of its seven 16-B loads),
// a triangle test one fetch of a record's first vector; for groups of rays
// taken together (32: a warp of the primary or shadow pass) the distinct
// nodes and triangles the group fetched are what its warp asks of the
// memory system, once each.
#include <algorithm>
#include <cstring>
#include <vector>

#include "trace2.cuh"

namespace fire {
namespace {

enum RegionKind { kNodes = 0, kTris = 1, kOther = 2 };

struct Region {
  const char* base;
  size_t bytes;
  int kind;
};
thread_local std::vector<Region> g_regions;
thread_local uint64_t g_bad_loads = 0;

// visit records of the current group (node key = region << 40 | node index)
struct Visits {
  bool on = false;
  int64_t steps = 0, tests = 0;
  std::vector<int64_t> nodes, tris;
};
thread_local Visits g_visits;

template <class T>
bool load_ok(const T* p) {
  const char* c = reinterpret_cast<const char*>(p);
  for (size_t k = 0; k < g_regions.size(); ++k) {
    const Region& r = g_regions[k];
    if (c >= r.base && c + sizeof(T) <= r.base + r.bytes) {
      const size_t off = (size_t)(c - r.base);
      if (off % sizeof(T) != 0) return false;
      if (g_visits.on) {
        if (r.kind == kNodes && sizeof(T) == 16 && off % sizeof(Node4) == 96) {  // a node's link vector
          ++g_visits.steps;
          g_visits.nodes.push_back(((int64_t)k << 40) | (int64_t)(off / sizeof(Node4)));
        } else if (r.kind == kTris && off % 48 == 0) {  // a record's first vector
          ++g_visits.tests;
          g_visits.tris.push_back((int64_t)(off / 48));
        }
      }
      return true;
    }
  }
  return false;
}

template <class T>
T checked_load(const T* p) {
  if (!load_ok(p)) {
    ++g_bad_loads;
    T z;
    memset(&z, 0, sizeof(z));
    return z;
  }
  return *p;
}

// (host and device members only because the traversal is a host-and-device
// template; the device side is never called)
struct HostCheckedLoads {
#ifdef __CUDA_ARCH__
  __host__ __device__ static float4 f4(const float4*) { return make_float4(0.0f, 0.0f, 0.0f, 0.0f); }
  __host__ __device__ static int4 i4(const int4*) { return make_int4(0, 0, 0, 0); }
  __host__ __device__ static float f1(const float*) { return 0.0f; }
  __host__ __device__ static int i1(const int32_t*) { return 0; }
  __host__ __device__ static void fail(uint32_t*, uint32_t) {}
#else
  __host__ __device__ static float4 f4(const float4* p) { return checked_load(p); }
  __host__ __device__ static int4 i4(const int4* p) { return checked_load(p); }
  __host__ __device__ static float f1(const float* p) { return checked_load(p); }
  __host__ __device__ static int i1(const int32_t* p) { return checked_load(p); }
  __host__ __device__ static void fail(uint32_t* e, uint32_t bits) { *e |= bits; }
#endif
};

// Totals over groups: [0] rays, [1] node steps, [2] triangle tests, [3] sum
// of the distinct nodes per group, [4] of the distinct triangles, [5] groups.
struct GroupTotals {
  int64_t v[6] = {0, 0, 0, 0, 0, 0};
  void close_group() {
    auto distinct = [](std::vector<int64_t>& x) {
      std::sort(x.begin(), x.end());
      const int64_t n = std::unique(x.begin(), x.end()) - x.begin();
      x.clear();
      return n;
    };
    v[1] += g_visits.steps;
    v[2] += g_visits.tests;
    v[3] += distinct(g_visits.nodes);
    v[4] += distinct(g_visits.tris);
    v[5] += 1;
    g_visits.steps = g_visits.tests = 0;
  }
};

// One ray through the structure the view describes.
template <int STACK>
bool trace_one(const Trace2View* v2, const TraceCtx* v1, float3 o, float3 d, bool any, float tmax, int skip, int& p,
               float& tb) {
  int pos = -1;
  if (v2) {
    if (any) return traverse2<HostCheckedLoads, STACK, true>(*v2, o, d, tmax, skip, p, pos, tb);
    traverse2<HostCheckedLoads, STACK, false>(*v2, o, d, 0.0f, -1, p, pos, tb);
  } else {
    if (any) return traverse<HostCheckedLoads, STACK, true>(*v1, o, d, tmax, skip, p, pos, tb);
    traverse<HostCheckedLoads, STACK, false>(*v1, o, d, 0.0f, -1, p, pos, tb);
  }
  return p >= 0;
}

template <int STACK>
void run(const Trace2View* v2, const TraceCtx* v1, const float* o3, const float* d3, const float* tmax,
         const int32_t* skip, int64_t n, bool any, int32_t* prim, float* t, uint8_t* hit, int group,
         GroupTotals* tot, int32_t* steps) {
  for (int64_t i = 0; i < n; ++i) {
    if (tot && i > 0 && i % group == 0) tot->close_group();
    const float3 o = f3(o3[3 * i], o3[3 * i + 1], o3[3 * i + 2]);
    const float3 d = f3(d3[3 * i], d3[3 * i + 1], d3[3 * i + 2]);
    int p = -1;
    float tb = 0.0f;
    const int64_t s0 = g_visits.steps;
    const bool h = trace_one<STACK>(v2, v1, o, d, any, tmax ? tmax[i] : inf_f(), skip ? skip[i] : -1, p, tb);
    if (steps) steps[i] = (int32_t)(g_visits.steps - s0);
    if (prim) prim[i] = any ? -1 : p;
    if (t) t[i] = any ? 0.0f : tb;
    if (hit) hit[i] = h ? 1 : 0;
  }
  if (tot && n > 0) tot->close_group();
  if (tot) tot->v[0] += n;
}

template <class T>
int fetch(std::vector<T>& h, const void* dev, size_t count) {
  h.resize(count > 0 ? count : 1);
  if (count == 0) return FIRE_OK;
  return cuda_check(cudaMemcpy(h.data(), dev, count * sizeof(T), cudaMemcpyDeviceToHost), "emulation copy");
}

// Copies the scene's current structures and runs the rays (group > 0:
// visit totals into tot).
int emulate(fire_scene s, const float* o3, const float* d3, const float* tmax, const int32_t* skip, int64_t n,
            bool any, int32_t* prim, float* t, uint8_t* hit, uint32_t* err_out, int group, GroupTotals* tot,
            int32_t* steps) {
  if (!s->built) return set_error(FIRE_ERR_NOT_BUILT, "emulation before build");
  *err_out = 0;
  if (int e = cuda_check(cudaDeviceSynchronize(), "sync")) return e;
  std::vector<Node4> tlas, nodes;
  std::vector<float4> tris;
  std::vector<int32_t> inst;  // top-level entries (bottom-level node, body)
  std::vector<float4> xf;  // 3 rows per body (16-B aligned, as the device buffer)
  std::vector<TlasInfo> info;
  const size_t nb = (size_t)s->nbody;
  const int64_t cap = s->iter_cap > 0 ? s->iter_cap : 2 * s->nt + 64;
  if (int e = fetch(nodes, s->nodes4, (size_t)s->n4)) return e;
  if (int e = fetch(tris, s->tris, 3 * (size_t)s->nt)) return e;
  g_regions.clear();
  if (s->two_level) {
    if (int e = fetch(info, s->tinfo, 1)) return e;
    if (int e = fetch(tlas, s->tlas, (size_t)kMaxTlasBodies + 2)) return e;
    if (int e = fetch(inst, s->inst, 2 * (size_t)kMaxTlasBodies)) return e;
    if (int e = fetch(xf, s->xf_buf[s->cur], 3 * nb)) return e;
    if (info[0].err) *err_out |= kErrStack;
    g_regions.push_back({reinterpret_cast<const char*>(tlas.data()), sizeof(Node4) * ((size_t)kMaxTlasBodies + 2),
                         kNodes});
  }
  g_regions.push_back({reinterpret_cast<const char*>(nodes.data()), sizeof(Node4) * (size_t)s->n4, kNodes});
  g_regions.push_back({reinterpret_cast<const char*>(tris.data()), sizeof(float4) * 3 * (size_t)s->nt, kTris});
  if (s->two_level) {
    g_regions.push_back({reinterpret_cast<const char*>(inst.data()), 8 * (size_t)kMaxTlasBodies, kOther});
    g_regions.push_back({reinterpret_cast<const char*>(xf.data()), 48 * nb, kOther});
  }
  g_bad_loads = 0;
  g_visits = Visits{};
  uint32_t err = 0;
  Trace2View v2{};
  TraceCtx v1{};
  if (s->two_level) {
    const TlasInfo ti = info[0];
    v2 = Trace2View{tlas.data(), std::min<int64_t>(ti.n, (int64_t)kMaxTlasBodies + 2), nodes.data(), s->n4,
                    tris.data(), s->nt, inst.data(), kMaxTlasBodies, reinterpret_cast<const float*>(xf.data()),
                    s->nbody, ti.span, cap, &err};
  } else {
    v1 = TraceCtx{nodes.data(), s->n4, scene_span<HostCheckedLoads>(nodes.data(), s->nt), tris.data(), s->nt, cap,
                  &err};
  }
  g_visits.on = tot != nullptr;  // (after the span's root-box loads)
  const Trace2View* p2 = s->two_level ? &v2 : nullptr;
  const TraceCtx* p1 = s->two_level ? nullptr : &v1;
  switch (stack_for_height(stack_need(s), 0)) {
    case 32: run<32>(p2, p1, o3, d3, tmax, skip, n, any, prim, t, hit, group, tot, steps); break;
    case 64: run<64>(p2, p1, o3, d3, tmax, skip, n, any, prim, t, hit, group, tot, steps); break;
    default: run<128>(p2, p1, o3, d3, tmax, skip, n, any, prim, t, hit, group, tot, steps); break;
  }
  g_visits = Visits{};
  g_regions.clear();
  *err_out |= err;
  if (g_bad_loads) *err_out |= 0x100u;
  return FIRE_OK;
}

}  // namespace
}  // namespace fire

using namespace fire;

extern "C" int fire_debug_trace_host(fire_scene s, const float* o3, const float* d3, const float* tmax,
                                     const int32_t* skip, int64_t n, int32_t any, int32_t* prim, float* t,
                                     uint8_t* hit, uint32_t* err_out) {
  set_error(FIRE_OK, "");
  if (!s || !err_out || (n > 0 && (!o3 || !d3)) || n < 0)
    return set_error(FIRE_ERR_INVALID_ARG, "NULL argument");
  return emulate(s, o3, d3, tmax, skip, n, any != 0, prim, t, hit, err_out, 0, nullptr, nullptr);
}

extern "C" int fire_debug_trace_stats(fire_scene s, const float* o3, const float* d3, const float* tmax,
                                      const int32_t* skip, int64_t n, int32_t any, int32_t group, int64_t* out8,
                                      int32_t* steps) {
  set_error(FIRE_OK, "");
  if (!s || !out8 || (n > 0 && (!o3 || !d3)) || n < 0) return set_error(FIRE_ERR_INVALID_ARG, "NULL argument");
  if (group < 1) return set_error(FIRE_ERR_INVALID_ARG, "group must be >= 1");
  GroupTotals tot;
  uint32_t err = 0;
  if (int e = emulate(s, o3, d3, tmax, skip, n, any != 0, nullptr, nullptr, nullptr, &err, group, &tot, steps))
    return e;
  for (int k = 0; k < 6; ++k) out8[k] = tot.v[k];
  out8[6] = g_bad_loads;
  out8[7] = err;
  return FIRE_OK;
}
