// Host emulation of the two-level traversal (a check, not a render path):
// the device structures of a built two-level scene are copied to host
// memory and the traversal code the render kernels run (traverse2, compiled
// here for the host) walks them for the caller's rays.  Every load goes
// through HostCheckedLoads, which verifies that the address lies inside one
// of the copied arrays and is aligned for its width (16 B for the vector
// loads, 4 B for scalars -- the device arrays themselves are 256-B aligned by
// cudaMalloc, which fire_scene checks); a violation is counted, the load
// returns zeros, and the call reports it.  The kernels' own index checks run
// here unchanged.
#include <cstring>
#include <vector>

#include "trace2.cuh"

namespace fire {
namespace {

struct Region {
  const char* base;
  size_t bytes;
};
thread_local std::vector<Region> g_regions;
thread_local uint64_t g_bad_loads = 0;

template <class T>
bool load_ok(const T* p) {
  const char* c = reinterpret_cast<const char*>(p);
  for (const Region& r : g_regions)
    if (c >= r.base && c + sizeof(T) <= r.base + r.bytes) return ((size_t)(c - r.base) % sizeof(T)) == 0;
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

// (host and device members only because traverse2 is a host-and-device
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

template <int STACK>
void run(const Trace2View& v, const float* o3, const float* d3, const float* tmax, const int32_t* skip, int64_t n,
         bool any, int32_t* prim, float* t, uint8_t* hit) {
  for (int64_t i = 0; i < n; ++i) {
    const float3 o = f3(o3[3 * i], o3[3 * i + 1], o3[3 * i + 2]);
    const float3 d = f3(d3[3 * i], d3[3 * i + 1], d3[3 * i + 2]);
    int p = -1, pos = -1;
    float tb = 0.0f;
    bool h;
    if (any) {
      h = traverse2<HostCheckedLoads, STACK, true>(v, o, d, tmax ? tmax[i] : inf_f(), skip ? skip[i] : -1, p, pos,
                                                   tb);
    } else {
      traverse2<HostCheckedLoads, STACK, false>(v, o, d, 0.0f, -1, p, pos, tb);
      h = p >= 0;
    }
    if (prim) prim[i] = any ? -1 : p;
    if (t) t[i] = any ? 0.0f : tb;
    if (hit) hit[i] = h ? 1 : 0;
  }
}

template <class T>
int fetch(std::vector<T>& h, const void* dev, size_t count) {
  h.resize(count > 0 ? count : 1);
  if (count == 0) return FIRE_OK;
  return cuda_check(cudaMemcpy(h.data(), dev, count * sizeof(T), cudaMemcpyDeviceToHost), "emulation copy");
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
  if (!s->built) return set_error(FIRE_ERR_NOT_BUILT, "emulation before build");
  if (!s->two_level) return set_error(FIRE_ERR_INVALID_ARG, "the emulation covers the two-level structure");
  *err_out = 0;
  if (int e = cuda_check(cudaDeviceSynchronize(), "sync")) return e;
  std::vector<Node4> tlas, blas;
  std::vector<float4> tris;
  std::vector<int32_t> roots;
  std::vector<float> xf;
  std::vector<TlasInfo> info;
  const size_t nb = (size_t)s->nbody;
  if (int e = fetch(info, s->tinfo, 1)) return e;
  if (int e = fetch(tlas, s->tlas, nb + 2)) return e;
  if (int e = fetch(blas, s->nodes4, (size_t)s->n4)) return e;
  if (int e = fetch(tris, s->tris, 3 * (size_t)s->nt)) return e;
  if (int e = fetch(roots, s->blas_root, nb)) return e;
  if (int e = fetch(xf, s->xf_buf[s->cur], 12 * nb)) return e;
  const TlasInfo ti = info[0];
  if (ti.err) *err_out |= kErrStack;
  g_regions.clear();
  g_regions.push_back({reinterpret_cast<const char*>(tlas.data()), sizeof(Node4) * (nb + 2)});
  g_regions.push_back({reinterpret_cast<const char*>(blas.data()), sizeof(Node4) * (size_t)s->n4});
  g_regions.push_back({reinterpret_cast<const char*>(tris.data()), sizeof(float4) * 3 * (size_t)s->nt});
  g_regions.push_back({reinterpret_cast<const char*>(roots.data()), 4 * nb});
  g_regions.push_back({reinterpret_cast<const char*>(xf.data()), 48 * nb});
  g_bad_loads = 0;
  uint32_t err = 0;
  Trace2View v{tlas.data(), std::min<int64_t>(ti.n, (int64_t)nb + 2), blas.data(), s->n4, tris.data(), s->nt,
               roots.data(), xf.data(), s->nbody, ti.span, s->iter_cap > 0 ? s->iter_cap : 2 * s->nt + 64, &err};
  switch (stack_for_height(stack_need(s), 0)) {
    case 32: run<32>(v, o3, d3, tmax, skip, n, any != 0, prim, t, hit); break;
    case 64: run<64>(v, o3, d3, tmax, skip, n, any != 0, prim, t, hit); break;
    default: run<128>(v, o3, d3, tmax, skip, n, any != 0, prim, t, hit); break;
  }
  g_regions.clear();
  *err_out |= err;
  if (g_bad_loads) *err_out |= 0x100u;
  return FIRE_OK;
}
