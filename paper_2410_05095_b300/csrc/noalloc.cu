// Allocation-free entry point: the shading backward with its scratch memory
// (block counters and the FP64 gradient accumulator) in a fixed array that
// is part of the library image instead of memory the library allocates.
//
// Who needs it: callers that cannot call cudaMalloc while they run -- for
// example a frame loop whose device memory is fixed at start-up and may not
// grow, or a host application that must not pay the device-wide
// synchronisation a first cudaMalloc/cudaFree can cause in the middle of a
// frame.  They pass inputs and outputs as usual; this call allocates nothing
// on the device or the host.
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "fire_internal.cuh"

namespace fire {
namespace {

constexpr int kNoAllocMaxParams = 4096;  // nmat * 5 + nlights
constexpr size_t kNoAllocCtrlBytes = 256;

// Scratch: 256 B of counters, then kNoAllocMaxParams doubles (33,024 B in
// all).  Every GPU that loads the library holds this array until the process
// exits.  All calls share it: calls whose work overlaps on the GPU (on
// different streams, or from different host threads) race on it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocCtrlBytes + 8 * kNoAllocMaxParams];

std::mutex g_scratch_mu;
constexpr int kMaxDevices = 256;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch on the current device.  In host code the
// array's name only stands in for the symbol, so the address is looked up
// once per device (with that device current) and cached.  The first lookup
// on a device can load this file's module there (CUDA loads modules lazily
// by default), which is when the driver allocates the array; a cached
// address goes stale if the process resets the device (cudaDeviceReset).
int scratch_address(unsigned char** out) {
  int dev = 0;
  if (cudaError_t e = cudaGetDevice(&dev)) return cuda_check(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return set_error(FIRE_ERR_INVALID_ARG, "device index out of range");
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_check(e, "cudaGetSymbolAddress(scratch)");
    g_scratch_ptr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_scratch_ptr[dev]);
  return FIRE_OK;
}

bool finite3f(const float* v) { return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]); }

}  // namespace
}  // namespace fire

using namespace fire;

extern "C" int fire_shade_backward_noalloc(fire_scene s, const fire_gbuffer_rec* gbuf, const fire_camera* cam,
                                           const fire_light* lights, int32_t nlights, const float* params,
                                           const float* inten, const float* dL_drgba, float* dparams,
                                           float* dinten, void* stream) {
  set_error(FIRE_OK, "");
  if (!s) return set_error(FIRE_ERR_INVALID_ARG, "NULL scene");
  if (!s->built) return set_error(FIRE_ERR_NOT_BUILT, "backward before build");
  if (!cam || cam->width <= 0 || cam->height <= 0 || (cam->spp != 1 && cam->spp != 4) ||
      (int64_t)cam->width * cam->height * cam->spp >= ((int64_t)1 << 28) || !finite3f(cam->pos) ||
      !finite3f(cam->target) || !finite3f(cam->up) || !(cam->vfov_deg > 0 && cam->vfov_deg < 180))
    return set_error(FIRE_ERR_INVALID_ARG, "invalid camera");
  if (!gbuf || !params || !dL_drgba || !dparams || (nlights > 0 && (!inten || !dinten)))
    return set_error(FIRE_ERR_INVALID_ARG, "NULL buffer");
  const int64_t nacc = (int64_t)s->nmat * 5 + nlights;
  if (nacc > kNoAllocMaxParams)
    return set_error(FIRE_ERR_INVALID_ARG, "nmat*5 + nlights = " + std::to_string(nacc) +
                                               " exceeds the allocation-free maximum of " +
                                               std::to_string(kNoAllocMaxParams));
  RenderArgs a;
  memset(&a, 0, sizeof(a));
  if (int e = make_lights(lights, nlights, &a.lights)) return e;
  a.nodes4 = s->nodes4;
  a.n4 = s->n4;
  a.tris = s->tris;
  a.nt = s->nt;
  a.cam = make_cam(*cam);
  a.mats.p = params;
  a.mats.n = s->nmat;
  a.row_begin = 0;
  a.row_end = cam->height;
  a.iter_cap = 2 * s->nt + 64;
  set_smooth_args(&a, s);
  set_level_args(&a, s);
  a.g = const_cast<fire_gbuffer_rec*>(gbuf);
  unsigned char* base = nullptr;
  if (int e = scratch_address(&base)) return e;
  uint32_t* ctrl = reinterpret_cast<uint32_t*>(base);
  double* acc = reinterpret_cast<double*>(base + kNoAllocCtrlBytes);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // the counters and the accumulator must start at zero (the array keeps the
  // last call's contents)
  if (int e = cuda_check(cudaMemsetAsync(ctrl, 0, kNoAllocCtrlBytes, st), "clear scratch")) return e;
  if (int e = cuda_check(cudaMemsetAsync(acc, 0, sizeof(double) * nacc, st), "clear scratch")) return e;
  a.ctrl = ctrl;
  // later calls that default to the scene's last stream (fire_debug_dump,
  // fire_sync_status) see this one, as after fire_shade_backward
  s->last_stream = st;
  frame_acquire(s, st);
  // timed as the backward stage, as in fire_shade_backward (the profiler's
  // events are host objects: no device memory)
  prof_begin(s, kStageBackward, st);
  const int e = shade_backward_on(a, inten, dL_drgba, dparams, dinten, acc, st);
  prof_end(s, kStageBackward, st);
  frame_release(s, st);
  return e;
}
