// Per-frame render kernels:
//   k_primary      nearest hit per sample (replaces the rasterised main pass
//                  of §IV-A-1; 4-spp supersampling in the role of the MSAA
//                  of §IV-B-2)
//   k_shade        per sample: any-hit shadow ray per light (§IV-B-3), Cook-
//                  Torrance GGX + Lambert shading (§IV-B-1), box-filter
//                  resolve of the pixel's samples (§IV-B-2)
//   k_shade_gbuf   shading of a stored G-buffer with device parameters
//   k_shade_bwd    its backward: dL/d(material params, light intensities)
// All of them are persistent: a grid of SMs x k blocks whose warps pull
// 32-sample tasks from an atomic counter until the image is done.
#include <algorithm>
#include <cstdio>
#include <mutex>

#include "trace_device.cuh"

namespace fire {
namespace {

template <int STACK>
__global__ void __launch_bounds__(128) k_primary(RenderArgs a, TaskGrid g, int ntasks) {
  const int lane = threadIdx.x & 31;
  TraceCtx c{a.nodes, a.tris, a.nt, a.iter_cap, a.ctrl + 8};
  while (true) {
    int task = 0;
    if (lane == 0) task = atomicAdd(a.ctrl + 0, 1);
    task = __shfl_sync(kFull, task, 0);
    if (task >= ntasks) return;
    int x, y, k;
    if (task_sample(g, task, lane, x, y, k)) {
      float3 o = f3(a.cam.ox, a.cam.oy, a.cam.oz);
      float3 d = cam_dir(a.cam, x, y, k);
      int prim, pos;
      float t;
      trace_nearest<STACK>(c, o, d, prim, pos, t);
      int64_t sid = ((int64_t)y * a.cam.W + x) * a.cam.spp + k;
      fire_gbuffer_rec r;
      r.prim = prim;
      r.t = t;
      r.vis = 0;
      r.pad = (uint32_t)pos;
      reinterpret_cast<int4*>(a.g)[sid] = *reinterpret_cast<int4*>(&r);
    }
  }
}

// Sum the spp samples of each pixel in sample order (lanes 4q..4q+3 for
// spp 4), divide by spp, write rgba (alpha = hit fraction).
__device__ __forceinline__ void resolve_write(const RenderArgs& a, int lane, bool valid, int x, int y,
                                              float3 rad, int hit) {
  if (a.cam.spp == 4) {
    int base = lane & ~3;
    float3 acc = f3(0.0f, 0.0f, 0.0f);
    int hits = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float rx = __shfl_sync(kFull, rad.x, base + k), ry = __shfl_sync(kFull, rad.y, base + k),
            rz = __shfl_sync(kFull, rad.z, base + k);
      acc = f3(acc.x + rx, acc.y + ry, acc.z + rz);
      hits += __shfl_sync(kFull, hit, base + k);
    }
    if (valid && (lane & 3) == 0)
      reinterpret_cast<float4*>(a.out)[(int64_t)y * a.cam.W + x] =
          make_float4(acc.x / 4.0f, acc.y / 4.0f, acc.z / 4.0f, (float)hits / 4.0f);
  } else if (valid) {
    float3 acc = f3(0.0f + rad.x, 0.0f + rad.y, 0.0f + rad.z);
    reinterpret_cast<float4*>(a.out)[(int64_t)y * a.cam.W + x] = make_float4(acc.x, acc.y, acc.z, (float)hit);
  }
}

// TRACE: cast the shadow rays (fire_render); otherwise read visibility from
// the G-buffer (fire_shade).  inten: device intensities or nullptr.
template <int STACK, bool TRACE>
__global__ void __launch_bounds__(128) k_shade(RenderArgs a, TaskGrid g, int ntasks, const float* inten) {
  const int lane = threadIdx.x & 31;
  TraceCtx c{a.nodes, a.tris, a.nt, a.iter_cap, a.ctrl + 8};
  const float eps = scene_eps(a.nodes, a.nt);
  while (true) {
    int task = 0;
    if (lane == 0) task = atomicAdd(a.ctrl + 1, 1);
    task = __shfl_sync(kFull, task, 0);
    if (task >= ntasks) return;
    int x, y, k;
    bool valid = task_sample(g, task, lane, x, y, k);
    float3 rad = f3(0.0f, 0.0f, 0.0f);
    int hit = 0;
    if (valid) {
      int64_t sid = ((int64_t)y * a.cam.W + x) * a.cam.spp + k;
      int4 rr = reinterpret_cast<const int4*>(a.g)[sid];
      int prim = rr.x, pos = rr.w;
      uint32_t vis = TRACE ? 0u : (uint32_t)rr.z;
      if (prim >= 0) {
        hit = 1;
        float t = __int_as_float(rr.y);
        float3 o = f3(a.cam.ox, a.cam.oy, a.cam.oz);
        float3 d = cam_dir(a.cam, x, y, k);
        float4 B = __ldg(a.tris + 3 * (int64_t)pos + 1), C = __ldg(a.tris + 3 * (int64_t)pos + 2);
        float3 n, po;
        hit_frame(B, C, o, d, t, eps, n, po);
        float3 v = neg3(d);
        const float* mp = a.mats.p + 5 * (int64_t)__float_as_uint(B.w);
        float ar = __ldg(mp), ag = __ldg(mp + 1), ab = __ldg(mp + 2), rough = __ldg(mp + 3), metal = __ldg(mp + 4);
        for (int j = 0; j < a.lights.n; ++j) {
          float I = inten ? __ldg(inten + j) : a.lights.I[j];
          float3 l;
          float E, tmax;
          light_vec(a.lights, j, I, po, l, E, tmax);
          float ndl = dot3(n, l);
          if (!(ndl > 0.0f)) continue;
          if (TRACE) {
            vis |= 1u << (8 + j);
            if (trace_any<STACK>(c, po, l, tmax, prim)) continue;
            vis |= 1u << j;
          } else if (!((vis >> j) & 1u)) {
            continue;
          }
          float3 f = brdf(n, v, l, ar, ag, ab, rough, metal);
          float En = E * ndl;
          rad = f3(rad.x + f.x * En, rad.y + f.y * En, rad.z + f.z * En);
        }
      }
      if (TRACE && a.write_vis) reinterpret_cast<int4*>(a.g)[sid].z = (int)vis;
    }
    resolve_write(a, lane, valid, x, y, rad, hit);
  }
}

// Backward of k_shade<.., false> for L(image): per sample, the upstream
// gradient of the pixel divided by spp, chained through
//   rad_c = sum_j I_j g_j (n.l_j) f_c(albedo, r, m)
// with g_j = 1/d^2 (point) or 1.  Derivatives of f_c (a = r^2, a2 = a^2,
// dd = (1-nh)(1+nh) + nh^2 a2, the form of nh^2 (a2-1) + 1 without
// cancellation near the highlight peak):
//   dD/dr   = ((1-nh)(1+nh) - a2 nh^2) / (pi dd^3) * 4 r^3
//   dvis/dr = -vis ((1 - nl)/gl + (1 - nv)/gv) (r + 1)/4
//   df/dalb = (1-F)(1-m)/pi + (D vis - (1-m) alb/pi)(1 - w5) m
//   df/dm   = (D vis - (1-m) alb/pi)(1 - w5)(alb - 0.04) - (1-F) alb/pi
//   df/dr   = F (dD/dr vis + D dvis/dr)
// Per-sample terms are FP32; sums are FP64: per warp (shuffles) when the
// warp shares one material, else shared-memory atomics, then each block
// stores its partials and the last block to finish adds them in block order
// (deterministic) into the FP32 outputs.
__global__ void __launch_bounds__(128) k_shade_bwd(RenderArgs a, TaskGrid g, int ntasks, const float* inten,
                                                   const float* dL, float* dparams, float* dinten,
                                                   double* partials) {
  extern __shared__ double sacc[];  // [nmat*5 + nlights]
  __shared__ bool last_block;
  const int nm5 = a.mats.n * 5;
  const int nacc = nm5 + a.lights.n;
  for (int i = threadIdx.x; i < nacc; i += blockDim.x) sacc[i] = 0.0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const float eps = scene_eps(a.nodes, a.nt);
  while (true) {
    int task = 0;
    if (lane == 0) task = atomicAdd(a.ctrl + 2, 1);
    task = __shfl_sync(kFull, task, 0);
    if (task >= ntasks) break;
    int x, y, k;
    bool valid = task_sample(g, task, lane, x, y, k);
    double gm[5] = {0, 0, 0, 0, 0};
    double gl[kMaxLights];
#pragma unroll
    for (int j = 0; j < kMaxLights; ++j) gl[j] = 0.0;
    int mat = -1;
    if (valid) {
      int64_t sid = ((int64_t)y * a.cam.W + x) * a.cam.spp + k;
      int4 rr = reinterpret_cast<const int4*>(a.g)[sid];
      if (rr.x >= 0) {
        float4 up4 = reinterpret_cast<const float4*>(dL)[(int64_t)y * a.cam.W + x];
        float inv_spp = 1.0f / (float)a.cam.spp;
        float up[3] = {up4.x * inv_spp, up4.y * inv_spp, up4.z * inv_spp};
        float3 o = f3(a.cam.ox, a.cam.oy, a.cam.oz);
        float3 d = cam_dir(a.cam, x, y, k);
        float4 B = __ldg(a.tris + 3 * (int64_t)rr.w + 1), C = __ldg(a.tris + 3 * (int64_t)rr.w + 2);
        float3 n, po;
        hit_frame(B, C, o, d, __int_as_float(rr.y), eps, n, po);
        float3 v = neg3(d);
        mat = (int)__float_as_uint(B.w);
        const float* mp = a.mats.p + 5 * (int64_t)mat;
        float alb[3] = {__ldg(mp), __ldg(mp + 1), __ldg(mp + 2)};
        float r = __ldg(mp + 3), m = __ldg(mp + 4);
        for (int j = 0; j < a.lights.n; ++j) {
          if (!((rr.z >> j) & 1)) continue;
          float I = __ldg(inten + j);
          float3 l;
          float E, tmax;
          light_vec(a.lights, j, 1.0f, po, l, E, tmax);  // E = g_j here
          float ndl = dot3(n, l);
          if (!(ndl > 0.0f)) continue;
          float3 h = normalize3(add3(l, v));
          float nl = fmaxf(ndl, 0.0f), nv = fmaxf(dot3(n, v), 0.0f);
          float nh = fmaxf(dot3(n, h), 0.0f), vh = fmaxf(dot3(v, h), 0.0f);
          float aa = r * r, a2 = aa * aa;
          float s1 = (1.0f - nh) * (1.0f + nh), nh2a2 = (nh * nh) * a2;
          float dd = s1 + nh2a2;
          float D = a2 / ((kPi * dd) * dd);
          float dD_dr = (s1 - nh2a2) / (kPi * dd * dd * dd) * (4.0f * r * r * r);
          float kk = (r + 1.0f) * (r + 1.0f) * 0.125f, dk_dr = (r + 1.0f) * 0.25f;
          float gL = fmaf(nl, 1.0f - kk, kk), gV = fmaf(nv, 1.0f - kk, kk);
          float vis = 0.25f / (gL * gV);
          float dvis_dr = -vis * ((1.0f - nl) / gL + (1.0f - nv) / gV) * dk_dr;
          float w = 1.0f - vh, w5 = (w * w) * (w * w) * w;
          float wI = E * ndl;  // g_j (n.l)
#pragma unroll
          for (int ch = 0; ch < 3; ++ch) {
            float F0 = fmaf(m, alb[ch] - 0.04f, 0.04f);
            float F = fmaf(1.0f - F0, w5, F0);
            float dfdF = D * vis - (1.0f - m) * alb[ch] * kInvPi;
            float f = (1.0f - F) * (1.0f - m) * alb[ch] * kInvPi + D * vis * F;
            float dalb = (1.0f - F) * (1.0f - m) * kInvPi + dfdF * (1.0f - w5) * m;
            float dm = dfdF * (1.0f - w5) * (alb[ch] - 0.04f) - (1.0f - F) * alb[ch] * kInvPi;
            float dr = F * (dD_dr * vis + D * dvis_dr);
            float u = up[ch] * wI;
            gm[ch] += (double)(u * I * dalb);
            gm[3] += (double)(u * I * dr);
            gm[4] += (double)(u * I * dm);
            gl[j] += (double)(u * f);
          }
        }
      }
    }
    // warp aggregation when the whole warp shares one material
    unsigned peers = __match_any_sync(kFull, mat);
    if (peers == kFull) {
#pragma unroll
      for (int q = 0; q < 5; ++q)
        for (int off = 16; off; off >>= 1) gm[q] += __shfl_xor_sync(kFull, gm[q], off);
      for (int j = 0; j < a.lights.n; ++j)
        for (int off = 16; off; off >>= 1) gl[j] += __shfl_xor_sync(kFull, gl[j], off);
      if (lane == 0 && mat >= 0) {
#pragma unroll
        for (int q = 0; q < 5; ++q) atomicAdd(&sacc[5 * mat + q], gm[q]);
        for (int j = 0; j < a.lights.n; ++j) atomicAdd(&sacc[nm5 + j], gl[j]);
      }
    } else if (mat >= 0) {
#pragma unroll
      for (int q = 0; q < 5; ++q) atomicAdd(&sacc[5 * mat + q], gm[q]);
      for (int j = 0; j < a.lights.n; ++j) atomicAdd(&sacc[nm5 + j], gl[j]);
    }
  }
  __syncthreads();
  double* part = partials + (int64_t)blockIdx.x * nacc;
  for (int i = threadIdx.x; i < nacc; i += blockDim.x) part[i] = sacc[i];
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last_block = atomicAdd(a.ctrl + 3, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last_block) return;
  __threadfence();
  for (int i = threadIdx.x; i < nacc; i += blockDim.x) {
    double s = 0.0;
    for (unsigned b = 0; b < gridDim.x; ++b) s += __ldcg(partials + (int64_t)b * nacc + i);
    float* o = i < nm5 ? dparams + i : dinten + (i - nm5);
    *o = *o + (float)s;
  }
}

// -- launch helpers ----------------------------------------------------------
template <typename K>
int occupancy_blocks(K kernel, int threads, size_t smem) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem) != cudaSuccess || n < 1) n = 1;
  return n;
}

template <int STACK>
int launch_render(fire_scene_s* s, const RenderArgs& a, const TaskGrid& g, int ntasks,
                  const fire_render_opts& o, cudaStream_t st) {
  const int threads = 128;
  static int occ_p = 0, occ_s = 0;
  static std::once_flag once;
  std::call_once(once, [] {
    occ_p = occupancy_blocks(k_primary<STACK>, 128, 0);
    occ_s = occupancy_blocks(k_shade<STACK, true>, 128, 0);
  });
  int sms = sm_count();
  int bp = o.blocks_per_sm > 0 ? o.blocks_per_sm : occ_p;
  int bs = o.blocks_per_sm > 0 ? o.blocks_per_sm : occ_s;
  int gp = std::max(1, std::min(sms * bp, (ntasks + 3) / 4));
  int gs = std::max(1, std::min(sms * bs, (ntasks + 3) / 4));
  prof_begin(s, kStagePrimary, st);
  k_primary<STACK><<<gp, threads, 0, st>>>(a, g, ntasks);
  prof_end(s, kStagePrimary, st);
  prof_begin(s, kStageShade, st);
  k_shade<STACK, true><<<gs, threads, 0, st>>>(a, g, ntasks, nullptr);
  prof_end(s, kStageShade, st);
  return cuda_check(cudaGetLastError(), "render kernels");
}

}  // namespace

int stack_for_height(int height, int requested) {
  int need = requested > 0 ? requested : height;
  if (need <= 8) return 8;  // only reachable through the shallow-stack test hook
  if (need <= 32) return 32;
  if (need <= 64) return 64;
  return 128;
}

int render_frame(fire_scene_s* s, const RenderArgs& a, const fire_render_opts& o, cudaStream_t st) {
  TaskGrid g = make_grid(a.cam.W, a.row_begin, a.row_end, a.cam.spp);
  int ntasks = g.tiles_x * g.tiles_y;
  if (ntasks == 0) return FIRE_OK;
  if (int e = cuda_check(cudaMemsetAsync(a.ctrl, 0, 4 * 4, st), "memset")) return e;
  switch (stack_for_height(s->height, o.stack_depth)) {
    case 8: return launch_render<8>(s, a, g, ntasks, o, st);
    case 32: return launch_render<32>(s, a, g, ntasks, o, st);
    case 64: return launch_render<64>(s, a, g, ntasks, o, st);
    default: return launch_render<128>(s, a, g, ntasks, o, st);
  }
}

int shade_from_gbuffer(fire_scene_s* s, const RenderArgs& a, const float* inten, cudaStream_t st) {
  TaskGrid g = make_grid(a.cam.W, 0, a.cam.H, a.cam.spp);
  int ntasks = g.tiles_x * g.tiles_y;
  if (ntasks == 0) return FIRE_OK;
  if (int e = cuda_check(cudaMemsetAsync(a.ctrl, 0, 4 * 4, st), "memset")) return e;
  int grid = std::max(1, std::min(sm_count() * 8, (ntasks + 3) / 4));
  prof_begin(s, kStageShadeGbuf, st);
  k_shade<32, false><<<grid, 128, 0, st>>>(a, g, ntasks, inten);
  prof_end(s, kStageShadeGbuf, st);
  return cuda_check(cudaGetLastError(), "k_shade_gbuf");
}

int shade_backward(fire_scene_s* s, const RenderArgs& a, const float* inten, const float* dL, float* dparams,
                   float* dinten, cudaStream_t st) {
  TaskGrid g = make_grid(a.cam.W, 0, a.cam.H, a.cam.spp);
  int ntasks = g.tiles_x * g.tiles_y;
  if (ntasks == 0) return FIRE_OK;
  const int nacc = a.mats.n * 5 + a.lights.n;
  size_t smem = sizeof(double) * nacc;
  if (smem > 48 * 1024) {
    if (int e = cuda_check(cudaFuncSetAttribute(k_shade_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                           "smem attr"))
      return e;
  }
  int grid = std::max(1, std::min(sm_count() * 4, (ntasks + 3) / 4));
  size_t need = (size_t)grid * nacc;
  if (s->bwd_partials_n < need) {
    if (s->bwd_partials) cudaFree(s->bwd_partials);
    s->bwd_partials = nullptr;
    s->bwd_partials_n = 0;
    if (cudaError_t e = dev_alloc((void**)&s->bwd_partials, need * sizeof(double), &s->bytes))
      return cuda_check(e, "backward partials");
    s->bwd_partials_n = need;
  }
  if (int e = cuda_check(cudaMemsetAsync(a.ctrl, 0, 4 * 4, st), "memset")) return e;
  prof_begin(s, kStageBackward, st);
  k_shade_bwd<<<grid, 128, smem, st>>>(a, g, ntasks, inten, dL, dparams, dinten, s->bwd_partials);
  prof_end(s, kStageBackward, st);
  return cuda_check(cudaGetLastError(), "k_shade_bwd");
}

}  // namespace fire
