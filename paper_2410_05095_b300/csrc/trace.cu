// Per-frame render kernels:
//   k_primary      nearest hit per sample (replaces the rasterised main pass
//                  of §IV-A-1; 4-spp supersampling in the role of the MSAA
//                  of §IV-B-2); queues one shadow ray per lit light
//   k_shadow       the queued any-hit shadow rays (§IV-B-3), one visibility
//                  bit per sample and light
//   k_shade        per sample: Cook-Torrance GGX + Lambert shading of the
//                  visible lights (§IV-B-1), box-filter resolve of the
//                  pixel's samples (§IV-B-2); also shades a stored G-buffer
//                  with device parameters (fire_shade)
//   k_shade_bwd    its backward: dL/d(material params, light intensities)
// All of them are persistent: a grid of SMs x k blocks whose warps pull
// work (32-sample tasks, or 32 queued rays) from an atomic counter until
// the image is done.
#include <algorithm>
#include <cstdio>
#include <mutex>

#include "trace2.cuh"

namespace fire {
namespace {

// Two-level mode: the view of the traversal, and the frame's lift and slack
// from the top level's record (single level: from the tree's root box).
__device__ __forceinline__ Trace2View view2(const RenderArgs& a) {
  const TlasInfo ti = *a.tinfo;
  return Trace2View{a.tlas, ti.n, a.nodes4, a.n4, a.tris, a.nt, a.inst, kMaxTlasBodies, a.bxf, a.nbody, ti.span,
                    a.iter_cap, a.ctrl + 8};
}
__device__ __forceinline__ float frame_eps(const RenderArgs& a) {
  return a.tlas ? __ldg(&a.tinfo->eps) : scene_eps(a.nodes4, a.nt);
}

// Hit frame of the record's triangle (B = e1, C = e2): the single-level
// world record, or a two-level rest record turned by its body's rotation
// (body id in C.w).
__device__ __forceinline__ void hit_frame_of(const RenderArgs& a, float4 B, float4 C, float3 o, float3 d, float t,
                                             float eps, float3& n, float3& po) {
  if (a.tlas) {
    const uint32_t b = __float_as_uint(C.w);
    float m[12];
    const bool ok = b < (uint32_t)a.nbody;
#pragma unroll
    for (int k = 0; k < 12; ++k) m[k] = ok ? __ldg(a.bxf + 12 * b + k) : 0.0f;
    if (!ok) atomicOr(a.ctrl + 8, kErrCorrupt);
    hit_frame2(B, C, m, o, d, t, eps, n, po);
  } else {
    hit_frame(B, C, o, d, t, eps, n, po);
  }
}

// Nearest hit per sample; writes the sample's record (prim, t, cast bits,
// leaf position) and, for every light with n.l > 0 at the hit, a shadow ray
// (lifted origin, unit direction, range, sample|light) into the task's own
// 32 slots of that light's segment, lanes ranked by the popcount of the lower
// lanes, and the task's count of rays per light (no atomics: the queue is
// put in task order by k_qsum/k_qperm before the shadow pass).
// MODE 0: traversal.  After a raster pass (raster.cu): MODE 1 traverses only
// if that pass fell back, MODE 2 takes each sample's hit from its key
// otherwise; exactly one of the two does the work.
// Single level: 64 registers, 8 blocks of 128 per SM.  Two level: 72
// registers, 7 blocks (primary 1.81 -> 1.64 ms against 64 registers, which
// spill 206 B; 80 registers at 6 blocks give 1.72).
template <int STACK, int MODE, bool TWO>
__global__ void __launch_bounds__(128, TWO ? 7 : 8) k_primary(RenderArgs a, TaskGrid g, int ntasks, float4* __restrict__ jobs) {
  if (MODE != 0 && (MODE == 1) != (a.ctrl[kCtrlRasterFlag] != 0u)) return;
  const int lane = threadIdx.x & 31;
  const unsigned lower = (1u << lane) - 1u;
  TraceCtx c{a.nodes4, a.n4, TWO ? 0.0f : scene_span(a.nodes4, a.nt), a.tris, a.nt, a.iter_cap, a.ctrl + 8};
  Trace2View c2{};
  if (TWO) c2 = view2(a);
  const float eps = frame_eps(a);
  while (true) {
    int task = 0;
    if (lane == 0) task = atomicAdd(a.ctrl + 0, 1);
    task = __shfl_sync(kFull, task, 0);
    if (task >= ntasks) return;
    int x, y, k;
    const bool valid = task_sample(g, task, lane, x, y, k);
    int prim = -1, pos = -1;
    float t = inf_f();
    int64_t sid = 0;
    float3 o = f3(a.cam.ox, a.cam.oy, a.cam.oz), n = f3(0, 0, 0), po = f3(0, 0, 0);
    if (valid) {
      float3 d = cam_dir(a.cam, x, y, k);
      sid = ((int64_t)y * a.cam.W + x) * a.cam.spp + k;
      if (MODE == 2) {
        const unsigned long long key = a.rkeys[sid];
        if (key != ~0ull) {
          prim = (int)(uint32_t)key;
          t = __uint_as_float((uint32_t)(key >> 32));
          pos = __ldg(a.rank + prim);
        }
      } else if (TWO) {
        traverse2<DeviceLoads, STACK, false>(c2, o, d, 0.0f, -1, prim, pos, t);
      } else {
        trace_nearest<STACK>(c, o, d, prim, pos, t);
      }
      if (prim >= 0) {
        float4 B = __ldg(a.tris + 3 * (int64_t)pos + 1), C = __ldg(a.tris + 3 * (int64_t)pos + 2);
        hit_frame_of(a, B, C, o, d, t, eps, n, po);
        if (a.vnrm)
          n = shading_normal(SmoothCtx{a.vnrm, a.bxf, a.sidx, a.vbody}, pos, __ldg(a.tris + 3 * (int64_t)pos), B,
                             C, o, d, n);
      }
    }
    uint32_t cast = 0;
    for (int j = 0; j < a.lights.n; ++j) {
      float3 l = f3(0, 0, 0);
      float E, tmax = 0.0f;
      bool want = false;
      if (prim >= 0) {
        light_vec(a.lights, j, a.lights.I[j], po, l, E, tmax);
        want = dot3(n, l) > 0.0f;
      }
      unsigned m = __ballot_sync(kFull, want);
      if (lane == 0) a.qcnt[(int64_t)j * ntasks + task] = __popc(m);  // every task and light
      if (m == 0) continue;
      if (want) {
        cast |= 1u << (8 + j);
        int64_t slot = (int64_t)j * a.qseg + 32 * (int64_t)task + __popc(m & lower);
        jobs[2 * slot] = make_float4(po.x, po.y, po.z, tmax);
        jobs[2 * slot + 1] = make_float4(l.x, l.y, l.z, __int_as_float((int)(sid * 8 + j)));
      }
    }
    if (valid)
      reinterpret_cast<int4*>(a.g)[sid] = make_int4(prim, __float_as_int(t), (int)cast, pos);
  }
}

// Task order of the shadow queue.  Per light, k_qsum adds up the tasks' ray
// counts per block of kQTasks tasks; k_qperm (one block per kQTasks tasks) scans
// its tasks' counts, starts at the sum of the earlier blocks' totals, and
// writes its dense range in order, each position holding the sparse slot of
// its ray (a warp writes its tasks' ranges one task at a time, one lane per
// ray), so a warp of the shadow pass takes the rays of one or two
// neighbouring 4x2-pixel tasks; the last block writes the light's ray count
// to ctrl[24 + j].  Blocks of 256 threads: when the next frame's refit
// overlaps the render, they find room beside its blocks (1024-thread
// blocks waited 0.17 ms for whole SMs).
constexpr int kQTasks = 256;
constexpr int kQWarps = kQTasks / 32;

__global__ void __launch_bounds__(kQTasks) k_qsum(const int32_t* __restrict__ cnt, int32_t* __restrict__ bsum, int ntasks,
                                               int nblk) {
  __shared__ int32_t wsum[kQWarps];
  const int j = blockIdx.y, b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int t = b * kQTasks + tid;
  int32_t v = t < ntasks ? cnt[(int64_t)j * ntasks + t] : 0;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  if (lane == 0) wsum[w] = v;
  __syncthreads();
  if (w == 0) {
    int32_t y = lane < kQWarps ? wsum[lane] : 0;
    for (int o = 16; o > 0; o >>= 1) y += __shfl_xor_sync(kFull, y, o);
    if (lane == 0) bsum[(int64_t)j * nblk + b] = y;
  }
}

__global__ void __launch_bounds__(kQTasks) k_qperm(const int32_t* __restrict__ cnt, const int32_t* __restrict__ bsum,
                                                int32_t* __restrict__ perm, uint32_t* __restrict__ len, int ntasks,
                                                int nblk, int64_t qseg) {
  __shared__ int32_t wsum[kQWarps];
  __shared__ int32_t sbase;
  const int j = blockIdx.y, b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if (w == 0) {  // the earlier blocks' rays
    int32_t y = 0;
    for (int i = lane; i < b; i += 32) y += bsum[(int64_t)j * nblk + i];
    for (int o = 16; o > 0; o >>= 1) y += __shfl_xor_sync(kFull, y, o);
    if (lane == 0) sbase = y;
  }
  const int t = b * kQTasks + tid;
  const int32_t v = t < ntasks ? cnt[(int64_t)j * ntasks + t] : 0;
  int32_t x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  if (w == 0) {
    int32_t y = lane < kQWarps ? wsum[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t z = __shfl_up_sync(kFull, y, o);
      if (lane >= o) y += z;
    }
    if (lane < kQWarps) wsum[lane] = y;  // inclusive sums of the warps
  }
  __syncthreads();
  const int32_t total = wsum[kQWarps - 1], base = sbase;
  const int32_t excl = x - v + (w ? wsum[w - 1] : 0);
  int32_t* out = perm + (int64_t)j * qseg + base;
  // the warp's tasks with rays, one after another, each written by its lanes
  for (unsigned nz = __ballot_sync(kFull, v > 0); nz; nz &= nz - 1) {
    const int k = __ffs(nz) - 1;
    const int32_t c = __shfl_sync(kFull, v, k), o = __shfl_sync(kFull, excl, k);
    if (lane < c) out[o + lane] = 32 * (b * kQTasks + w * 32 + k) + lane;
  }
  if (b == nblk - 1 && tid == 0) len[j] = (uint32_t)(base + total);
}

// Shadow rays from the dense queue: one segment per light (light j's rays
// from j * qseg; lengths in ctrl[24 + j]), so a warp's 32 consecutive
// rays never mix lights (shadow 1.35 -> 1.33 ms on the 7.3M-triangle frame);
// each warp takes 32 consecutive rays of the segments laid end to end (all
// lanes busy until the tail); an unoccluded ray sets its light's bit in the
// sample's record.  (A lane-level ray pool -- refilling idle lanes
// every 16 node visits -- measured 7% slower: the idle lanes come from the
// branches inside each node step, not from rays of different lengths.)
// The single-level kernel is held to 56 registers (9 blocks of 128 per SM,
// no spills; 1.081 -> 1.062 ms against 62 registers and 8 blocks; 48
// registers spill and cost 1.19 ms).  The two-level kernel is held to 70
// registers (7 blocks per SM, no spills): its shadow pass went 1.91 -> 1.63
// ms against the uncapped 93 registers; 64 registers spill and give 1.71.
template <int STACK, bool TWO>
__global__ void __launch_bounds__(128, TWO ? 7 : 9) k_shadow(RenderArgs a, const float4* __restrict__ jobs,
                                                const int32_t* __restrict__ perm) {
  const int lane = threadIdx.x & 31;
  TraceCtx c{a.nodes4, a.n4, TWO ? 0.0f : scene_span(a.nodes4, a.nt), a.tris, a.nt, a.iter_cap, a.ctrl + 8};
  Trace2View c2{};
  if (TWO) c2 = view2(a);
  uint32_t cnt[8];
  uint32_t njobs = 0;
  for (int j = 0; j < 8; ++j) {
    cnt[j] = j < a.lights.n ? a.ctrl[kCtrlShadowLen + j] : 0u;
    njobs += cnt[j];
  }
  const int64_t seg = a.qseg;
  int4* rec = reinterpret_cast<int4*>(a.g);
  while (true) {
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(a.ctrl + 5, 32u);
    base = __shfl_sync(kFull, base, 0);
    if (base >= njobs) return;
    uint32_t jb = base + lane;
    if (jb < njobs) {
      uint32_t off = jb;
      int lj = 0;
      while (lj < 7 && off >= cnt[lj]) {
        off -= cnt[lj];
        ++lj;
      }
      const int64_t js = (int64_t)lj * seg + __ldg(perm + (int64_t)lj * seg + off);
      float4 A = jobs[2 * js], B = jobs[2 * js + 1];
      int sj = __float_as_int(B.w);
      int64_t sid = sj >> 3;
      int light = sj & 7;
      int skip = rec[sid].x;
      bool occ;
      if (TWO) {
        int prim, pos;
        float tb;
        occ = traverse2<DeviceLoads, STACK, true>(c2, f3(A.x, A.y, A.z), f3(B.x, B.y, B.z), A.w, skip, prim, pos, tb);
      } else {
        occ = trace_any<STACK>(c, f3(A.x, A.y, A.z), f3(B.x, B.y, B.z), A.w, skip);
      }
      if (!occ) atomicOr(reinterpret_cast<unsigned*>(&rec[sid].z), 1u << light);
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

// Shading + resolve of the samples' records, visibility read from the
// records (fire_render's last pass and fire_shade).  inten: device
// intensities or nullptr (the lights' own).  Held to 56 registers, 9 blocks
// of 128 per SM (the pass is latency-bound; 0.119 -> 0.114 ms on the
// 7.3M-triangle frame against 69 registers and 7 blocks; 64 registers:
// 0.117).
__global__ void __launch_bounds__(128, 9) k_shade(RenderArgs a, TaskGrid g, int ntasks, const float* inten) {
  const int lane = threadIdx.x & 31;
  const float eps = frame_eps(a);
  // tasks by a static warp stride (the work per task is even: no counter
  // round trip), the next task's record loaded before this task is shaded
  const int stride = (int)((gridDim.x * (int64_t)blockDim.x) >> 5);
  int task = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  int x = 0, y = 0, k = 0;
  bool valid = task < ntasks && task_sample(g, task, lane, x, y, k);
  int4 next = valid ? reinterpret_cast<const int4*>(a.g)[((int64_t)y * a.cam.W + x) * a.cam.spp + k]
                    : make_int4(-1, 0, 0, 0);
  for (; task < ntasks; task += stride) {
    const int4 rr = next;
    const int cx = x, cy = y, ck = k;
    const bool cvalid = valid;
    valid = task + stride < ntasks && task_sample(g, task + stride, lane, x, y, k);
    if (valid) next = reinterpret_cast<const int4*>(a.g)[((int64_t)y * a.cam.W + x) * a.cam.spp + k];
    float3 rad = f3(0.0f, 0.0f, 0.0f);
    int hit = 0;
    if (cvalid) {
      const int x = cx, y = cy, k = ck;
      int prim = rr.x, pos = rr.w;
      const uint32_t vis = (uint32_t)rr.z;
      if (prim >= 0) {
        hit = 1;
        float t = __int_as_float(rr.y);
        float3 o = f3(a.cam.ox, a.cam.oy, a.cam.oz);
        float3 d = cam_dir(a.cam, x, y, k);
        float4 B = __ldg(a.tris + 3 * (int64_t)pos + 1), C = __ldg(a.tris + 3 * (int64_t)pos + 2);
        float3 n, po;
        hit_frame_of(a, B, C, o, d, t, eps, n, po);
        if (a.vnrm)
          n = shading_normal(SmoothCtx{a.vnrm, a.bxf, a.sidx, a.vbody}, pos, __ldg(a.tris + 3 * (int64_t)pos), B,
                             C, o, d, n);
        float3 v = neg3(d);
        const float* mp = a.mats.p + 5 * (int64_t)__float_as_uint(B.w);
        float ar = __ldg(mp), ag = __ldg(mp + 1), ab = __ldg(mp + 2), rough = __ldg(mp + 3), metal = __ldg(mp + 4);
        for (int j = 0; j < a.lights.n; ++j) {
          float I = inten ? __ldg(inten + j) : a.lights.I[j];
          float3 l;
          float E, tmax;
          light_vec(a.lights, j, I, po, l, E, tmax);
          float ndl = dot3(n, l);
          if (!(ndl > 0.0f) || !((vis >> j) & 1u)) continue;
          float3 f = brdf(n, v, l, ar, ag, ab, rough, metal);
          float En = E * ndl;
          rad = f3(rad.x + f.x * En, rad.y + f.y * En, rad.z + f.z * En);
        }
      }
    }
    resolve_write(a, lane, cvalid, cx, cy, rad, hit);
  }
}

// Backward of k_shade for L(image): per sample, the upstream
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
// Per-sample terms, per-warp sums (shuffles; material terms per group of
// lanes sharing a material) and the block's sums of a few warp sums (shared
// atomics) are FP32; the sums over blocks are FP64: global atomics into
// `acc` (nmat*5 + nlights doubles, zero on entry), and the last block to
// finish adds `acc` into the FP32 outputs and zeroes it.
__global__ void __launch_bounds__(128, 8) k_shade_bwd(RenderArgs a, TaskGrid g, int ntasks, const float* inten,
                                                   const float* dL, float* dparams, float* dinten,
                                                   double* acc) {
  extern __shared__ float sacc[];  // [nmat*5 + nlights]
  __shared__ bool last_block;
  const int nm5 = a.mats.n * 5;
  const int nacc = nm5 + a.lights.n;
  for (int i = threadIdx.x; i < nacc; i += blockDim.x) sacc[i] = 0.0f;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const float eps = frame_eps(a);
  // tasks by a static warp stride, the next task's record loaded first (as
  // in k_shade)
  const int stride = (int)((gridDim.x * (int64_t)blockDim.x) >> 5);
  int task = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  int nx = 0, ny = 0, nk = 0;
  bool nvalid = task < ntasks && task_sample(g, task, lane, nx, ny, nk);
  int4 next = nvalid ? reinterpret_cast<const int4*>(a.g)[((int64_t)ny * a.cam.W + nx) * a.cam.spp + nk]
                     : make_int4(-1, 0, 0, 0);
  for (; task < ntasks; task += stride) {
    const int x = nx, y = ny, k = nk;
    const bool valid = nvalid;
    const int4 rr = next;
    nvalid = task + stride < ntasks && task_sample(g, task + stride, lane, nx, ny, nk);
    if (nvalid) next = reinterpret_cast<const int4*>(a.g)[((int64_t)ny * a.cam.W + nx) * a.cam.spp + nk];
    float gm[5] = {0, 0, 0, 0, 0};
    float gl[kMaxLights];
#pragma unroll
    for (int j = 0; j < kMaxLights; ++j) gl[j] = 0.0f;
    int mat = -1;
    if (valid) {
      if (rr.x >= 0) {
        float4 up4 = reinterpret_cast<const float4*>(dL)[(int64_t)y * a.cam.W + x];
        float inv_spp = 1.0f / (float)a.cam.spp;
        float up[3] = {up4.x * inv_spp, up4.y * inv_spp, up4.z * inv_spp};
        float3 o = f3(a.cam.ox, a.cam.oy, a.cam.oz);
        float3 d = cam_dir(a.cam, x, y, k);
        float4 B = __ldg(a.tris + 3 * (int64_t)rr.w + 1), C = __ldg(a.tris + 3 * (int64_t)rr.w + 2);
        float3 n, po;
        hit_frame_of(a, B, C, o, d, __int_as_float(rr.y), eps, n, po);
        if (a.vnrm)
          n = shading_normal(SmoothCtx{a.vnrm, a.bxf, a.sidx, a.vbody}, rr.w, __ldg(a.tris + 3 * (int64_t)rr.w), B,
                             C, o, d, n);
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
          float rdd = 1.0f / (s1 + nh2a2);
          float D = a2 * kInvPi * rdd * rdd;
          float dD_dr = (s1 - nh2a2) * kInvPi * (rdd * rdd * rdd) * (4.0f * r * r * r);
          float kk = (r + 1.0f) * (r + 1.0f) * 0.125f, dk_dr = (r + 1.0f) * 0.25f;
          float rgL = 1.0f / fmaf(nl, 1.0f - kk, kk), rgV = 1.0f / fmaf(nv, 1.0f - kk, kk);
          float vis = 0.25f * rgL * rgV;
          float dvis_dr = -vis * ((1.0f - nl) * rgL + (1.0f - nv) * rgV) * dk_dr;
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
            gm[ch] += u * I * dalb;
            gm[3] += u * I * dr;
            gm[4] += u * I * dm;
            gl[j] += u * f;
          }
        }
      }
    }
    // FP32 warp sums: the light terms over the whole warp, the material
    // terms over each group of lanes sharing a material (one pass per
    // distinct material); one shared atomic per sum, by one lane
    unsigned todo = __ballot_sync(kFull, mat >= 0);
    if (todo == 0) continue;
    for (int j = 0; j < a.lights.n; ++j) {
      float v = gl[j];
      for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
      if (lane == 0) atomicAdd(&sacc[nm5 + j], v);
    }
    while (todo) {
      const int leader = __ffs(todo) - 1;
      const int m = __shfl_sync(kFull, mat, leader);
      const bool mine = mat == m;
      todo &= ~__ballot_sync(kFull, mine);
      float v[5];
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        v[q] = mine ? gm[q] : 0.0f;
        for (int off = 16; off; off >>= 1) v[q] += __shfl_xor_sync(kFull, v[q], off);
      }
      if (lane == leader) {
#pragma unroll
        for (int q = 0; q < 5; ++q) atomicAdd(&sacc[5 * m + q], v[q]);
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nacc; i += blockDim.x)
    if (sacc[i] != 0.0f) atomicAdd(acc + i, (double)sacc[i]);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last_block = atomicAdd(a.ctrl + 3, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last_block) return;
  __threadfence();
  for (int i = threadIdx.x; i < nacc; i += blockDim.x) {
    double s = __ldcg(acc + i);
    acc[i] = 0.0;  // ready for the next call
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

template <int STACK, bool TWO>
int launch_render(fire_scene_s* s, const RenderArgs& a, const TaskGrid& g, int ntasks,
                  const fire_render_opts& o, bool raster, cudaStream_t st) {
  const int threads = 128;
  static int occ_p = 0, occ_s = 0, occ_r = 0;
  static std::once_flag once;
  std::call_once(once, [] {
    occ_p = occupancy_blocks(k_primary<STACK, 0, TWO>, 128, 0);
    occ_s = occupancy_blocks(k_shadow<STACK, TWO>, 128, 0);
    occ_r = occupancy_blocks(k_shade, 128, 0);
  });
  int sms = sm_count();
  // blocks_per_sm limits the primary pass only: a refit of the next frame
  // on another stream starts with this frame's render and overlaps its
  // primary pass; the shadow and resolve passes run at full occupancy
  // (pipelined frame7m: 3.01 ms with all three passes at 6 blocks per SM,
  // 2.90 ms with only the primary pass)
  int bp = o.blocks_per_sm > 0 ? o.blocks_per_sm : occ_p;
  int bs = occ_s;
  int br = occ_r;
  int gp = std::max(1, std::min(sms * bp, (ntasks + 3) / 4));
  // the shadow queue holds at most samples x lights rays; its length is only
  // known on the device, so the grid covers the worst case
  int64_t maxjobs = (int64_t)ntasks * 32 * std::max(1, a.lights.n);
  int gs = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * bs, (maxjobs + 127) / 128));
  int gr = std::max(1, std::min(sms * br, (ntasks + 3) / 4));
  prof_begin(s, kStagePrimary, st);
  if (raster) {
    RasterArgs r{a.tris, a.nt, a.nodes4, a.cam, a.row_begin, a.row_end, s->rkeys, s->rdirs, s->pieces,
                 (int64_t)s->pieces_n, s->graze, (int64_t)s->graze_n, a.ctrl};
    if (int e = raster_primary(s, r, st)) return e;
    RenderArgs ak = a;
    ak.rkeys = s->rkeys;
    ak.rank = s->rank;
    k_primary<STACK, 1, false><<<gp, threads, 0, st>>>(a, g, ntasks, s->jobs);
    k_primary<STACK, 2, false><<<gp, threads, 0, st>>>(ak, g, ntasks, s->jobs);
  } else {
    k_primary<STACK, 0, TWO><<<gp, threads, 0, st>>>(a, g, ntasks, s->jobs);
  }
  prof_end(s, kStagePrimary, st, raster ? (a.nt > 0 ? 6 : 3) : 1);
  if (a.lights.n > 0) {
    prof_begin(s, kStageQueue, st);
    const int nl = a.lights.n;
    const int nblk = (ntasks + kQTasks - 1) / kQTasks;
    int32_t* bsum = a.qcnt + (int64_t)nl * ntasks;
    k_qsum<<<dim3(nblk, nl), kQTasks, 0, st>>>(a.qcnt, bsum, ntasks, nblk);
    k_qperm<<<dim3(nblk, nl), kQTasks, 0, st>>>(a.qcnt, bsum, s->qperm, a.ctrl + kCtrlShadowLen, ntasks, nblk,
                                                a.qseg);
    prof_end(s, kStageQueue, st, 2);
    prof_begin(s, kStageShadow, st);
    k_shadow<STACK, TWO><<<gs, threads, 0, st>>>(a, s->jobs, s->qperm);
    prof_end(s, kStageShadow, st);
  }
  prof_begin(s, kStageResolve, st);
  k_shade<<<gr, threads, 0, st>>>(a, g, ntasks, nullptr);
  prof_end(s, kStageResolve, st);
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
  // task counters, queue length and queue cursor (the error word at [8] stays)
  if (int e = cuda_check(cudaMemsetAsync(a.ctrl, 0, 8 * 4, st), "memset")) return e;
  // per-light shadow-queue lengths
  if (int e = cuda_check(cudaMemsetAsync(a.ctrl + kCtrlShadowLen, 0, 8 * 4, st), "memset")) return e;
  // primary pass: traversal unless the raster pass is asked for (it
  // measured slower on the scenes of sub-pixel triangles this library is
  // timed on, and equal at best elsewhere)
  bool raster = (o.flags & FIRE_RENDER_RASTER_PRIMARY) != 0;
  raster = raster && s->rkeys && s->pieces && s->graze && a.cam.W < 65536 && a.cam.H < 65536;
  s->rendered = true;
  s->last_raster = raster;
  s->last_qseg = a.qseg;
  s->last_nlights = a.lights.n;
  if (a.tlas) {  // two-level (no raster pass: fire_render refuses the flag)
    switch (stack_for_height(stack_need(s), o.stack_depth)) {
      case 8: return launch_render<8, true>(s, a, g, ntasks, o, false, st);
      case 32: return launch_render<32, true>(s, a, g, ntasks, o, false, st);
      case 64: return launch_render<64, true>(s, a, g, ntasks, o, false, st);
      default: return launch_render<128, true>(s, a, g, ntasks, o, false, st);
    }
  }
  switch (stack_for_height(stack_need(s), o.stack_depth)) {
    case 8: return launch_render<8, false>(s, a, g, ntasks, o, raster, st);
    case 32: return launch_render<32, false>(s, a, g, ntasks, o, raster, st);
    case 64: return launch_render<64, false>(s, a, g, ntasks, o, raster, st);
    default: return launch_render<128, false>(s, a, g, ntasks, o, raster, st);
  }
}

int shade_from_gbuffer(fire_scene_s* s, const RenderArgs& a, const float* inten, cudaStream_t st) {
  TaskGrid g = make_grid(a.cam.W, 0, a.cam.H, a.cam.spp);
  int ntasks = g.tiles_x * g.tiles_y;
  if (ntasks == 0) return FIRE_OK;
  if (int e = cuda_check(cudaMemsetAsync(a.ctrl, 0, 4 * 4, st), "memset")) return e;
  int grid = std::max(1, std::min(sm_count() * 8, (ntasks + 3) / 4));
  prof_begin(s, kStageShadeGbuf, st);
  k_shade<<<grid, 128, 0, st>>>(a, g, ntasks, inten);
  prof_end(s, kStageShadeGbuf, st);
  return cuda_check(cudaGetLastError(), "k_shade_gbuf");
}

int shade_backward(fire_scene_s* s, const RenderArgs& a, const float* inten, const float* dL, float* dparams,
                   float* dinten, cudaStream_t st) {
  TaskGrid g = make_grid(a.cam.W, 0, a.cam.H, a.cam.spp);
  int ntasks = g.tiles_x * g.tiles_y;
  if (ntasks == 0) return FIRE_OK;
  const int nacc = a.mats.n * 5 + a.lights.n;
  size_t smem = sizeof(float) * nacc;
  if (smem > 48 * 1024) {
    if (int e = cuda_check(cudaFuncSetAttribute(k_shade_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                           "smem attr"))
      return e;
  }
  int grid = std::max(1, std::min(sm_count() * occupancy_blocks(k_shade_bwd, 128, smem), (ntasks + 3) / 4));
  size_t need = (size_t)nacc;
  if (s->bwd_partials_n < need) {
    if (s->bwd_partials) cudaFree(s->bwd_partials);
    s->bwd_partials = nullptr;
    s->bwd_partials_n = 0;
    if (cudaError_t e = dev_alloc((void**)&s->bwd_partials, need * sizeof(double), &s->bytes))
      return cuda_check(e, "backward accumulator");
    if (int e = cuda_check(cudaMemsetAsync(s->bwd_partials, 0, need * sizeof(double), st), "memset")) return e;
    s->bwd_partials_n = need;
  }
  if (int e = cuda_check(cudaMemsetAsync(a.ctrl, 0, 4 * 4, st), "memset")) return e;
  prof_begin(s, kStageBackward, st);
  k_shade_bwd<<<grid, 128, smem, st>>>(a, g, ntasks, inten, dL, dparams, dinten, s->bwd_partials);
  prof_end(s, kStageBackward, st);
  return cuda_check(cudaGetLastError(), "k_shade_bwd");
}

// The same backward kernel on caller-provided scratch: `acc` holds
// nmat*5 + nlights doubles (at most 6144, so the block's copy fits the
// default shared memory) and a.ctrl at least 4 counter words, all zero on
// entry.  Nothing is allocated here.
int shade_backward_on(const RenderArgs& a, const float* inten, const float* dL, float* dparams, float* dinten,
                      double* acc, cudaStream_t st) {
  TaskGrid g = make_grid(a.cam.W, 0, a.cam.H, a.cam.spp);
  int ntasks = g.tiles_x * g.tiles_y;
  if (ntasks == 0) return FIRE_OK;
  const int nacc = a.mats.n * 5 + a.lights.n;
  if (nacc > 6144) return set_error(FIRE_ERR_INVALID_ARG, "too many parameters for the scratch backward");
  int grid = std::max(1, std::min(sm_count() * occupancy_blocks(k_shade_bwd, 128, sizeof(float) * nacc),
                                  (ntasks + 3) / 4));
  k_shade_bwd<<<grid, 128, sizeof(float) * nacc, st>>>(a, g, ntasks, inten, dL, dparams, dinten, acc);
  return cuda_check(cudaGetLastError(), "k_shade_bwd");
}

}  // namespace fire
