// Batched rendering: many cameras over many scenes (uneven triangle counts
// and resolutions) in three launches for the whole batch, replayed as one
// CUDA graph while the batch is unchanged:
//   k_bprimary  warps pull 32-sample tasks from one counter spanning every
//               camera's tiles (camera found by binary search over the task
//               prefix sums); nearest hit into one G-buffer indexed by a
//               global sample id; shadow rays appended to one dense queue
//   k_bshadow   the queue, 32 consecutive rays per warp (camera found from
//               the sample id), any-hit against that camera's scene
//   k_bresolve  shading + box resolve into each camera's image
// The per-sample arithmetic is the single-frame path's, so every image
// equals a separate fire_render bit for bit.  Threads per block, blocks per
// SM are chosen by timing candidates on the first call of each batch shape
// (autotuner), unless the caller fixes them.
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "trace_device.cuh"

namespace fire {
namespace {

struct BatchCam {
  const Node4* nodes4;
  int64_t n4;
  const float4* tris;
  int64_t nt;
  const float* mats;
  SmoothCtx sm;           // smooth shading inputs (sm.vnrm == nullptr: flat)
  float* out;
  uint32_t* err;          // the scene's sticky error word
  int64_t sample_base;    // first global sample id of this camera
  CamParams cam;
  LightParams lights;
  int task_begin;
  int pad;
};

__device__ __forceinline__ int find_task_cam(const BatchCam* __restrict__ cams, int ncams, int task) {
  int lo = 0, hi = ncams - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (cams[mid].task_begin <= task) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ int find_sample_cam(const BatchCam* __restrict__ cams, int ncams, int64_t sid) {
  int lo = 0, hi = ncams - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (cams[mid].sample_base <= sid) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Work shape chosen by the autotuner: log2 of the task width at 1 and 4 spp
// and the tasks a warp takes per atomic grab.
struct BatchShape {
  int lw1, lw4, grab;
};

template <int STACK>
__global__ void __launch_bounds__(128) k_bprimary(const BatchCam* __restrict__ cams, int ncams, int ntasks,
                                                  uint32_t* ctrl, int4* __restrict__ gbuf, float4* __restrict__ jobs,
                                                  int64_t cap, BatchShape sh) {
  const int lane = threadIdx.x & 31;
  const unsigned lower = (1u << lane) - 1u;
  int grabbed = 0, left = 0;
  while (true) {
    if (left == 0) {
      if (lane == 0) grabbed = atomicAdd(ctrl + 0, sh.grab);
      grabbed = __shfl_sync(kFull, grabbed, 0);
      left = sh.grab;
    }
    const int task = grabbed++;
    --left;
    if (task >= ntasks) return;
    const BatchCam& bc = cams[find_task_cam(cams, ncams, task)];
    TaskGrid g = make_grid_w(bc.cam.W, 0, bc.cam.H, bc.cam.spp, bc.cam.spp == 4 ? sh.lw4 : sh.lw1);
    int x, y, k;
    const bool valid = task_sample(g, task - bc.task_begin, lane, x, y, k);
    TraceCtx c{bc.nodes4, bc.n4, scene_span(bc.nodes4, bc.nt), bc.tris, bc.nt, cap, bc.err};
    const float eps = scene_eps(bc.nodes4, bc.nt);
    int prim = -1, pos = -1;
    float t = inf_f();
    int64_t sid = 0;
    float3 o = f3(bc.cam.ox, bc.cam.oy, bc.cam.oz), n = f3(0, 0, 0), po = f3(0, 0, 0);
    if (valid) {
      float3 d = cam_dir(bc.cam, x, y, k);
      trace_nearest<STACK>(c, o, d, prim, pos, t);
      sid = bc.sample_base + ((int64_t)y * bc.cam.W + x) * bc.cam.spp + k;
      if (prim >= 0) {
        float4 B = __ldg(bc.tris + 3 * (int64_t)pos + 1), C = __ldg(bc.tris + 3 * (int64_t)pos + 2);
        hit_frame(B, C, o, d, t, eps, n, po);
        if (bc.sm.vnrm) n = shading_normal(bc.sm, pos, __ldg(bc.tris + 3 * (int64_t)pos), B, C, o, d, n);
      }
    }
    uint32_t cast = 0;
    for (int j = 0; j < bc.lights.n; ++j) {
      float3 l = f3(0, 0, 0);
      float E, tmax = 0.0f;
      bool want = false;
      if (prim >= 0) {
        light_vec(bc.lights, j, bc.lights.I[j], po, l, E, tmax);
        want = dot3(n, l) > 0.0f;
      }
      unsigned m = __ballot_sync(kFull, want);
      if (m == 0) continue;
      uint32_t base = 0;
      if (lane == __ffs(m) - 1) base = atomicAdd(ctrl + 4, (uint32_t)__popc(m));
      base = __shfl_sync(kFull, base, __ffs(m) - 1);
      if (want) {
        cast |= 1u << (8 + j);
        int64_t slot = (int64_t)base + __popc(m & lower);
        jobs[2 * slot] = make_float4(po.x, po.y, po.z, tmax);
        jobs[2 * slot + 1] = make_float4(l.x, l.y, l.z, __int_as_float((int)(sid * 8 + j)));
      }
    }
    if (valid) gbuf[sid] = make_int4(prim, __float_as_int(t), (int)cast, pos);
  }
}

template <int STACK>
__global__ void __launch_bounds__(128) k_bshadow(const BatchCam* __restrict__ cams, int ncams, uint32_t* ctrl,
                                                 int4* gbuf, const float4* __restrict__ jobs, int64_t cap) {
  const int lane = threadIdx.x & 31;
  const uint32_t njobs = ctrl[4];
  while (true) {
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(ctrl + 5, 32u);
    base = __shfl_sync(kFull, base, 0);
    if (base >= njobs) return;
    uint32_t jb = base + lane;
    if (jb < njobs) {
      float4 A = jobs[2 * (int64_t)jb], B = jobs[2 * (int64_t)jb + 1];
      int sj = __float_as_int(B.w);
      int64_t sid = sj >> 3;
      const BatchCam& bc = cams[find_sample_cam(cams, ncams, sid)];
      TraceCtx c{bc.nodes4, bc.n4, scene_span(bc.nodes4, bc.nt), bc.tris, bc.nt, cap, bc.err};
      int skip = gbuf[sid].x;
      if (!trace_any<STACK>(c, f3(A.x, A.y, A.z), f3(B.x, B.y, B.z), A.w, skip))
        atomicOr(reinterpret_cast<unsigned*>(&gbuf[sid].z), 1u << (sj & 7));
    }
  }
}

__global__ void __launch_bounds__(128) k_bresolve(const BatchCam* __restrict__ cams, int ncams, int ntasks,
                                                  uint32_t* ctrl, const int4* __restrict__ gbuf, BatchShape sh) {
  const int lane = threadIdx.x & 31;
  int grabbed = 0, left = 0;
  while (true) {
    if (left == 0) {
      if (lane == 0) grabbed = atomicAdd(ctrl + 1, sh.grab);
      grabbed = __shfl_sync(kFull, grabbed, 0);
      left = sh.grab;
    }
    const int task = grabbed++;
    --left;
    if (task >= ntasks) return;
    const BatchCam& bc = cams[find_task_cam(cams, ncams, task)];
    TaskGrid g = make_grid_w(bc.cam.W, 0, bc.cam.H, bc.cam.spp, bc.cam.spp == 4 ? sh.lw4 : sh.lw1);
    int x, y, k;
    const bool valid = task_sample(g, task - bc.task_begin, lane, x, y, k);
    float3 rad = f3(0.0f, 0.0f, 0.0f);
    int hit = 0;
    if (valid) {
      const int64_t sid = bc.sample_base + ((int64_t)y * bc.cam.W + x) * bc.cam.spp + k;
      const int4 rr = gbuf[sid];
      if (rr.x >= 0) {
        hit = 1;
        const float eps = scene_eps(bc.nodes4, bc.nt);
        float3 o = f3(bc.cam.ox, bc.cam.oy, bc.cam.oz);
        float3 d = cam_dir(bc.cam, x, y, k);
        float4 B = __ldg(bc.tris + 3 * (int64_t)rr.w + 1), C = __ldg(bc.tris + 3 * (int64_t)rr.w + 2);
        float3 n, po;
        hit_frame(B, C, o, d, __int_as_float(rr.y), eps, n, po);
        if (bc.sm.vnrm) n = shading_normal(bc.sm, rr.w, __ldg(bc.tris + 3 * (int64_t)rr.w), B, C, o, d, n);
        float3 v = neg3(d);
        const float* mp = bc.mats + 5 * (int64_t)__float_as_uint(B.w);
        float ar = __ldg(mp), ag = __ldg(mp + 1), ab = __ldg(mp + 2), rough = __ldg(mp + 3), metal = __ldg(mp + 4);
        for (int j = 0; j < bc.lights.n; ++j) {
          if (!((rr.z >> j) & 1)) continue;
          float3 l;
          float E, tmax;
          light_vec(bc.lights, j, bc.lights.I[j], po, l, E, tmax);
          float ndl = dot3(n, l);
          if (!(ndl > 0.0f)) continue;
          float3 f = brdf(n, v, l, ar, ag, ab, rough, metal);
          float En = E * ndl;
          rad = f3(rad.x + f.x * En, rad.y + f.y * En, rad.z + f.z * En);
        }
      }
    }
    // resolve (same order as the single-frame path)
    if (bc.cam.spp == 4) {
      int base = lane & ~3;
      float3 acc = f3(0.0f, 0.0f, 0.0f);
      int hits = 0;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float rx = __shfl_sync(kFull, rad.x, base + q), ry = __shfl_sync(kFull, rad.y, base + q),
              rz = __shfl_sync(kFull, rad.z, base + q);
        acc = f3(acc.x + rx, acc.y + ry, acc.z + rz);
        hits += __shfl_sync(kFull, hit, base + q);
      }
      if (valid && (lane & 3) == 0)
        reinterpret_cast<float4*>(bc.out)[(int64_t)y * bc.cam.W + x] =
            make_float4(acc.x / 4.0f, acc.y / 4.0f, acc.z / 4.0f, (float)hits / 4.0f);
    } else if (valid) {
      reinterpret_cast<float4*>(bc.out)[(int64_t)y * bc.cam.W + x] =
          make_float4(0.0f + rad.x, 0.0f + rad.y, 0.0f + rad.z, (float)hit);
    }
  }
}

// Tile shapes: log2 task width at (1 spp, 4 spp): 8 x 4 / 4 x 2 pixels
// (the single-frame path's), 4 x 8 / 2 x 4, 16 x 2 / 8 x 1.
constexpr int kTileLw[3][2] = {{3, 2}, {2, 1}, {4, 3}};

struct TuneCfg {
  int threads = 128, bps = 0, stack = 64, tile = 0, grab = 1;
  BatchShape shape() const { return BatchShape{kTileLw[tile][0], kTileLw[tile][1], grab}; }
};

struct BatchCache {
  std::mutex mu;
  BatchCam* d_cams = nullptr;
  size_t cap_cams = 0;
  uint32_t* d_ctrl = nullptr;
  int4* d_gbuf = nullptr;
  size_t cap_samples = 0;
  float4* d_jobs = nullptr;
  size_t cap_jobs = 0;
  std::vector<unsigned char> last_bytes;
  // everything the captured graph bakes in besides the descriptor contents
  struct Key {
    TuneCfg cfg;
    int ncams = 0, ntasks = 0;
    int64_t maxjobs = 0, cap = 0;
    const void* ptrs[4] = {nullptr, nullptr, nullptr, nullptr};
    bool operator==(const Key& k) const {
      return cfg.threads == k.cfg.threads && cfg.bps == k.cfg.bps && cfg.stack == k.cfg.stack &&
             cfg.tile == k.cfg.tile && cfg.grab == k.cfg.grab && ncams == k.ncams && ntasks == k.ntasks &&
             maxjobs == k.maxjobs && cap == k.cap && memcmp(ptrs, k.ptrs, sizeof(ptrs)) == 0;
    }
  } last_key;
  cudaGraphExec_t exec = nullptr;
  struct Tuned {
    TuneCfg cfg;
    int tried = 0;
    float best_ms = 0, worst_ms = 0;
  };
  std::map<std::vector<int64_t>, Tuned> tuned;
  int32_t info[4] = {0, 0, 0, 0};
  Tuned last_tuning;
  bool last_tuned_now = false;
};

BatchCache& cache() {
  static BatchCache* c = new BatchCache();  // lives until exit
  return *c;
}

template <typename K>
int grid_of(K kernel, const TuneCfg& t, int64_t work_warps) {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, t.threads, 0) != cudaSuccess || occ < 1) occ = 1;
  int bps = t.bps > 0 ? std::min(t.bps, occ) : occ;
  int warps = t.threads / 32;
  return (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sm_count() * bps, (work_warps + warps - 1) / warps));
}

template <int STACK>
void launch_batch(const TuneCfg& t, const BatchCam* cams, int ncams, int ntasks, int64_t maxjobs, uint32_t* ctrl,
                  int4* gbuf, float4* jobs, int64_t cap, cudaStream_t st) {
  cudaMemsetAsync(ctrl, 0, 32, st);
  const BatchShape sh = t.shape();
  k_bprimary<STACK><<<grid_of(k_bprimary<STACK>, t, ntasks), t.threads, 0, st>>>(cams, ncams, ntasks, ctrl, gbuf,
                                                                                   jobs, cap, sh);
  if (maxjobs > 0)
    k_bshadow<STACK><<<grid_of(k_bshadow<STACK>, t, (maxjobs + 31) / 32), t.threads, 0, st>>>(cams, ncams, ctrl, gbuf,
                                                                                             jobs, cap);
  k_bresolve<<<grid_of(k_bresolve, t, ntasks), t.threads, 0, st>>>(cams, ncams, ntasks, ctrl, gbuf, sh);
}

void launch_cfg(const TuneCfg& t, const BatchCam* cams, int ncams, int ntasks, int64_t maxjobs, uint32_t* ctrl,
                int4* gbuf, float4* jobs, int64_t cap, cudaStream_t st) {
  if (t.stack <= 8) launch_batch<8>(t, cams, ncams, ntasks, maxjobs, ctrl, gbuf, jobs, cap, st);
  else if (t.stack <= 32) launch_batch<32>(t, cams, ncams, ntasks, maxjobs, ctrl, gbuf, jobs, cap, st);
  else if (t.stack <= 64) launch_batch<64>(t, cams, ncams, ntasks, maxjobs, ctrl, gbuf, jobs, cap, st);
  else launch_batch<128>(t, cams, ncams, ntasks, maxjobs, ctrl, gbuf, jobs, cap, st);
}

template <typename T>
int grow(T** p, size_t* cap, size_t need, const char* what) {
  if (*cap >= need) return FIRE_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  if (cudaError_t e = dev_alloc((void**)p, need * sizeof(T), nullptr)) return cuda_check(e, what);
  *cap = need;
  return FIRE_OK;
}

}  // namespace

int batch_last_info(int32_t* out4) {
  BatchCache& C = cache();
  std::lock_guard<std::mutex> lk(C.mu);
  memcpy(out4, C.info, sizeof(C.info));
  return FIRE_OK;
}

int batch_last_tuning(int32_t* out8, float* ms2) {
  BatchCache& C = cache();
  std::lock_guard<std::mutex> lk(C.mu);
  const BatchCache::Tuned& t = C.last_tuning;
  out8[0] = t.cfg.threads;
  out8[1] = t.cfg.bps;
  out8[2] = t.cfg.stack;
  out8[3] = 1 << kTileLw[t.cfg.tile][0];
  out8[4] = 1 << kTileLw[t.cfg.tile][1];
  out8[5] = t.cfg.grab;
  out8[6] = t.tried;
  out8[7] = C.last_tuned_now ? 1 : 0;
  ms2[0] = t.best_ms;
  ms2[1] = t.worst_ms;
  return FIRE_OK;
}

int render_batch(const fire_scene* scenes, int nscenes, const fire_camera* cams, const int32_t* cam_scene,
                 int ncams, const fire_light* lights, const int32_t* light_off, float* const* outs,
                 const fire_render_opts* opts, cudaStream_t st) {
  BatchCache& C = cache();
  std::lock_guard<std::mutex> lk(C.mu);
  std::vector<BatchCam> h(ncams);
  std::vector<int64_t> shape;
  int ntasks = 0, maxh = 0, maxl = 0;
  int64_t cap = 64, nsamples = 0;
  for (int i = 0; i < ncams; ++i) {
    fire_scene_s* s = scenes[cam_scene[i]];
    BatchCam& b = h[i];
    memset(&b, 0, sizeof(b));
    b.nodes4 = s->nodes4;
    b.n4 = s->n4;
    b.tris = s->tris;
    b.nt = s->nt;
    b.mats = s->mats;
    b.sm = SmoothCtx{s->vnrm, s->xf_buf[s->cur], s->sidx, s->vbody};
    b.out = outs[i];
    b.cam = make_cam(cams[i]);
    int sc = cam_scene[i];
    int e = make_lights(lights + light_off[sc], light_off[sc + 1] - light_off[sc], &b.lights);
    if (e) return e;
    b.err = s->ctrl + 8;
    b.sample_base = nsamples;
    nsamples += (int64_t)b.cam.W * b.cam.H * b.cam.spp;
    maxh = std::max(maxh, stack_need(s));
    maxl = std::max(maxl, b.lights.n);
    cap = std::max(cap, 2 * s->nt + 64);
    shape.push_back(s->nt);
    shape.push_back(b.cam.W);
    shape.push_back(b.cam.H);
    shape.push_back(b.cam.spp);
    shape.push_back(b.lights.n);
  }
  // tasks of every camera for a tile shape (task_begin prefix sums)
  auto layout = [&](int tile) {
    int n = 0;
    for (int i = 0; i < ncams; ++i) {
      const TaskGrid g = make_grid_w(h[i].cam.W, 0, h[i].cam.H, h[i].cam.spp, kTileLw[tile][h[i].cam.spp == 4 ? 1 : 0]);
      h[i].task_begin = n;
      n += g.tiles_x * g.tiles_y;
    }
    return n;
  };
  ntasks = layout(0);
  if (ncams == 0 || ntasks == 0) return FIRE_OK;
  if (nsamples >= ((int64_t)1 << 28)) return set_error(FIRE_ERR_INVALID_ARG, "batch has 2^28 samples or more");
  const int64_t maxjobs = nsamples * maxl;
  const BatchCam* old_cams = C.d_cams;
  if (int e = grow(&C.d_cams, &C.cap_cams, (size_t)ncams, "batch descriptors")) return e;
  if (C.d_cams != old_cams) C.last_bytes.clear();
  if (int e = grow(&C.d_gbuf, &C.cap_samples, (size_t)nsamples, "batch records")) return e;
  if (int e = grow(&C.d_jobs, &C.cap_jobs, (size_t)std::max<int64_t>(2 * maxjobs, 2), "batch shadow queue")) return e;
  if (!C.d_ctrl) {
    if (cudaError_t e = dev_alloc((void**)&C.d_ctrl, 64, nullptr)) return cuda_check(e, "batch ctrl");
    cudaMemsetAsync(C.d_ctrl, 0, 64, st);
  }
  const size_t nbytes = sizeof(BatchCam) * ncams;
  auto upload = [&]() -> int {
    bool same = C.last_bytes.size() == nbytes && memcmp(C.last_bytes.data(), h.data(), nbytes) == 0;
    if (same) return FIRE_OK;
    if (int e = cuda_check(cudaMemcpyAsync(C.d_cams, h.data(), nbytes, cudaMemcpyHostToDevice, st), "upload"))
      return e;
    // the pageable copy is staged before cudaMemcpyAsync returns
    C.last_bytes.assign((unsigned char*)h.data(), (unsigned char*)h.data() + nbytes);
    return FIRE_OK;
  };
  // the scenes' current frame buffers: wait for their build/refit (the
  // tuning launches below read them too)
  for (int i = 0; i < nscenes; ++i) frame_acquire(scenes[i], st);
  // configuration: caller's, else tuned once per batch shape
  fire_render_opts o{};
  if (opts) o = *opts;
  if (o.stack_depth > 0 && o.stack_depth < maxh)
    return set_error(FIRE_ERR_INVALID_ARG, "stack_depth below a scene's tree requirement");
  int need = stack_for_height(maxh, o.stack_depth);
  TuneCfg cfg;
  cfg.stack = need;
  bool tuned_now = false;
  BatchCache::Tuned record;
  if (o.block_threads > 0 || o.blocks_per_sm > 0) {
    cfg.threads = o.block_threads > 0 ? o.block_threads : 128;
    cfg.bps = o.blocks_per_sm;
    const int tile_sel = (o.flags >> 8) & 3;  // FIRE_BATCH_TILE(n): shape n - 1
    cfg.tile = tile_sel > 0 ? tile_sel - 1 : 0;
    cfg.grab = (o.flags & FIRE_BATCH_GRAB2) ? 2 : 1;
    record.cfg = cfg;
  } else {
    auto it = C.tuned.find(shape);
    if (it != C.tuned.end()) {
      record = it->second;
      cfg = record.cfg;
    } else {
      // coordinate search, each candidate timed once after a warm launch:
      // threads x persistent blocks per SM, then the task tile shape, then
      // the tasks a warp grabs at once, then a deeper stack than the trees
      // need (every candidate gives the same images)
      cudaEvent_t e0, e1;
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
      float best = 1e30f, worst = 0.0f;
      int tried = 0;
      TuneCfg bestc = cfg;
      auto time_cfg = [&](const TuneCfg& t) -> int {
        const int n = layout(t.tile);
        if (int e = upload()) return e;
        launch_cfg(t, C.d_cams, ncams, n, maxjobs, C.d_ctrl, C.d_gbuf, C.d_jobs, cap, st);  // warm
        cudaEventRecord(e0, st);
        launch_cfg(t, C.d_cams, ncams, n, maxjobs, C.d_ctrl, C.d_gbuf, C.d_jobs, cap, st);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        ++tried;
        worst = std::max(worst, ms);
        if (ms < best) {
          best = ms;
          bestc = t;
        }
        return FIRE_OK;
      };
      for (int thr : {64, 128})
        for (int bps : {2, 4, 8, 0}) {
          TuneCfg t = cfg;
          t.threads = thr;
          t.bps = bps;
          if (int e = time_cfg(t)) return e;
        }
      const TuneCfg base1 = bestc;
      for (int tile : {1, 2}) {
        TuneCfg t = base1;
        t.tile = tile;
        if (int e = time_cfg(t)) return e;
      }
      const TuneCfg base2 = bestc;
      {
        TuneCfg t = base2;
        t.grab = 2;
        if (int e = time_cfg(t)) return e;
      }
      if (need < 128) {
        TuneCfg t = bestc;
        t.stack = need * 2 > 128 ? 128 : need * 2;
        if (int e = time_cfg(t)) return e;
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      if (int e = cuda_check(cudaGetLastError(), "autotune")) return e;
      cfg = bestc;
      record.cfg = cfg;
      record.tried = tried;
      record.best_ms = best;
      record.worst_ms = worst;
      C.tuned[shape] = record;
      tuned_now = true;
    }
  }
  ntasks = layout(cfg.tile);
  if (int e = upload()) return e;
  C.last_tuning = record;
  C.last_tuned_now = tuned_now;
  C.info[0] = cfg.threads;
  C.info[1] = cfg.bps;
  C.info[2] = cfg.stack;
  C.info[3] = tuned_now ? 1 : 0;
  // graph: (re)capture when the launch shape or a scratch buffer changed
  BatchCache::Key key;
  key.cfg = cfg;
  key.ncams = ncams;
  key.ntasks = ntasks;
  key.maxjobs = maxjobs;
  key.cap = cap;
  key.ptrs[0] = C.d_cams;
  key.ptrs[1] = C.d_ctrl;
  key.ptrs[2] = C.d_gbuf;
  key.ptrs[3] = C.d_jobs;
  if (!(C.exec && C.last_key == key)) {
    sm_count();  // cached before capture
    if (C.exec) {
      cudaGraphExecDestroy(C.exec);
      C.exec = nullptr;
    }
    cudaStream_t cs;
    if (int e = cuda_check(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "stream")) return e;
    cudaGraph_t graph;
    cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    launch_cfg(cfg, C.d_cams, ncams, ntasks, maxjobs, C.d_ctrl, C.d_gbuf, C.d_jobs, cap, cs);
    cudaError_t ce = cudaStreamEndCapture(cs, &graph);
    cudaStreamDestroy(cs);
    if (int e = cuda_check(ce, "graph capture")) return e;
    ce = cudaGraphInstantiate(&C.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (int e = cuda_check(ce, "graph instantiate")) return e;
    C.last_key = key;
  }
  const int e = cuda_check(cudaGraphLaunch(C.exec, st), "graph launch");
  for (int i = 0; i < nscenes; ++i) frame_release(scenes[i], st);
  return e;
}

void batch_free(fire_scene_s*) {}

}  // namespace fire
