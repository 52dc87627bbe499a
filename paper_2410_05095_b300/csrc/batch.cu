// Batched rendering: many cameras over many scenes (uneven triangle counts
// and resolutions) in ONE persistent launch.  Each warp pulls a 32-sample
// task from a single atomic counter that spans every camera's tiles, finds
// its camera by binary search over the task prefix sums, and runs the whole
// per-sample path (nearest hit, shadow rays, shading, resolve) in registers.
// The launch (counter reset + kernel) is captured once as a CUDA graph and
// replayed while the batch is unchanged.  Threads per block, blocks per SM
// and stack depth are chosen by timing candidates on the first call of each
// batch shape (autotuner), unless the caller fixes them.
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
  float* out;
  CamParams cam;
  LightParams lights;
  uint32_t* err;  // the scene's sticky error word
  int task_begin;
  int pad;
};

template <int STACK>
__global__ void __launch_bounds__(256) k_batch(const BatchCam* __restrict__ cams, int ncams, int ntasks,
                                               uint32_t* ctrl, int64_t cap) {
  const int lane = threadIdx.x & 31;
  while (true) {
    int task = 0;
    if (lane == 0) task = atomicAdd(ctrl, 1);
    task = __shfl_sync(kFull, task, 0);
    if (task >= ntasks) return;
    int lo = 0, hi = ncams - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (cams[mid].task_begin <= task) lo = mid; else hi = mid - 1;
    }
    const BatchCam& bc = cams[lo];
    TaskGrid g = make_grid(bc.cam.W, 0, bc.cam.H, bc.cam.spp);
    int x, y, k;
    bool valid = task_sample(g, task - bc.task_begin, lane, x, y, k);
    TraceCtx c{bc.nodes4, bc.n4, scene_span(bc.nodes4, bc.nt), bc.tris, bc.nt, cap, bc.err};
    float3 rad = f3(0.0f, 0.0f, 0.0f);
    int hit = 0;
    if (valid) {
      float3 o = f3(bc.cam.ox, bc.cam.oy, bc.cam.oz);
      float3 d = cam_dir(bc.cam, x, y, k);
      int prim, pos;
      float t;
      trace_nearest<STACK>(c, o, d, prim, pos, t);
      if (prim >= 0) {
        hit = 1;
        const float eps = scene_eps(bc.nodes4, bc.nt);
        float4 B = __ldg(bc.tris + 3 * (int64_t)pos + 1), C = __ldg(bc.tris + 3 * (int64_t)pos + 2);
        float3 n, po;
        hit_frame(B, C, o, d, t, eps, n, po);
        float3 v = neg3(d);
        const float* mp = bc.mats + 5 * (int64_t)__float_as_uint(B.w);
        float ar = __ldg(mp), ag = __ldg(mp + 1), ab = __ldg(mp + 2), rough = __ldg(mp + 3), metal = __ldg(mp + 4);
        for (int j = 0; j < bc.lights.n; ++j) {
          float3 l;
          float E, tmax;
          light_vec(bc.lights, j, bc.lights.I[j], po, l, E, tmax);
          float ndl = dot3(n, l);
          if (!(ndl > 0.0f)) continue;
          if (trace_any<STACK>(c, po, l, tmax, prim)) continue;
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

struct TuneCfg {
  int threads = 128, bps = 0, stack = 64;
};

struct BatchCache {
  std::mutex mu;
  BatchCam* d_cams = nullptr;
  size_t cap_cams = 0;
  uint32_t* d_ctrl = nullptr;
  std::vector<unsigned char> last_bytes;
  TuneCfg last_cfg;
  int last_ncams = 0, last_ntasks = 0;
  cudaGraphExec_t exec = nullptr;
  std::map<std::vector<int64_t>, TuneCfg> tuned;
  int32_t info[4] = {0, 0, 0, 0};
};

BatchCache& cache() {
  static BatchCache* c = new BatchCache();  // lives until exit
  return *c;
}

template <int STACK>
void launch_batch(const TuneCfg& t, const BatchCam* cams, int ncams, int ntasks, uint32_t* ctrl,
                  int64_t cap, cudaStream_t st) {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch<STACK>, t.threads, 0) != cudaSuccess || occ < 1)
    occ = 1;
  int bps = t.bps > 0 ? std::min(t.bps, occ) : occ;
  int warps = t.threads / 32;
  int grid = std::max(1, std::min(sm_count() * bps, (ntasks + warps - 1) / warps));
  k_batch<STACK><<<grid, t.threads, 0, st>>>(cams, ncams, ntasks, ctrl, cap);
}

void launch_cfg(const TuneCfg& t, const BatchCam* cams, int ncams, int ntasks, uint32_t* ctrl, int64_t cap,
                cudaStream_t st) {
  cudaMemsetAsync(ctrl, 0, 4, st);
  if (t.stack <= 8) launch_batch<8>(t, cams, ncams, ntasks, ctrl, cap, st);
  else if (t.stack <= 32) launch_batch<32>(t, cams, ncams, ntasks, ctrl, cap, st);
  else if (t.stack <= 64) launch_batch<64>(t, cams, ncams, ntasks, ctrl, cap, st);
  else launch_batch<128>(t, cams, ncams, ntasks, ctrl, cap, st);
}

}  // namespace

int batch_last_info(int32_t* out4) {
  BatchCache& C = cache();
  std::lock_guard<std::mutex> lk(C.mu);
  memcpy(out4, C.info, sizeof(C.info));
  return FIRE_OK;
}

int render_batch(const fire_scene* scenes, int nscenes, const fire_camera* cams, const int32_t* cam_scene,
                 int ncams, const fire_light* lights, const int32_t* light_off, float* const* outs,
                 const fire_render_opts* opts, cudaStream_t st) {
  BatchCache& C = cache();
  std::lock_guard<std::mutex> lk(C.mu);
  std::vector<BatchCam> h(ncams);
  std::vector<int64_t> shape;
  int ntasks = 0, maxh = 0;
  int64_t cap = 64;  // safety bound: a ray visits each node at most once
  for (int i = 0; i < ncams; ++i) {
    fire_scene_s* s = scenes[cam_scene[i]];
    BatchCam& b = h[i];
    memset(&b, 0, sizeof(b));
    b.nodes4 = s->nodes4;
    b.n4 = s->n4;
    b.tris = s->tris;
    b.nt = s->nt;
    b.mats = s->mats;
    b.out = outs[i];
    b.cam = make_cam(cams[i]);
    int sc = cam_scene[i];
    int e = make_lights(lights + light_off[sc], light_off[sc + 1] - light_off[sc], &b.lights);
    if (e) return e;
    b.err = s->ctrl + 8;
    b.task_begin = ntasks;
    TaskGrid g = make_grid(b.cam.W, 0, b.cam.H, b.cam.spp);
    ntasks += g.tiles_x * g.tiles_y;
    maxh = std::max(maxh, stack_need(s));
    cap = std::max(cap, 2 * s->nt + 64);
    shape.push_back(s->nt);
    shape.push_back(b.cam.W);
    shape.push_back(b.cam.H);
    shape.push_back(b.cam.spp);
    shape.push_back(b.lights.n);
  }
  if (ncams == 0 || ntasks == 0) return FIRE_OK;
  // cameras whose image has no tasks still work: binary search skips them
  if ((size_t)ncams > C.cap_cams) {
    if (C.d_cams) cudaFree(C.d_cams);
    C.d_cams = nullptr;
    C.cap_cams = 0;
    if (cudaError_t e = dev_alloc((void**)&C.d_cams, sizeof(BatchCam) * ncams, nullptr)) {
      return cuda_check(e, "batch descriptors");
    }
    C.cap_cams = ncams;
    C.last_bytes.clear();
  }
  if (!C.d_ctrl) {
    if (cudaError_t e = dev_alloc((void**)&C.d_ctrl, 64, nullptr)) return cuda_check(e, "batch ctrl");
    cudaMemsetAsync(C.d_ctrl, 0, 64, st);
  }
  const size_t nbytes = sizeof(BatchCam) * ncams;
  bool same = C.last_bytes.size() == nbytes && memcmp(C.last_bytes.data(), h.data(), nbytes) == 0;
  if (!same) {
    if (int e = cuda_check(cudaMemcpyAsync(C.d_cams, h.data(), nbytes, cudaMemcpyHostToDevice, st), "upload"))
      return e;
    // the pageable copy is staged before cudaMemcpyAsync returns
    C.last_bytes.assign((unsigned char*)h.data(), (unsigned char*)h.data() + nbytes);
  }
  // configuration: caller's, else tuned once per batch shape
  fire_render_opts o{};
  if (opts) o = *opts;
  if (o.stack_depth > 0 && o.stack_depth < maxh)
    return set_error(FIRE_ERR_INVALID_ARG, "stack_depth below a scene's tree height");
  int need = stack_for_height(maxh, o.stack_depth);
  TuneCfg cfg;
  cfg.stack = need;
  bool tuned_now = false;
  if (o.block_threads > 0 || o.blocks_per_sm > 0) {
    cfg.threads = o.block_threads > 0 ? o.block_threads : 128;
    cfg.bps = o.blocks_per_sm;
  } else {
    auto it = C.tuned.find(shape);
    if (it != C.tuned.end()) {
      cfg = it->second;
    } else {
      cudaEvent_t e0, e1;
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
      float best = 1e30f;
      TuneCfg bestc = cfg;
      const int thr_list[3] = {64, 128, 256};
      const int bps_list[5] = {1, 2, 4, 8, 0};
      const int stk_list[1] = {need};  // deeper stacks are never faster
      for (int stk : stk_list)
        for (int thr : thr_list)
          for (int bps : bps_list) {
            TuneCfg t{thr, bps, stk};
            launch_cfg(t, C.d_cams, ncams, ntasks, C.d_ctrl, cap, st);  // warm
            cudaEventRecord(e0, st);
            launch_cfg(t, C.d_cams, ncams, ntasks, C.d_ctrl, cap, st);
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) { best = ms; bestc = t; }
          }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      if (int e = cuda_check(cudaGetLastError(), "autotune")) return e;
      cfg = bestc;
      C.tuned[shape] = cfg;
      tuned_now = true;
    }
  }
  C.info[0] = cfg.threads;
  C.info[1] = cfg.bps;
  C.info[2] = cfg.stack;
  C.info[3] = tuned_now ? 1 : 0;
  // graph: (re)capture when the launch shape changed
  bool relaunch = C.exec && C.last_cfg.threads == cfg.threads && C.last_cfg.bps == cfg.bps &&
                  C.last_cfg.stack == cfg.stack && C.last_ncams == ncams && C.last_ntasks == ntasks;
  if (!relaunch) {
    sm_count();  // cached before capture
    if (C.exec) {
      cudaGraphExecDestroy(C.exec);
      C.exec = nullptr;
    }
    cudaStream_t cs;
    if (int e = cuda_check(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "stream")) return e;
    cudaGraph_t graph;
    cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    launch_cfg(cfg, C.d_cams, ncams, ntasks, C.d_ctrl, cap, cs);
    cudaError_t ce = cudaStreamEndCapture(cs, &graph);
    cudaStreamDestroy(cs);
    if (int e = cuda_check(ce, "graph capture")) return e;
    ce = cudaGraphInstantiate(&C.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (int e = cuda_check(ce, "graph instantiate")) return e;
    C.last_cfg = cfg;
    C.last_ncams = ncams;
    C.last_ntasks = ntasks;
  }
  return cuda_check(cudaGraphLaunch(C.exec, st), "graph launch");
}

void batch_free(fire_scene_s*) {}

}  // namespace fire
