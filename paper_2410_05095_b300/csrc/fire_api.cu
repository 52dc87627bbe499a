// C ABI of libfire: handles, validation, device memory, error codes.
// Every entry point checks its arguments on the host, enqueues work on the
// caller's stream and returns without synchronising unless fire.h says so.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <vector>

#include "trace_device.cuh"

namespace fire {

namespace {
thread_local std::string g_err;
thread_local int g_fail_alloc = 0;
}  // namespace

int set_error(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

int cuda_check(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return FIRE_OK;
  cudaGetLastError();  // clear a non-sticky error
  if (e == cudaErrorMemoryAllocation) return set_error(FIRE_ERR_OOM, std::string(what) + ": out of device memory");
  return set_error(FIRE_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

cudaError_t dev_alloc(void** p, size_t bytes, size_t* counter) {
  *p = nullptr;
  if (g_fail_alloc > 0 && --g_fail_alloc == 0) return cudaErrorMemoryAllocation;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaSuccess && counter) *counter += bytes;
  return e;
}

int sm_count() {
  static int n = 0;
  static std::once_flag once;
  std::call_once(once, [] {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 1;
  });
  return n;
}

namespace {
// Host FP32 vector helpers in the same operation order as the device ones
// (the host compiler runs with -ffp-contract=off).
struct H3 { float x, y, z; };
H3 hsub(H3 a, H3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
float hdot(H3 a, H3 b) { return std::fmaf(a.x, b.x, std::fmaf(a.y, b.y, a.z * b.z)); }
H3 hcross(H3 a, H3 b) {
  return {std::fmaf(a.y, b.z, -(a.z * b.y)), std::fmaf(a.z, b.x, -(a.x * b.z)), std::fmaf(a.x, b.y, -(a.y * b.x))};
}
H3 hnorm(H3 v) {
  float len = std::sqrt(hdot(v, v));
  return {v.x / len, v.y / len, v.z / len};
}
bool finite3(const float* v) { return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]); }
}  // namespace

// forward = normalize(target - pos), right = normalize(forward x up),
// up' = right x forward, sys = float(tan(vfov/2)) (double tan), sxs = sys * (W/H).
CamParams make_cam(const fire_camera& c) {
  CamParams p;
  H3 pos{c.pos[0], c.pos[1], c.pos[2]}, tgt{c.target[0], c.target[1], c.target[2]}, up{c.up[0], c.up[1], c.up[2]};
  H3 f = hnorm(hsub(tgt, pos));
  H3 r = hnorm(hcross(f, up));
  H3 u = hcross(r, f);
  p.ox = pos.x; p.oy = pos.y; p.oz = pos.z;
  p.fx = f.x; p.fy = f.y; p.fz = f.z;
  p.rx = r.x; p.ry = r.y; p.rz = r.z;
  p.ux = u.x; p.uy = u.y; p.uz = u.z;
  p.sys = (float)std::tan((double)c.vfov_deg * 3.14159265358979323846 / 360.0);
  p.sxs = p.sys * ((float)c.width / (float)c.height);
  p.W = c.width;
  p.H = c.height;
  p.spp = c.spp;
  return p;
}

int make_lights(const fire_light* lights, int n, LightParams* out) {
  if (n < 0 || n > kMaxLights) return set_error(FIRE_ERR_INVALID_ARG, "nlights must be in [0, 8]");
  if (n > 0 && !lights) return set_error(FIRE_ERR_INVALID_ARG, "lights is NULL");
  memset(out, 0, sizeof(*out));
  out->n = n;
  for (int j = 0; j < n; ++j) {
    const fire_light& L = lights[j];
    if ((L.type != 0 && L.type != 1) || !finite3(L.v) || !std::isfinite(L.intensity) || L.intensity < 0)
      return set_error(FIRE_ERR_INVALID_ARG, "invalid light " + std::to_string(j));
    H3 v{L.v[0], L.v[1], L.v[2]};
    if (L.type == 1) {
      if (hdot(v, v) == 0.0f) return set_error(FIRE_ERR_INVALID_ARG, "directional light with zero direction");
      v = hnorm(v);
    }
    out->type[j] = L.type;
    out->x[j] = v.x;
    out->y[j] = v.y;
    out->z[j] = v.z;
    out->I[j] = L.intensity;
  }
  return FIRE_OK;
}

namespace {

int check_cam(const fire_camera* c) {
  if (!c) return set_error(FIRE_ERR_INVALID_ARG, "camera is NULL");
  if (c->spp != 1 && c->spp != 4) return set_error(FIRE_ERR_INVALID_ARG, "spp must be 1 or 4");
  // sample ids (and sample id x 8 + light in the shadow queue) stay below 2^31
  if (c->width <= 0 || c->height <= 0 || (int64_t)c->width * c->height * c->spp >= (int64_t)1 << 28)
    return set_error(FIRE_ERR_INVALID_ARG, "camera size out of range");
  if (!finite3(c->pos) || !finite3(c->target) || !finite3(c->up) || !(c->vfov_deg > 0 && c->vfov_deg < 180))
    return set_error(FIRE_ERR_INVALID_ARG, "camera parameters not finite / fov out of (0,180)");
  H3 f = hsub(H3{c->target[0], c->target[1], c->target[2]}, H3{c->pos[0], c->pos[1], c->pos[2]});
  H3 r = hcross(f, H3{c->up[0], c->up[1], c->up[2]});
  if (hdot(f, f) == 0.0f || hdot(r, r) == 0.0f) return set_error(FIRE_ERR_INVALID_ARG, "degenerate camera basis");
  return FIRE_OK;
}

int check_mats(const fire_material* m, int n) {
  if (n < 1 || !m) return set_error(FIRE_ERR_INVALID_ARG, "need at least one material");
  for (int i = 0; i < n; ++i) {
    bool ok = finite3(m[i].albedo) && std::isfinite(m[i].roughness) && std::isfinite(m[i].metallic) &&
              m[i].roughness > 0.0f && m[i].roughness <= 1.0f && m[i].metallic >= 0.0f && m[i].metallic <= 1.0f;
    for (int c = 0; c < 3; ++c) ok = ok && m[i].albedo[c] >= 0.0f && m[i].albedo[c] <= 1.0f;
    if (!ok) return set_error(FIRE_ERR_INVALID_ARG, "material " + std::to_string(i) + " out of range");
  }
  return FIRE_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// Stage profiler: an event pair per kernel launch, resolved lazily (the
// oldest pairs are synchronised only when many are pending or on read).
// ---------------------------------------------------------------------------
struct Profiler {
  struct Pending { int stage, launches; cudaEvent_t a, b; };
  std::vector<cudaEvent_t> pool;
  std::deque<Pending> pending;
  cudaEvent_t open[kStages] = {};
  double ms[kStages] = {};
  int64_t n[kStages] = {};
  cudaEvent_t get() {
    if (pool.empty()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      return e;
    }
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  void drain(size_t keep) {
    while (pending.size() > keep) {
      Pending p = pending.front();
      pending.pop_front();
      float t = 0.0f;
      cudaEventSynchronize(p.b);
      cudaEventElapsedTime(&t, p.a, p.b);
      ms[p.stage] += t;
      n[p.stage] += p.launches;
      pool.push_back(p.a);
      pool.push_back(p.b);
    }
  }
  ~Profiler() {
    drain(0);
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
    for (cudaEvent_t e : open)
      if (e) cudaEventDestroy(e);
  }
};

void prof_begin(fire_scene_s* s, int stage, cudaStream_t st) {
  if (!s->prof) return;
  Profiler* P = static_cast<Profiler*>(s->prof);
  if (P->open[stage]) P->pool.push_back(P->open[stage]);
  P->open[stage] = P->get();
  cudaEventRecord(P->open[stage], st);
}

void prof_end(fire_scene_s* s, int stage, cudaStream_t st, int launches) {
  if (!s->prof) return;
  Profiler* P = static_cast<Profiler*>(s->prof);
  if (!P->open[stage]) return;
  cudaEvent_t e = P->get();
  cudaEventRecord(e, st);
  P->pending.push_back({stage, launches, P->open[stage], e});
  P->open[stage] = nullptr;
  if (P->pending.size() > 1024) P->drain(512);
}

namespace {

void free_scene(fire_scene_s* s) {
  delete static_cast<Profiler*>(s->prof);
  s->prof = nullptr;
  void* ptrs0[] = {s->vnrm, s->xf_buf[0], s->xf_buf[1]};
  for (void* p : ptrs0)
    if (p) cudaFree(p);
  void* ptrs[] = {s->rest, s->idx, s->tmat, s->vbody, s->mats, s->xf, s->keys, s->keys_orig, s->order,
                  s->sidx, s->smat, s->nodes, s->leaf_slot, s->node_slot, s->counters, s->tris_buf[0],
                  s->tris_buf[1], s->nodes4_buf[0], s->nodes4_buf[1], s->cen,
                  s->keys_alt, s->vals_alt, s->hist, s->ctrl, s->gscratch, s->bwd_partials, s->jobs,
                  s->lvl_aux, s->q4, s->rank, s->rkeys, s->rdirs, s->pieces, s->graze,
                  s->blas_root, s->body_box, s->body_range, s->xf_ident, s->inst, s->inst_box, s->tlas_buf[0],
                  s->tlas_buf[1],
                  s->tinfo_buf[0], s->tinfo_buf[1], s->stage, s->qperm, s->qaux, s->tl_node, s->tl_refs,
                  s->tl_info, s->tl_top, s->tl_grp, s->nunion, s->tl_scratch};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (int b = 0; b < 2; ++b) {
    if (s->ready_ev[b]) cudaEventDestroy(s->ready_ev[b]);
    if (s->used_ev[b]) cudaEventDestroy(s->used_ev[b]);
  }
}

int upload_mats(fire_scene_s* s, const fire_material* m, cudaStream_t st) {
  std::vector<float> h(5 * (size_t)s->nmat);
  for (int i = 0; i < s->nmat; ++i) {
    h[5 * i] = m[i].albedo[0];
    h[5 * i + 1] = m[i].albedo[1];
    h[5 * i + 2] = m[i].albedo[2];
    h[5 * i + 3] = m[i].roughness;
    h[5 * i + 4] = m[i].metallic;
  }
  s->h_mats.assign(m, m + s->nmat);
  int e = cuda_check(cudaMemcpyAsync(s->mats, h.data(), h.size() * 4, cudaMemcpyHostToDevice, st), "materials");
  if (e) return e;
  return cuda_check(cudaStreamSynchronize(st), "materials");  // h is a stack buffer
}

int load_xforms(fire_scene_s* s, const float* xf, int on_device, cudaStream_t st) {
  if (!xf) return set_error(FIRE_ERR_INVALID_ARG, "body_xforms is NULL");
  size_t n = 12 * (size_t)s->nbody;
  if (on_device) {
    return cuda_check(cudaMemcpyAsync(s->xf, xf, n * 4, cudaMemcpyDeviceToDevice, st), "xforms");
  }
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(xf[i])) return set_error(FIRE_ERR_INVALID_ARG, "non-finite body transform");
  return cuda_check(cudaMemcpyAsync(s->xf, xf, n * 4, cudaMemcpyHostToDevice, st), "xforms");
}

int alloc_lbvh(fire_scene_s* s) {
  const int64_t T = s->nt;
  if (T == 0 || s->keys) return FIRE_OK;
  const int64_t ntiles = (T + kSortTile - 1) / kSortTile;
  struct A { void** p; size_t b; } list[] = {
      {(void**)&s->keys, 8 * (size_t)T},          {(void**)&s->keys_orig, 8 * (size_t)T},
      {(void**)&s->order, 4 * (size_t)T},         {(void**)&s->sidx, 16 * (size_t)T},
      {(void**)&s->smat, 4 * (size_t)T},          {(void**)&s->nodes, 64 * (size_t)std::max<int64_t>(T - 1, 1)},
      {(void**)&s->leaf_slot, 4 * (size_t)T},     {(void**)&s->node_slot, 4 * (size_t)std::max<int64_t>(T - 1, 1)},
      {(void**)&s->counters, 4 * (size_t)std::max<int64_t>(T - 1, 1)}, {(void**)&s->tris_buf[0], 48 * (size_t)T},
      {(void**)&s->tris_buf[1], 48 * (size_t)T},
      {(void**)&s->cen, 16 * (size_t)T},          {(void**)&s->keys_alt, 8 * (size_t)T},
      {(void**)&s->vals_alt, 4 * (size_t)T},      {(void**)&s->hist, 4 * (size_t)(kSortBins * (ntiles + 1))},
      {(void**)&s->rank, 4 * (size_t)T},
      {(void**)&s->stage, 24 * (size_t)T},
      {(void**)&s->tl_node, 8 * (size_t)T},       {(void**)&s->tl_refs, 16 * (size_t)T},
      {(void**)&s->tl_info, 16 * (size_t)T},
      {(void**)&s->tl_top, 4 * (size_t)T},        {(void**)&s->tl_grp, 8 * (size_t)(kMaxDepth4 + 1)},
      {(void**)&s->nunion, 24 * (size_t)T},
      {(void**)&s->tl_scratch, 4 * (12 * (size_t)T + (size_t)T / 1024 + 64 + kMaxDepth4)},
      {(void**)&s->lvl_aux, 12 * (size_t)kMaxDepth4 + 16},
      {(void**)&s->nodes4_buf[0], 128 * (size_t)std::max<int64_t>(T, 1)},
      {(void**)&s->nodes4_buf[1], 128 * (size_t)std::max<int64_t>(T, 1)},
      {(void**)&s->q4, 16 * (size_t)std::max<int64_t>(T - 1, 1)},
  };
  for (auto& a : list)
    if (cudaError_t e = dev_alloc(a.p, a.b, &s->bytes)) return cuda_check(e, "LBVH buffers");
  for (int b = 0; b < 2; ++b) {
    if (int e = cuda_check(cudaEventCreateWithFlags(&s->ready_ev[b], cudaEventDisableTiming), "event")) return e;
    if (int e = cuda_check(cudaEventCreateWithFlags(&s->used_ev[b], cudaEventDisableTiming), "event")) return e;
  }
  s->cur = 0;
  s->tris = s->tris_buf[0];
  s->nodes4 = s->nodes4_buf[0];
  return FIRE_OK;
}

// Two-level buffers (first two-level build): bottom-level roots, rest boxes,
// body ranges, identity matrices, the top level's entries and their rest
// boxes, and per frame buffer the top level and its record.
int alloc_two_level(fire_scene_s* s, cudaStream_t st) {
  if (s->blas_root) return FIRE_OK;
  const size_t nb = (size_t)s->nbody;
  struct A { void** p; size_t b; } list[] = {
      {(void**)&s->blas_root, 4 * nb},     {(void**)&s->body_box, 32 * nb},
      {(void**)&s->body_range, 8 * nb},    {(void**)&s->xf_ident, 48 * nb},
      {(void**)&s->inst, 8 * (size_t)kMaxTlasBodies}, {(void**)&s->inst_box, 32 * (size_t)kMaxTlasBodies},
      {(void**)&s->tlas_buf[0], 128 * ((size_t)kMaxTlasBodies + 2)},
      {(void**)&s->tlas_buf[1], 128 * ((size_t)kMaxTlasBodies + 2)},
      {(void**)&s->tinfo_buf[0], sizeof(TlasInfo)}, {(void**)&s->tinfo_buf[1], sizeof(TlasInfo)},
  };
  for (auto& a : list)
    if (cudaError_t e = dev_alloc(a.p, a.b, &s->bytes)) return cuda_check(e, "two-level buffers");
  // every pointer the traversal reads with 16-B loads is 16-B aligned (cudaMalloc gives 256)
  for (const void* p : {(const void*)s->tlas_buf[0], (const void*)s->tlas_buf[1], (const void*)s->tinfo_buf[0],
                        (const void*)s->tinfo_buf[1], (const void*)s->body_box, (const void*)s->inst_box})
    if (reinterpret_cast<uintptr_t>(p) & 15u) return set_error(FIRE_ERR_CUDA, "misaligned two-level buffer");
  std::vector<float> id(12 * nb, 0.0f);
  for (size_t b = 0; b < nb; ++b) id[12 * b] = id[12 * b + 5] = id[12 * b + 10] = 1.0f;
  if (int e = cuda_check(cudaMemcpyAsync(s->xf_ident, id.data(), 48 * nb, cudaMemcpyHostToDevice, st), "copy"))
    return e;
  for (int b = 0; b < 2; ++b)
    if (int e = cuda_check(cudaMemsetAsync(s->tinfo_buf[b], 0, sizeof(TlasInfo), st), "memset")) return e;
  return cuda_check(cudaStreamSynchronize(st), "sync");  // id is a host vector
}

cudaStream_t as_stream(void* st) { return reinterpret_cast<cudaStream_t>(st); }

// Point the scene's current frame data at buffer b (two-level: the bottom
// levels stay in buffer 0; the top level and its record follow b).
void select_buffer(fire_scene_s* s, int b) {
  s->cur = b;
  s->tris = s->two_level ? s->tris_buf[0] : s->tris_buf[b];
  s->nodes4 = s->two_level ? s->nodes4_buf[0] : s->nodes4_buf[b];
  s->tlas = s->tlas_buf[b];
  s->tinfo = s->tinfo_buf[b];
}

}  // namespace

void frame_acquire(fire_scene_s* s, cudaStream_t st) {
  if (s->ready_rec[s->cur]) cudaStreamWaitEvent(st, s->ready_ev[s->cur], 0);
}

void frame_release(fire_scene_s* s, cudaStream_t st) {
  if (!s->used_ev[s->cur]) return;
  cudaEventRecord(s->used_ev[s->cur], st);
  s->used_rec[s->cur] = true;
}

}  // namespace fire

using namespace fire;

extern "C" {

const char* fire_last_error(void) { return g_err.c_str(); }
const char* fire_version(void) { return "fire-b300 1.0 (sm_103a)"; }

int fire_debug_fail_alloc(int32_t nth) {
  g_fail_alloc = nth > 0 ? nth : 0;
  return FIRE_OK;
}

int fire_scene_create(const float* verts_xyzw, int64_t nv, const uint32_t* tri_idx, int64_t nt,
                      const uint32_t* tri_mat, const uint16_t* vert_body, const fire_material* mats, int32_t nmat,
                      int32_t nbody, void* stream, fire_scene* out) {
  g_err.clear();
  if (!out) return set_error(FIRE_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (nv < 0 || nt < 0 || nbody < 1 || nbody > 65536 || nt >= ((int64_t)1 << 31) - 1 || nv >= ((int64_t)1 << 32))
    return set_error(FIRE_ERR_INVALID_ARG, "sizes out of range");
  if ((nv > 0 && (!verts_xyzw || !vert_body)) || (nt > 0 && (!tri_idx || !tri_mat)))
    return set_error(FIRE_ERR_INVALID_ARG, "NULL geometry pointer");
  if (int e = check_mats(mats, nmat)) return e;
  cudaStream_t st = as_stream(stream);
  fire_scene_s* s = new fire_scene_s();
  cudaGetDevice(&s->device);
  s->nv = nv;
  s->nt = nt;
  s->nmat = nmat;
  s->nbody = nbody;
  s->last_stream = st;
  struct A { void** p; size_t b; } list[] = {
      {(void**)&s->rest, 16 * (size_t)nv}, {(void**)&s->idx, 12 * (size_t)nt}, {(void**)&s->tmat, 4 * (size_t)nt},
      {(void**)&s->vbody, 2 * (size_t)nv}, {(void**)&s->mats, 20 * (size_t)nmat},
      {(void**)&s->xf, 48 * (size_t)nbody}, {(void**)&s->xf_buf[0], 48 * (size_t)nbody},
      {(void**)&s->xf_buf[1], 48 * (size_t)nbody}, {(void**)&s->ctrl, 128}};
  for (auto& a : list) {
    if (cudaError_t e = dev_alloc(a.p, a.b, &s->bytes)) {
      int rc = cuda_check(e, "scene buffers");
      free_scene(s);
      delete s;
      return rc;
    }
  }
  int rc = FIRE_OK;
  if (nv > 0) rc = rc ? rc : cuda_check(cudaMemcpyAsync(s->rest, verts_xyzw, 16 * nv, cudaMemcpyDefault, st), "copy");
  if (nv > 0) rc = rc ? rc : cuda_check(cudaMemcpyAsync(s->vbody, vert_body, 2 * nv, cudaMemcpyDefault, st), "copy");
  if (nt > 0) rc = rc ? rc : cuda_check(cudaMemcpyAsync(s->idx, tri_idx, 12 * nt, cudaMemcpyDefault, st), "copy");
  if (nt > 0) rc = rc ? rc : cuda_check(cudaMemcpyAsync(s->tmat, tri_mat, 4 * nt, cudaMemcpyDefault, st), "copy");
  rc = rc ? rc : cuda_check(cudaMemsetAsync(s->ctrl, 0, 128, st), "memset");
  rc = rc ? rc : upload_mats(s, mats, st);
  uint32_t bad = 0;
  rc = rc ? rc : lbvh_validate(s, st, &bad);
  if (!rc && bad) rc = set_error(FIRE_ERR_INVALID_ARG, "out-of-range index or non-finite vertex (" + std::to_string(bad) + ")");
  if (rc) {
    free_scene(s);
    delete s;
    return rc;
  }
  *out = s;
  return FIRE_OK;
}

int fire_scene_destroy(fire_scene s) {
  g_err.clear();
  if (!s) return set_error(FIRE_ERR_INVALID_ARG, "NULL scene");
  cudaDeviceSynchronize();
  free_scene(s);
  delete s;
  return FIRE_OK;
}

int fire_scene_set_materials(fire_scene s, const fire_material* mats, int32_t nmat) {
  return fire_scene_set_materials_ex(s, mats, nmat, 0);
}

int fire_scene_set_materials_ex(fire_scene s, const fire_material* mats, int32_t nmat, int32_t flags) {
  g_err.clear();
  if (!s) return set_error(FIRE_ERR_INVALID_ARG, "NULL scene");
  if (nmat != s->nmat) return set_error(FIRE_ERR_INVALID_ARG, "material count differs from the scene's");
  if (flags & ~FIRE_MATERIALS_SRGB_ALBEDO) return set_error(FIRE_ERR_INVALID_ARG, "unknown material flags");
  if (int e = check_mats(mats, nmat)) return e;
  if (int e = upload_mats(s, mats, s->last_stream)) return e;
  if (flags & FIRE_MATERIALS_SRGB_ALBEDO) return srgb_decode_materials(s->mats, s->nmat, s->last_stream);
  return FIRE_OK;
}

int fire_scene_set_normals(fire_scene s, const float* normals, int32_t on_device, void* stream) {
  g_err.clear();
  if (!s) return set_error(FIRE_ERR_INVALID_ARG, "NULL scene");
  cudaStream_t st = as_stream(stream);
  if (!normals) {
    if (s->vnrm) {
      // renders in flight may still read the normals
      if (int e = cuda_check(cudaDeviceSynchronize(), "sync")) return e;
      cudaFree(s->vnrm);
      s->bytes -= 16 * (size_t)s->nv;
      s->vnrm = nullptr;
    }
    return FIRE_OK;
  }
  if (!on_device)
    for (int64_t i = 0; i < 4 * s->nv; ++i)
      if (i % 4 != 3 && !std::isfinite(normals[i])) return set_error(FIRE_ERR_INVALID_ARG, "non-finite normal");
  if (!s->vnrm) {
    if (cudaError_t e = dev_alloc((void**)&s->vnrm, 16 * (size_t)s->nv, &s->bytes)) return cuda_check(e, "normals");
  } else {
    // renders in flight may still read the old normals
    if (int e = cuda_check(cudaDeviceSynchronize(), "sync")) return e;
  }
  s->last_stream = st;
  if (s->nv == 0) return FIRE_OK;
  if (int e = cuda_check(cudaMemcpyAsync(s->vnrm, normals, 16 * (size_t)s->nv, cudaMemcpyDefault, st), "normals"))
    return e;
  return on_device ? FIRE_OK : cuda_check(cudaStreamSynchronize(st), "normals");
}

int fire_scene_info(fire_scene s, int64_t* out8) {
  g_err.clear();
  if (!s || !out8) return set_error(FIRE_ERR_INVALID_ARG, "NULL argument");
  out8[0] = s->nv;
  out8[1] = s->nt;
  out8[2] = s->nmat;
  out8[3] = s->nbody;
  out8[4] = s->height;
  out8[5] = (int64_t)s->bytes;
  out8[6] = s->n4;
  out8[7] = s->height4;
  return FIRE_OK;
}

int fire_display(const float* hdr_rgba, int32_t width, int32_t height, float exposure, int32_t flags,
                 float* scratch_rgba, uint8_t* out_rgba8, void* stream) {
  g_err.clear();
  if (width < 0 || height < 0 || (int64_t)width * height >= ((int64_t)1 << 31))
    return set_error(FIRE_ERR_INVALID_ARG, "image size out of range");
  if (!std::isfinite(exposure) || !(exposure > 0.0f)) return set_error(FIRE_ERR_INVALID_ARG, "exposure must be > 0");
  if ((flags & ~FIRE_DISPLAY_FXAA) != 0) return set_error(FIRE_ERR_INVALID_ARG, "unknown display flags");
  if ((int64_t)width * height > 0 && (!hdr_rgba || !out_rgba8 || ((flags & FIRE_DISPLAY_FXAA) && !scratch_rgba)))
    return set_error(FIRE_ERR_INVALID_ARG, "NULL buffer");
  return display_image(hdr_rgba, width, height, exposure, (flags & FIRE_DISPLAY_FXAA) != 0, scratch_rgba, out_rgba8,
                       as_stream(stream));
}

int fire_render_info(fire_scene s, int64_t* out4) {
  g_err.clear();
  if (!s || !out4) return set_error(FIRE_ERR_INVALID_ARG, "NULL argument");
  memset(out4, 0, 4 * sizeof(int64_t));
  if (!s->rendered) return FIRE_OK;
  if (int e = cuda_check(cudaDeviceSynchronize(), "sync")) return e;
  uint32_t w[32];
  if (int e = cuda_check(cudaMemcpy(w, s->ctrl, sizeof(w), cudaMemcpyDeviceToHost), "copy")) return e;
  out4[0] = s->last_raster ? 1 : 0;
  out4[1] = s->last_raster ? w[kCtrlRasterFlag] : 0;
  out4[2] = s->last_raster ? w[kCtrlRasterPieces] : 0;
  for (int j = 0; j < 8; ++j) out4[3] += w[kCtrlShadowLen + j];  // per-light queue segments
  return FIRE_OK;
}

int fire_bvh_build(fire_scene s, const float* body_xforms, int32_t xforms_on_device, void* stream) {
  g_err.clear();
  if (!s) return set_error(FIRE_ERR_INVALID_ARG, "NULL scene");
  cudaStream_t st = as_stream(stream);
  s->last_stream = st;
  if (int e = load_xforms(s, body_xforms, xforms_on_device, st)) return e;
  if (int e = alloc_lbvh(s)) return e;
  // both buffers are rewritten: wait for their last users
  for (int b = 0; b < 2; ++b)
    if (s->used_rec[b]) cudaStreamWaitEvent(st, s->used_ev[b], 0);
  if (s->two_level)
    if (int e = alloc_two_level(s, st)) return e;
  select_buffer(s, 0);
  if (int e = lbvh_build(s, st)) return e;
  if (s->two_level && s->nt > 0) {
    // bottom levels done (rest pose, built once); the top level of this frame
    if (int e = tlas_build(s, st)) return e;
    for (int b = 0; b < 2; ++b) {
      cudaEventRecord(s->ready_ev[b], st);
      s->ready_rec[b] = true;
    }
    return FIRE_OK;
  }
  if (s->nt > 0) {
    // buffer 1 gets the 4-wide links (a refit rewrites boxes and records only)
    if (int e = cuda_check(cudaMemcpyAsync(s->nodes4_buf[1], s->nodes4_buf[0], 128 * (size_t)std::max<int64_t>(s->n4, 1),
                                           cudaMemcpyDeviceToDevice, st), "copy"))
      return e;
    for (int b = 0; b < 2; ++b) {
      cudaEventRecord(s->ready_ev[b], st);
      s->ready_rec[b] = true;
    }
  }
  return FIRE_OK;
}

int fire_bvh_refit(fire_scene s, const float* body_xforms, int32_t xforms_on_device, void* stream) {
  g_err.clear();
  if (!s) return set_error(FIRE_ERR_INVALID_ARG, "NULL scene");
  if (!s->built) return set_error(FIRE_ERR_NOT_BUILT, "refit before build");
  cudaStream_t st = as_stream(stream);
  s->last_stream = st;
  if (s->nt == 0) return load_xforms(s, body_xforms, xforms_on_device, st);
  // write the buffer the current frame does not use, after its last reader
  // and after the build that laid out its links
  const int target = s->cur ^ 1;
  if (s->used_rec[target]) cudaStreamWaitEvent(st, s->used_ev[target], 0);
  if (s->ready_rec[target]) cudaStreamWaitEvent(st, s->ready_ev[target], 0);
  if (int e = load_xforms(s, body_xforms, xforms_on_device, st)) return e;
  const int prev = s->cur;
  select_buffer(s, target);
  // two-level: only the top level is rebuilt (the bottom levels are at rest)
  if (int e = s->two_level ? tlas_build(s, st) : lbvh_refit(s, st)) {
    select_buffer(s, prev);
    return e;
  }
  cudaEventRecord(s->ready_ev[target], st);
  s->ready_rec[target] = true;
  return FIRE_OK;
}

static int fill_args(fire_scene s, const fire_camera* cam, const fire_light* lights, int32_t nlights,
                     RenderArgs* a) {
  if (!s) return set_error(FIRE_ERR_INVALID_ARG, "NULL scene");
  if (!s->built) return set_error(FIRE_ERR_NOT_BUILT, "render before build");
  if (int e = check_cam(cam)) return e;
  memset(a, 0, sizeof(*a));
  if (int e = make_lights(lights, nlights, &a->lights)) return e;
  a->nodes4 = s->nodes4;
  a->n4 = s->n4;
  a->tris = s->tris;
  a->nt = s->nt;
  a->cam = make_cam(*cam);
  a->mats.p = s->mats;
  a->mats.n = s->nmat;
  a->row_begin = 0;
  a->row_end = cam->height;
  a->iter_cap = s->iter_cap > 0 ? s->iter_cap : 2 * s->nt + 64;
  a->ctrl = s->ctrl;
  set_smooth_args(a, s);
  set_level_args(a, s);
  if (s->two_level && s->vnrm)
    return set_error(FIRE_ERR_INVALID_ARG, "smooth normals need the single-level structure");
  return FIRE_OK;
}

static int ensure_scratch(fire_scene s, size_t n) {
  if (s->gscratch_n >= n) return FIRE_OK;
  if (s->gscratch) {
    cudaFree(s->gscratch);
    s->bytes -= s->gscratch_n * sizeof(fire_gbuffer_rec);
  }
  s->gscratch = nullptr;
  s->gscratch_n = 0;
  if (cudaError_t e = dev_alloc((void**)&s->gscratch, n * sizeof(fire_gbuffer_rec), &s->bytes))
    return cuda_check(e, "G-buffer scratch");
  s->gscratch_n = n;
  return FIRE_OK;
}

int fire_render(fire_scene s, const fire_camera* cam, const fire_light* lights, int32_t nlights,
                const fire_render_opts* opts, float* out_rgba, fire_gbuffer_rec* gbuf, void* stream) {
  g_err.clear();
  RenderArgs a;
  if (int e = fill_args(s, cam, lights, nlights, &a)) return e;
  if (!out_rgba) return set_error(FIRE_ERR_INVALID_ARG, "out_rgba is NULL");
  fire_render_opts o{};
  if (opts) o = *opts;
  if (o.row_begin != 0 || o.row_end != 0) {
    if (o.row_begin < 0 || o.row_end > cam->height || o.row_begin >= o.row_end)
      return set_error(FIRE_ERR_INVALID_ARG, "row range out of the image");
    a.row_begin = o.row_begin;
    a.row_end = o.row_end;
  }
  if (o.stack_depth < 0 || o.stack_depth > 128 || o.blocks_per_sm < 0 ||
      (o.flags & ~(FIRE_RENDER_ALLOW_SHALLOW_STACK | FIRE_RENDER_TRACE_PRIMARY | FIRE_RENDER_RASTER_PRIMARY)) != 0 ||
      ((o.flags & FIRE_RENDER_TRACE_PRIMARY) && (o.flags & FIRE_RENDER_RASTER_PRIMARY)))
    return set_error(FIRE_ERR_INVALID_ARG, "invalid render options");
  if (s->two_level && (o.flags & FIRE_RENDER_RASTER_PRIMARY))
    return set_error(FIRE_ERR_INVALID_ARG, "the raster primary pass needs the single-level structure");
  if (o.stack_depth > 0 && o.stack_depth < std::min(stack_need(s), 128) &&
      !(o.flags & FIRE_RENDER_ALLOW_SHALLOW_STACK))
    return set_error(FIRE_ERR_INVALID_ARG, "stack_depth below the " + std::to_string(stack_need(s)) +
                                               " entries the tree can need");
  cudaStream_t st = as_stream(stream);
  s->last_stream = st;
  size_t nsamp = (size_t)cam->width * cam->height * cam->spp;
  if (gbuf) {
    a.g = gbuf;
  } else {
    if (int e = ensure_scratch(s, nsamp)) return e;
    a.g = s->gscratch;
  }
  // shadow-ray queue: per light one segment of 32 slots per task of the
  // full image (sparse, written by the primary pass), the dense order of its
  // rays (task order, as slots), counts and offsets per task
  const TaskGrid tg = make_grid(cam->width, 0, cam->height, cam->spp);
  const size_t ntask_full = (size_t)tg.tiles_x * tg.tiles_y;
  const size_t qseg = 32 * ntask_full;
  size_t njobs = qseg * (size_t)std::max(1, nlights);
  if (s->jobs_n < njobs) {
    if (s->jobs) {
      cudaFree(s->jobs);
      cudaFree(s->qperm);
      s->bytes -= s->jobs_n * 36;
    }
    s->jobs = nullptr;
    s->qperm = nullptr;
    s->jobs_n = 0;
    if (cudaError_t e = dev_alloc((void**)&s->jobs, njobs * 32, &s->bytes)) return cuda_check(e, "shadow queue");
    if (cudaError_t e = dev_alloc((void**)&s->qperm, njobs * 4, &s->bytes)) return cuda_check(e, "shadow queue order");
    s->jobs_n = njobs;
  }
  const size_t nq = (size_t)std::max(1, nlights) * (ntask_full + (ntask_full + 255) / 256 + 1);  // counts, block sums
  if (s->qaux_n < nq) {
    if (s->qaux) {
      cudaFree(s->qaux);
      s->bytes -= s->qaux_n * 4;
    }
    s->qaux = nullptr;
    s->qaux_n = 0;
    if (cudaError_t e = dev_alloc((void**)&s->qaux, nq * 4, &s->bytes)) return cuda_check(e, "shadow queue counts");
    s->qaux_n = nq;
  }
  a.qcnt = s->qaux;
  a.qseg = (int64_t)qseg;
  // raster primary pass scratch: one key and one direction per sample, a
  // piece queue, a deferred-triangle list
  if ((o.flags & FIRE_RENDER_RASTER_PRIMARY) && s->rkeys_n < nsamp) {
    if (s->rkeys) {
      cudaFree(s->rkeys);
      cudaFree(s->rdirs);
      s->bytes -= s->rkeys_n * 24;
    }
    s->rkeys = nullptr;
    s->rdirs = nullptr;
    s->rkeys_n = 0;
    if (cudaError_t e = dev_alloc((void**)&s->rkeys, nsamp * 8, &s->bytes)) return cuda_check(e, "raster keys");
    if (cudaError_t e = dev_alloc((void**)&s->rdirs, nsamp * 16, &s->bytes)) {
      cudaFree(s->rkeys);
      s->rkeys = nullptr;
      s->bytes -= nsamp * 8;
      return cuda_check(e, "raster directions");
    }
    s->rkeys_n = nsamp;
  }
  if ((o.flags & FIRE_RENDER_RASTER_PRIMARY) && !s->pieces) {
    size_t cap = (size_t)std::min<int64_t>(std::max<int64_t>(s->nt / 4, 262144), 1 << 22);
    if (cudaError_t e = dev_alloc((void**)&s->pieces, cap * 16, &s->bytes)) return cuda_check(e, "raster queue");
    s->pieces_n = cap;
  }
  if ((o.flags & FIRE_RENDER_RASTER_PRIMARY) && !s->graze) {
    size_t cap = (size_t)std::min<int64_t>(std::max<int64_t>(s->nt / 4, 65536), 1 << 22);
    if (cudaError_t e = dev_alloc((void**)&s->graze, cap * 4, &s->bytes)) return cuda_check(e, "raster list");
    s->graze_n = cap;
  }
  a.out = out_rgba;
  frame_acquire(s, st);
  const int e = render_frame(s, a, o, st);
  frame_release(s, st);
  return e;
}

int fire_render_batch(const fire_scene* scenes, int32_t nscenes, const fire_camera* cams, const int32_t* cam_scene,
                      int32_t ncams, const fire_light* lights, const int32_t* light_off, float* const* outs,
                      const fire_render_opts* opts, void* stream) {
  g_err.clear();
  if (nscenes < 1 || ncams < 0 || !scenes || (ncams > 0 && (!cams || !cam_scene || !outs)) || !light_off)
    return set_error(FIRE_ERR_INVALID_ARG, "invalid batch arguments");
  for (int i = 0; i < nscenes; ++i) {
    if (!scenes[i]) return set_error(FIRE_ERR_INVALID_ARG, "NULL scene in batch");
    if (!scenes[i]->built) return set_error(FIRE_ERR_NOT_BUILT, "batch scene not built");
    if (scenes[i]->two_level) return set_error(FIRE_ERR_INVALID_ARG, "the batch needs single-level scenes");
    if (light_off[i + 1] < light_off[i] || light_off[i + 1] - light_off[i] > kMaxLights)
      return set_error(FIRE_ERR_INVALID_ARG, "light_off not ascending or > 8 lights");
  }
  if (light_off[0] != 0 || (light_off[nscenes] > 0 && !lights))
    return set_error(FIRE_ERR_INVALID_ARG, "light_off[0] must be 0");
  for (int i = 0; i < ncams; ++i) {
    if (cam_scene[i] < 0 || cam_scene[i] >= nscenes) return set_error(FIRE_ERR_INVALID_ARG, "cam_scene out of range");
    if (int e = check_cam(&cams[i])) return e;
    if (!outs[i]) return set_error(FIRE_ERR_INVALID_ARG, "NULL output");
  }
  if (opts && (opts->row_begin || opts->row_end || (opts->flags & ~(FIRE_BATCH_TILE(3) | FIRE_BATCH_GRAB2)) ||
               opts->stack_depth < 0 || opts->stack_depth > 128 ||
               opts->blocks_per_sm < 0 || opts->block_threads < 0 || opts->block_threads > 128 ||
               (opts->block_threads % 32) != 0))
    return set_error(FIRE_ERR_INVALID_ARG, "invalid batch options");
  return render_batch(scenes, nscenes, cams, cam_scene, ncams, lights, light_off, outs, opts, as_stream(stream));
}

int fire_shade(fire_scene s, const fire_gbuffer_rec* gbuf, const fire_camera* cam, const fire_light* lights,
               int32_t nlights, const float* params, const float* inten, float* out_rgba, void* stream) {
  g_err.clear();
  RenderArgs a;
  if (int e = fill_args(s, cam, lights, nlights, &a)) return e;
  if (!gbuf || !params || (!inten && nlights > 0) || !out_rgba) return set_error(FIRE_ERR_INVALID_ARG, "NULL buffer");
  a.g = const_cast<fire_gbuffer_rec*>(gbuf);
  a.mats.p = params;
  a.out = out_rgba;
  cudaStream_t st = as_stream(stream);
  s->last_stream = st;
  frame_acquire(s, st);
  const int e = shade_from_gbuffer(s, a, inten, st);
  frame_release(s, st);
  return e;
}

int fire_shade_backward(fire_scene s, const fire_gbuffer_rec* gbuf, const fire_camera* cam, const fire_light* lights,
                        int32_t nlights, const float* params, const float* inten, const float* dL_drgba,
                        float* dparams, float* dinten, void* stream) {
  g_err.clear();
  RenderArgs a;
  if (int e = fill_args(s, cam, lights, nlights, &a)) return e;
  if (!gbuf || !params || (nlights > 0 && (!inten || !dinten)) || !dL_drgba || !dparams)
    return set_error(FIRE_ERR_INVALID_ARG, "NULL buffer");
  if (s->nmat * 5 + nlights > 12288) return set_error(FIRE_ERR_INVALID_ARG, "too many materials for the backward");
  a.g = const_cast<fire_gbuffer_rec*>(gbuf);
  a.mats.p = params;
  cudaStream_t st = as_stream(stream);
  s->last_stream = st;
  frame_acquire(s, st);
  const int e = shade_backward(s, a, inten, dL_drgba, dparams, dinten, st);
  frame_release(s, st);
  return e;
}

int fire_debug_dump(fire_scene s, int32_t what, void* host_dst, size_t bytes) {
  g_err.clear();
  if (!s || !host_dst) return set_error(FIRE_ERR_INVALID_ARG, "NULL argument");
  if (!s->built) return set_error(FIRE_ERR_NOT_BUILT, "dump before build");
  const int64_t T = s->nt;
  if (cudaError_t e = cudaDeviceSynchronize()) return cuda_check(e, "sync");
  auto need = [&](size_t n) { return bytes == n; };
  auto get = [&](void* dst, const void* src, size_t n) {
    return cuda_check(cudaMemcpy(dst, src, n, cudaMemcpyDeviceToHost), "dump copy");
  };
  switch (what) {
    case 0: if (!need(8 * T)) break; return T ? get(host_dst, s->keys_orig, 8 * T) : FIRE_OK;
    case 1: if (!need(4 * T)) break; return T ? get(host_dst, s->order, 4 * T) : FIRE_OK;
    case 2:
    case 3:
    case 4: {
      int64_t ni = T > 1 ? T - 1 : 0;
      size_t want = what == 2 ? 8 * ni : what == 3 ? 4 * (size_t)(T ? 2 * T - 1 : 0) : 24 * (size_t)(T ? 2 * T - 1 : 0);
      if (!need(want)) break;
      if (T == 0) return FIRE_OK;
      std::vector<Node> nodes(std::max<int64_t>(ni, 1));
      if (int e = get(nodes.data(), s->nodes, 64 * nodes.size())) return e;
      // node = 16 floats: child 0 box [0..5], link [6], height [7]; child 1 at [8..15]
      auto link = [&](const Node& n, int side) {
        int v;
        memcpy(&v, reinterpret_cast<const float*>(&n) + 8 * side + 6, 4);
        return v;
      };
      auto code = [&](int c) { return c >= 0 ? c : (int)(T - 1) + ~c; };
      if (what == 2) {
        int32_t* o = (int32_t*)host_dst;
        for (int64_t i = 0; i < ni; ++i) {
          o[2 * i] = code(link(nodes[i], 0));
          o[2 * i + 1] = code(link(nodes[i], 1));
        }
      } else if (what == 3) {
        int32_t* o = (int32_t*)host_dst;
        o[0] = -1;
        for (int64_t i = 0; i < ni; ++i) {
          o[code(link(nodes[i], 0))] = (int32_t)i;
          o[code(link(nodes[i], 1))] = (int32_t)i;
        }
      } else {
        // The per-frame boxes live in the 4-wide tree: each 4-wide member is
        // one binary node (its box is copied out); a binary node collapsed
        // inside a 4-wide node gets the union of its two children (exact
        // min/max), computed bottom-up over the binary topology.
        std::vector<Node4> n4(std::max<int64_t>(s->n4, 1));
        if (int e = get(n4.data(), s->nodes4, 128 * n4.size())) return e;
        const int64_t ncode = 2 * T - 1;
        std::vector<float> box(6 * ncode, 0.0f);
        std::vector<char> have(ncode, 0);
        for (int64_t q = 0; q < s->n4; ++q) {
          const int src[4] = {n4[q].src.x, n4[q].src.y, n4[q].src.z, n4[q].src.w};
          const float* m = reinterpret_cast<const float*>(&n4[q]);
          for (int k = 0; k < 4; ++k) {
            if (src[k] < 0 || (src[k] >> 1) >= (int64_t)nodes.size()) continue;
            int c = code(link(nodes[src[k] >> 1], src[k] & 1));
            if (c < 0 || c >= ncode) continue;
            for (int j = 0; j < 6; ++j) box[6 * (int64_t)c + j] = m[4 * j + k];
            have[c] = 1;
          }
        }
        // collapsed internal nodes (they can sit below a member, inside a
        // 4-wide node): post-order walk over every internal node (explicit
        // stack; leaves are always 4-wide members)
        std::vector<std::pair<int64_t, int>> stk;
        if (T > 1) stk.push_back({0, 0});
        while (!stk.empty()) {
          const int64_t c = stk.back().first;
          if (c < 0 || c >= ni) { stk.pop_back(); continue; }
          const int a = code(link(nodes[c], 0)), b = code(link(nodes[c], 1));
          if (a < 0 || a >= ncode || b < 0 || b >= ncode) return set_error(FIRE_ERR_CUDA, "corrupt topology");
          if (stk.back().second == 0) {
            stk.back().second = 1;
            if (a < ni) stk.push_back({a, 0});
            if (b < ni) stk.push_back({b, 0});
            continue;
          }
          if (!have[c]) {
            for (int j = 0; j < 3; ++j) {
              box[6 * c + j] = std::fmin(box[6 * (int64_t)a + j], box[6 * (int64_t)b + j]);
              box[6 * c + 3 + j] = std::fmax(box[6 * (int64_t)a + 3 + j], box[6 * (int64_t)b + 3 + j]);
            }
            have[c] = 1;
          }
          stk.pop_back();
        }
        memcpy(host_dst, box.data(), 24 * (size_t)ncode);
      }
      return FIRE_OK;
    }
    case 5: {
      if (!need(48 * (size_t)T)) break;
      return T ? get(host_dst, s->tris, 48 * T) : FIRE_OK;
    }
    case 6: {
      if (!need(24)) break;
      uint32_t u[6];
      if (int e = get(u, s->ctrl + 9, 24)) return e;
      float* o = (float*)host_dst;
      for (int k = 0; k < 6; ++k) o[k] = ord2f(u[k]);
      return FIRE_OK;
    }
    case 7:  // 4-wide nodes of the current buffer (two-level: the bottom levels)
      if (!need(128 * (size_t)s->n4)) break;
      return s->n4 ? get(host_dst, s->nodes4, 128 * (size_t)s->n4) : FIRE_OK;
    case 8:
    case 9:
    case 10:
    case 11: {
      if (!s->two_level) return set_error(FIRE_ERR_INVALID_ARG, "two-level dump of a single-level scene");
      const size_t nb = (size_t)s->nbody;
      if (what == 8) return need(4 * nb) ? get(host_dst, s->blas_root, 4 * nb) : set_error(FIRE_ERR_INVALID_ARG, "dump size mismatch");
      const size_t ntl = (size_t)kMaxTlasBodies + 2;
      if (what == 9) return need(128 * ntl) ? get(host_dst, s->tlas, 128 * ntl) : set_error(FIRE_ERR_INVALID_ARG, "dump size mismatch");
      if (what == 10) return need(sizeof(TlasInfo)) ? get(host_dst, s->tinfo, sizeof(TlasInfo)) : set_error(FIRE_ERR_INVALID_ARG, "dump size mismatch");
      return need(48 * nb) ? get(host_dst, s->xf_buf[s->cur], 48 * nb) : set_error(FIRE_ERR_INVALID_ARG, "dump size mismatch");
    }
    case 12: {  // the last fire_render's shadow rays, in the order the shadow pass takes them
      int64_t cnt[kMaxLights] = {0}, nr = 0;
      if (s->rendered && s->jobs && s->qperm && s->last_nlights > 0) {
        uint32_t w[32];
        if (int e = get(w, s->ctrl, sizeof(w))) return e;
        for (int j = 0; j < s->last_nlights; ++j) nr += cnt[j] = w[kCtrlShadowLen + j];
      }
      if (!need(32 * (size_t)nr)) break;
      const int64_t seg = s->last_qseg;
      std::vector<int32_t> perm;
      std::vector<float4> jobs;
      float4* o = reinterpret_cast<float4*>(host_dst);
      for (int j = 0; j < s->last_nlights; ++j) {
        if (cnt[j] == 0) continue;
        if (cnt[j] > seg) return set_error(FIRE_ERR_CUDA, "shadow queue longer than its segment");
        perm.resize((size_t)cnt[j]);
        jobs.resize(2 * (size_t)seg);
        if (int e = get(perm.data(), s->qperm + j * seg, 4 * (size_t)cnt[j])) return e;
        if (int e = get(jobs.data(), s->jobs + 2 * j * seg, 32 * (size_t)seg)) return e;
        for (int64_t k = 0; k < cnt[j]; ++k) {
          if (perm[k] < 0 || perm[k] >= seg) return set_error(FIRE_ERR_CUDA, "shadow queue order out of range");
          *o++ = jobs[2 * (size_t)perm[k]];
          *o++ = jobs[2 * (size_t)perm[k] + 1];
        }
      }
      return FIRE_OK;
    }
    case 13:  // the top level's entries
      if (!s->two_level) return set_error(FIRE_ERR_INVALID_ARG, "two-level dump of a single-level scene");
      if (!need(8 * (size_t)kMaxTlasBodies)) break;
      return get(host_dst, s->inst, 8 * (size_t)kMaxTlasBodies);
    default:
      return set_error(FIRE_ERR_INVALID_ARG, "unknown dump selector");
  }
  return set_error(FIRE_ERR_INVALID_ARG, "dump size mismatch");
}

int fire_scene_set_two_level(fire_scene s, int32_t enable) {
  g_err.clear();
  if (!s) return set_error(FIRE_ERR_INVALID_ARG, "NULL scene");
  if (enable != 0 && enable != 1) return set_error(FIRE_ERR_INVALID_ARG, "enable must be 0 or 1");
  if ((bool)enable == s->two_level) return FIRE_OK;
  if (enable) {
    if (s->nbody > kMaxTlasBodies)
      return set_error(FIRE_ERR_INVALID_ARG, "two-level mode supports at most " + std::to_string(kMaxTlasBodies) +
                                                 " bodies");
    uint32_t bad = 0;
    if (int e = lbvh_count_mixed(s, s->last_stream, &bad)) return e;
    if (bad)
      return set_error(FIRE_ERR_INVALID_ARG, std::to_string(bad) + " triangles have vertices in different bodies");
    if (s->vnrm) return set_error(FIRE_ERR_INVALID_ARG, "smooth normals need the single-level structure");
  }
  // renders in flight may read the old structure
  if (int e = cuda_check(cudaDeviceSynchronize(), "sync")) return e;
  s->two_level = enable != 0;
  s->built = false;
  for (int b = 0; b < 2; ++b) s->ready_rec[b] = s->used_rec[b] = false;
  return FIRE_OK;
}

int fire_sync_status(fire_scene s, void* stream) {
  g_err.clear();
  if (!s) return set_error(FIRE_ERR_INVALID_ARG, "NULL scene");
  cudaStream_t st = as_stream(stream);
  uint32_t w = 0;
  if (int e = cuda_check(cudaStreamSynchronize(st), "sync")) return e;
  if (int e = cuda_check(cudaMemcpy(&w, s->ctrl + 8, 4, cudaMemcpyDeviceToHost), "status")) return e;
  if (int e = cuda_check(cudaMemset(s->ctrl + 8, 0, 4), "status")) return e;
  if (w & kErrStack) return set_error(FIRE_ERR_STACK_OVERFLOW, "traversal stack overflow");
  if (w & kErrTimeout) return set_error(FIRE_ERR_TIMEOUT, "traversal iteration cap reached");
  if (w & kErrCorrupt) return set_error(FIRE_ERR_CUDA, "traversal met a link outside the tree");
  return FIRE_OK;
}

int fire_debug_set_iteration_cap(fire_scene s, int64_t cap) {
  g_err.clear();
  if (!s || cap < 0) return set_error(FIRE_ERR_INVALID_ARG, "invalid argument");
  s->iter_cap = cap;
  return FIRE_OK;
}

int fire_profile_enable(fire_scene s, int32_t enable) {
  g_err.clear();
  if (!s) return set_error(FIRE_ERR_INVALID_ARG, "NULL scene");
  if (enable && !s->prof) s->prof = new Profiler();
  if (!enable && s->prof) {
    delete static_cast<Profiler*>(s->prof);
    s->prof = nullptr;
  }
  return FIRE_OK;
}

int fire_profile_read(fire_scene s, double* ms8, int64_t* launches8) {
  g_err.clear();
  if (!s || !ms8 || !launches8) return set_error(FIRE_ERR_INVALID_ARG, "NULL argument");
  for (int i = 0; i < kStages; ++i) { ms8[i] = 0.0; launches8[i] = 0; }
  if (!s->prof) return FIRE_OK;
  Profiler* P = static_cast<Profiler*>(s->prof);
  P->drain(0);
  for (int i = 0; i < kStages; ++i) {
    ms8[i] = P->ms[i];
    launches8[i] = P->n[i];
    P->ms[i] = 0.0;
    P->n[i] = 0;
  }
  return FIRE_OK;
}

int fire_batch_last_config(int32_t* out4) {
  g_err.clear();
  if (!out4) return set_error(FIRE_ERR_INVALID_ARG, "NULL argument");
  return batch_last_info(out4);
}

int fire_batch_last_tuning(int32_t* out8, float* ms2) {
  g_err.clear();
  if (!out8 || !ms2) return set_error(FIRE_ERR_INVALID_ARG, "NULL argument");
  return batch_last_tuning(out8, ms2);
}

}  // extern "C"
