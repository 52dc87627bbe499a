// Internal declarations of libfire (B300 / sm_103a).
//
// Compiled with -fmad=false: no multiply-add is fused unless written as
// fmaf(), and '/' and sqrtf() are IEEE correctly rounded (nvcc defaults), so
// every FP32 expression below has one fixed rounding sequence.  The integer
// decisions of the method (Morton codes, nearest-hit argmin, shadow
// visibility) depend on that sequence.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstring>
#include <string>
#include <vector>

#include "../../include/fire.h"

namespace fire {

// ---------------------------------------------------------------------------
// Device data layout
// ---------------------------------------------------------------------------
// Internal node of the binary LBVH, 64 B = two 32-B sectors, one per child:
// the child's box, its link and its subtree height.  One node fetch decides
// which children a ray enters (no separate fetch of the child's own box),
// and a refit writes each child as one whole sector (no partial-sector
// read-modify-write in L2/DRAM).
//   a = lo0.x lo0.y lo0.z hi0.x      sector 0 (child 0)
//   b = hi0.y hi0.z link0 height0
//   c = lo1.x lo1.y lo1.z hi1.x      sector 1 (child 1)
//   d = hi1.y hi1.z link1 height1
// link >= 0: internal node index; link < 0: leaf at sorted position ~link
// (links and heights are stored as the bits of the float lanes).
struct __align__(16) Node {
  float4 a, b, c, d;
};
static_assert(sizeof(Node) == 64, "node must be 64 bytes");

// 4-wide node collapsed from the binary tree (build), 128 B = 4 sectors:
// child boxes as structure-of-arrays (one float4 per coordinate, lane c =
// child c), the four child links (>= 0: 4-wide node, < 0: leaf ~position,
// kEmptyLink: unused slot) and, per child, the binary slot (2*parent + side)
// whose box the per-frame fill copies (-1: unused).
struct __align__(16) Node4 {
  float4 lox, loy, loz, hix, hiy, hiz;
  int4 link;
  int4 src;
};
static_assert(sizeof(Node4) == 128, "4-wide node must be 128 bytes");
constexpr int kEmptyLink = (int)0x80000000;

// Triangle record in leaf (sorted) order, 48 B:
//   v0.xyz, w = original triangle index (bits)
//   e1 = v1 - v0, w = material index (bits)
//   e2 = v2 - v0, w = 0 (two-level mode: the triangle's body, bits)
// e1/e2 are the same FP32 differences the ray/triangle test and the normal use.
// Single level: world coordinates of the frame; two-level: rest coordinates.

// Two-level acceleration structure (§IV-B-3: one bottom level per mesh,
// built once; a top level over the instances, rebuilt every frame).  The
// bottom levels are the bodies' 4-wide subtrees of an LBVH built over the
// rest pose with body-prefixed keys; the top level is a 4-wide tree over
// entries that cut the bodies' bottom levels into subtrees (the world box of
// an entry: the 8 corners of its rest box through its body's matrix), whose
// leaf links are ~entry.  Per frame buffer: the top-level nodes and this
// record.
struct __align__(16) TlasInfo {
  float eps;    // shadow-ray lift: 1e-4 x diagonal of the union of the instances' world boxes
  float span;   // largest |coordinate| of the instance world boxes and the rest boxes (box-test slack)
  int32_t n;    // top-level 4-wide nodes in use (root = node 0; 0 = no instance)
  int32_t err;  // nonzero: the top level was not built (deeper than kTlasMaxDepth4)
};
static_assert(sizeof(TlasInfo) == 16, "top-level record must be 16 bytes");
static_assert(alignof(TlasInfo) == 16, "top-level record must be 16-byte aligned");
static_assert(alignof(Node4) == 16 && sizeof(Node4) % 16 == 0, "4-wide nodes are read with 16-byte loads");
constexpr int kMaxTlasBodies = 1024;   // bodies of a two-level scene (one block builds the top level)
constexpr int kTlasMaxDepth4 = 16;     // top-level 4-wide depths
constexpr int kExitInstance = 0x7ffffffe;  // traversal stack marker: back to the world ray

constexpr int kMaxLights = 8;
constexpr int kMaxHeight = 128;              // tree height is at most 97 (64 + 32 prefix bits + 1)
constexpr int kMaxDepth4 = 2 * kMaxHeight;   // 4-wide depths (each consumes >= 1 binary level)
constexpr int kCoarseBits = 4;               // Morton bits per axis above the body field (single level)
constexpr int kSortBits = 9;                 // 7 passes x 9 bits = 63-bit keys
constexpr int kSortBins = 1 << kSortBits;
constexpr int kSortPasses = 7;
constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;

// Device error word bits
constexpr uint32_t kErrStack = 1u;
constexpr uint32_t kErrTimeout = 2u;
constexpr uint32_t kErrCorrupt = 4u;  // a link outside the tree (never for a built tree)

struct CamParams {
  float ox, oy, oz;     // position
  float fx, fy, fz;     // forward
  float rx, ry, rz;     // right
  float ux, uy, uz;     // true up
  float sxs, sys;       // tan(vfov/2) * aspect, tan(vfov/2)
  int W, H, spp;
};

struct LightParams {
  int n;
  int type[kMaxLights];
  float x[kMaxLights], y[kMaxLights], z[kMaxLights];  // position or unit direction
  float I[kMaxLights];
};

struct MatParams {  // device pointer to [nmat*5] (albedo rgb, roughness, metallic)
  const float* p;
  int n;
};

// ---------------------------------------------------------------------------
// Host-side scene object
// ---------------------------------------------------------------------------
}  // namespace fire

struct fire_scene_s {
  int device = 0;
  int64_t nv = 0, nt = 0;
  int32_t nmat = 0, nbody = 0;
  // rest-pose inputs (library copies)
  float4* rest = nullptr;       // [nv]
  uint32_t* idx = nullptr;      // [nt*3] original order
  uint32_t* tmat = nullptr;     // [nt]   original order
  uint16_t* vbody = nullptr;    // [nv]
  float* mats = nullptr;        // [nmat*5] device copy
  std::vector<fire_material> h_mats;
  float* xf = nullptr;          // [nbody*12]
  // smooth shading: rest-pose vertex normals (nullptr = flat normals) and,
  // per frame buffer, the body matrices the buffer was refit with (the
  // normals turn with them while the next refit loads new matrices)
  float4* vnrm = nullptr;       // [nv]
  float* xf_buf[2] = {nullptr, nullptr};  // [nbody*12] each
  // LBVH
  bool built = false;
  int height = 0;               // internal levels on the longest root-leaf path
  uint64_t* keys = nullptr;     // sorted keys [nt]
  uint64_t* keys_orig = nullptr;// keys by original triangle [nt] (debug dump)
  uint32_t* order = nullptr;    // [nt] sorted position -> original triangle
  uint4* sidx = nullptr;        // [nt] (i0, i1, i2, orig) in sorted order
  uint32_t* smat = nullptr;     // [nt] material in sorted order
  fire::Node* nodes = nullptr;  // [max(nt-1, 1)]
  int32_t* leaf_slot = nullptr; // [nt]   2*parent + side
  int32_t* node_slot = nullptr; // [nt-1] 2*parent + side (root -1)
  uint32_t* counters = nullptr; // [nt-1] arrival counters of the build's refit
  uint8_t* lvl_aux = nullptr;   // device: 4-wide depth starts (i64 [kMaxDepth4]), collapse queue
                                //   lengths (u32 [kMaxDepth4]) and the node counter (u32)
  std::vector<int64_t> lvl4;    // host: 4-wide nodes of depth L are [lvl4[L], lvl4[L+1])
  float* stage = nullptr;       // [nt*6] refit: every leaf's box (sorted order)
  // treelet refit (single-level; lbvh.cu)
  int2* tl_node = nullptr;      // [nt] per list slot: 4-wide node, depth below its treelet root
  int4* tl_refs = nullptr;      // [nt] per list slot: children (list slot, ~leaf offset, kEmptyLink)
  int4* tl_info = nullptr;      // [nt] per treelet: list offset, nodes | max depth << 16, first, last leaf
  int32_t* tl_top = nullptr;    // [nt] top nodes (above the treelets), deepest depth first
  int64_t* tl_grp = nullptr;    // [kMaxDepth4 + 1] top-list start of each depth
  float* nunion = nullptr;      // [nt*6] union box of each treelet root and top node, by 4-wide node
  int32_t* tl_scratch = nullptr;// build scratch [12*nt + nt/1024 + 64 + kMaxDepth4]
  int ntl = 0;                  // treelets
  int64_t norphan = 0;          // leaves whose parent is a top node
  std::vector<int64_t> tl_grp_host;  // host copy of tl_grp
  fire::Node4* nodes4 = nullptr;// [max(nt, 1)] 4-wide traversal tree (current buffer)
  int64_t n4 = 0;               // 4-wide nodes in use
  int height4 = 0;              // 4-wide levels
  int32_t* q4 = nullptr;        // build queue: 2 x [nt] (binary node, 4-wide node) pairs
  float4* tris = nullptr;       // [nt*3] triangle records of the current buffer
  // Per-frame data is double-buffered (triangle records + 4-wide boxes): a
  // refit writes the buffer the last render did not read, so a refit on one
  // stream can overlap a render of the previous frame on another.  Events
  // order the two: ready_ev[b] after the build/refit that wrote buffer b,
  // used_ev[b] after the last render/shade enqueued on buffer b.
  float4* tris_buf[2] = {nullptr, nullptr};
  fire::Node4* nodes4_buf[2] = {nullptr, nullptr};
  int cur = 0;
  cudaEvent_t ready_ev[2] = {nullptr, nullptr};
  cudaEvent_t used_ev[2] = {nullptr, nullptr};
  bool ready_rec[2] = {false, false};
  bool used_rec[2] = {false, false};
  // build scratch
  float4* cen = nullptr;        // [nt]
  uint64_t* keys_alt = nullptr; // [nt]
  uint32_t* vals_alt = nullptr; // [nt]
  uint32_t* hist = nullptr;     // [kSortBins * nblocks]
  uint32_t* ctrl = nullptr;     // [32]: [0..7] task counters, [8] error word, [9..14] bounds,
                                //       [15] mixed-body count, [16..22] raster pass,
                                //       [24..31] shadow rays queued per light
  int32_t* rank = nullptr;      // [nt] original triangle -> sorted position
  // render scratch
  fire_gbuffer_rec* gscratch = nullptr;
  size_t gscratch_n = 0;
  double* bwd_partials = nullptr;  // per-block gradient partials of the backward
  size_t bwd_partials_n = 0;
  unsigned long long* rkeys = nullptr;  // raster keys, one per sample
  float4* rdirs = nullptr;              // raster ray directions, one per sample
  size_t rkeys_n = 0;
  int4* pieces = nullptr;          // raster piece queue
  size_t pieces_n = 0;
  int32_t* graze = nullptr;        // raster deferred-triangle list
  size_t graze_n = 0;
  float4* jobs = nullptr;          // shadow rays per task (sparse), 32 B per ray
  int32_t* qperm = nullptr;        // per light: the queue in task order, as slots of the sparse segment
  size_t jobs_n = 0;               // capacity in rays (each)
  int32_t* qaux = nullptr;         // per light: ray counts [tasks]; then per light: block sums [tasks / 1024]
  size_t qaux_n = 0;
  // two-level mode (fire_scene_set_two_level): bottom levels in
  // nodes4_buf[0] / tris_buf[0] (rest pose, built once), top level per frame
  // buffer
  bool two_level = false;
  int32_t* blas_root = nullptr;   // [nbody] 4-wide node of each body's bottom level (-1: no triangles)
  float4* body_box = nullptr;     // [2*nbody] rest box of each body (lo, hi; xyz)
  int32_t* body_range = nullptr;  // [2*nbody] first and last sorted position of each body (build)
  float* xf_ident = nullptr;      // [nbody*12] identity matrices (the bottom levels are built at rest)
  int32_t* inst = nullptr;        // [2*kMaxTlasBodies] top-level entries: (bottom-level node, body); -1: unused
  float4* inst_box = nullptr;     // [2*kMaxTlasBodies] rest box of each entry (lo, hi; xyz)
  fire::Node4* tlas_buf[2] = {nullptr, nullptr};       // [kMaxTlasBodies + 2] each
  fire::TlasInfo* tinfo_buf[2] = {nullptr, nullptr};
  fire::Node4* tlas = nullptr;    // current frame buffer's top level
  fire::TlasInfo* tinfo = nullptr;
  // batch cache (see batch.cu)
  void* batch = nullptr;
  int64_t iter_cap = 0;
  size_t bytes = 0;
  cudaStream_t last_stream = nullptr;
  bool rendered = false;        // a fire_render ran (fire_render_info)
  bool last_raster = false;     // its primary pass rasterised
  int64_t last_qseg = 0;        // its shadow queue: slots per light segment
  int last_nlights = 0;         // and lights
  void* prof = nullptr;         // fire::Profiler when enabled
};

namespace fire {

// ---------------------------------------------------------------------------
// Host helpers (fire_api.cu)
// ---------------------------------------------------------------------------
int set_error(int code, const std::string& msg);
// Double-buffered frame data (fire_api.cu): frame_acquire makes `st` wait
// for the build/refit of the current buffer; frame_release marks the work
// enqueued on `st` as the buffer's last user.
void frame_acquire(fire_scene_s* s, cudaStream_t st);
void frame_release(fire_scene_s* s, cudaStream_t st);
int cuda_check(cudaError_t e, const char* what);
cudaError_t dev_alloc(void** p, size_t bytes, size_t* counter);
int sm_count();
CamParams make_cam(const fire_camera& c);
int make_lights(const fire_light* lights, int n, LightParams* out);

// Stage profiler (fire_api.cu): event pairs around kernels, read lazily.
enum Stage { kStageRefit = 0, kStagePrimary = 1, kStageShadow = 2, kStageBuild = 3, kStageShadeGbuf = 4,
             kStageBackward = 5, kStageResolve = 6, kStageQueue = 7, kStages = 8 };
void prof_begin(fire_scene_s* s, int stage, cudaStream_t st);
// launches: kernels launched between prof_begin and prof_end
void prof_end(fire_scene_s* s, int stage, cudaStream_t st, int launches = 1);

// lbvh.cu
int lbvh_build(fire_scene_s* s, cudaStream_t st);
int lbvh_refit(fire_scene_s* s, cudaStream_t st);
int treelet_build(fire_scene_s* s, cudaStream_t st);
// two-level mode: top level of the current frame buffer from s->xf (one
// block; also copies the matrices into the buffer's xf_buf)
int tlas_build(fire_scene_s* s, cudaStream_t st);
int lbvh_validate(fire_scene_s* s, cudaStream_t st, uint32_t* bad_host);

// trace.cu
struct RenderArgs {
  const Node4* nodes4;
  int64_t n4;
  const float4* tris;
  int64_t nt;
  CamParams cam;
  LightParams lights;
  MatParams mats;
  int row_begin, row_end;
  int64_t iter_cap;
  uint32_t* ctrl;               // counters + error word
  const unsigned long long* rkeys;  // raster keys (primary in key mode) or nullptr
  const int32_t* rank;          // [nt] original triangle -> sorted position
  // smooth shading (vnrm != nullptr): rest vertex normals, the frame's body
  // matrices, sorted index records (the hit triangle's vertices), vertex -> body
  const float4* vnrm;
  const float* bxf;
  const uint4* sidx;
  const uint16_t* vbody;
  fire_gbuffer_rec* g;          // per-sample records
  float* out;                   // [H*W*4]
  // shadow-ray queue (single-frame path): light j's rays of task t sit at
  // [j*qseg + 32t, +qcnt[j*ntasks + t]) of the primary pass's sparse queue
  int32_t* qcnt;
  int64_t qseg;                 // 32 x tasks of the full image
  // two-level mode (tlas != nullptr): top level, its record, the top
  // level's entries (bottom-level node, body); bxf holds the frame's body
  // matrices
  const Node4* tlas;
  const TlasInfo* tinfo;
  const int32_t* inst;
  int nbody;
};
// Raster primary pass (raster.cu).  Words of fire_scene_s::ctrl it uses:
constexpr int kCtrlRasterPieces = 16;  // queued pieces
constexpr int kCtrlRasterCursor = 17;  // next piece to take
constexpr int kCtrlRasterFlag = 18;    // != 0: traversal fallback for this frame
constexpr int kCtrlRasterGraze = 19;   // deferred triangles
constexpr int kCtrlRasterParams = 20;  // [20..22] zn, rn, slack (float bits)
constexpr int kCtrlShadowLen = 24;     // [24..31] shadow rays queued per light
struct RasterArgs {
  const float4* tris;
  int64_t nt;
  const Node4* nodes4;
  CamParams cam;
  int row_begin, row_end;
  unsigned long long* keys;  // [W*H*spp] per-sample (t bits << 32 | original index)
  float4* dirs;              // [W*H*spp] per-sample ray direction (xyz)
  int4* pieces;              // queued pieces: triangle, x0|x1<<16, y0|y1<<16
  int64_t cap_pieces;
  int32_t* graze;            // deferred triangles (sorted positions)
  int64_t cap_graze;
  uint32_t* ctrl;
};
int raster_primary(fire_scene_s* s, const RasterArgs& r, cudaStream_t st);
// display.cu
int display_image(const float* hdr, int W, int H, float exposure, bool fxaa, float* scratch, uint8_t* out,
                  cudaStream_t st);
int render_frame(fire_scene_s* s, const RenderArgs& a, const fire_render_opts& o, cudaStream_t st);
int shade_from_gbuffer(fire_scene_s* s, const RenderArgs& a, const float* inten, cudaStream_t st);
int shade_backward(fire_scene_s* s, const RenderArgs& a, const float* inten, const float* dL,
                   float* dparams, float* dinten, cudaStream_t st);
int stack_for_height(int height, int requested);
// Smooth-shading inputs of the scene's current frame buffer (vnrm stays
// nullptr for a scene without vertex normals: flat shading).
inline void set_smooth_args(RenderArgs* a, const fire_scene_s* s) {
  a->vnrm = s->vnrm;
  a->bxf = s->xf_buf[s->cur];
  a->sidx = s->sidx;
  a->vbody = s->vbody;
}
// Two-level inputs of the scene's current frame buffer (tlas == nullptr: single level).
inline void set_level_args(RenderArgs* a, const fire_scene_s* s) {
  a->tlas = s->two_level ? s->tlas : nullptr;
  a->tinfo = s->two_level ? s->tinfo : nullptr;
  a->inst = s->inst;
  a->nbody = s->nbody;
}
// lbvh.cu: number of triangles whose three vertices do not share one body
int lbvh_count_mixed(fire_scene_s* s, cudaStream_t st, uint32_t* bad_host);
// display.cu: sRGB-encoded albedo of the [nmat*5] material table -> linear
int srgb_decode_materials(float* mats, int nmat, cudaStream_t st);
// stack entries the 4-wide traversal of this scene can need: 3 per level +
// sentinel; two-level: 3 per bottom and top level + sentinel + exit marker
inline int stack_need(const fire_scene_s* s) {
  return s->two_level ? 3 * (s->height4 + kTlasMaxDepth4) + 2 : 3 * s->height4 + 1;
}
int shade_backward_on(const RenderArgs& a, const float* inten, const float* dL, float* dparams, float* dinten,
                      double* acc, cudaStream_t st);

// batch.cu
int render_batch(const fire_scene* scenes, int nscenes, const fire_camera* cams,
                 const int32_t* cam_scene, int ncams, const fire_light* lights,
                 const int32_t* light_off, float* const* outs, const fire_render_opts* opts,
                 cudaStream_t st);
void batch_free(fire_scene_s* s);
int batch_last_info(int32_t* out4);
int batch_last_tuning(int32_t* out8, float* ms2);

// ---------------------------------------------------------------------------
// Device math with the fixed operation order
//   dot(a,b)   = fma(ax,bx, fma(ay,by, az*bz))
//   cross(a,b) = (fma(ay,bz, -(az*by)), fma(az,bx, -(ax*bz)), fma(ax,by, -(ay*bx)))
//   normalize(v) = v / sqrt(dot(v,v))
// ---------------------------------------------------------------------------
// (host and device: the host build of this file runs with -ffp-contract=off,
// and fmaf, '/' and sqrtf are correctly rounded on both, so a host call gives
// the device's bits -- the host emulation of the traversal relies on it)
__host__ __device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__host__ __device__ __forceinline__ float3 sub3(float3 a, float3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__host__ __device__ __forceinline__ float3 add3(float3 a, float3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__host__ __device__ __forceinline__ float3 neg3(float3 a) { return f3(-a.x, -a.y, -a.z); }
__host__ __device__ __forceinline__ float dot3(float3 a, float3 b) {
  return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z));
}
__host__ __device__ __forceinline__ float3 cross3(float3 a, float3 b) {
  return f3(fmaf(a.y, b.z, -(a.z * b.y)), fmaf(a.z, b.x, -(a.x * b.z)), fmaf(a.x, b.y, -(a.y * b.x)));
}
__host__ __device__ __forceinline__ float3 normalize3(float3 v) {
  float len = sqrtf(dot3(v, v));
  return f3(v.x / len, v.y / len, v.z / len);
}
__host__ __device__ __forceinline__ float3 xyz(float4 v) { return f3(v.x, v.y, v.z); }

// Bit casts (device intrinsics; memcpy on the host).
__host__ __device__ __forceinline__ float bits_as_float(uint32_t u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float f;
  memcpy(&f, &u, 4);
  return f;
#endif
}
__host__ __device__ __forceinline__ int float_as_bits(float f) {
#ifdef __CUDA_ARCH__
  return __float_as_int(f);
#else
  int i;
  memcpy(&i, &f, 4);
  return i;
#endif
}

// Ordered-integer image of a float (monotone), for exact atomic min/max.
__device__ __forceinline__ uint32_t f2ord(float f) {
  uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__host__ __device__ __forceinline__ float ord2f(uint32_t u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
#else
  uint32_t b = (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
  float f;
  memcpy(&f, &b, 4);
  return f;
#endif
}

}  // namespace fire
