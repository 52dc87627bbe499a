/*
 * fire.h -- C ABI of the B300 renderer hot path (libfire.so).
 *
 * The per-frame data-parallel path of the FIRE-3DV renderer (arXiv 2410.05095)
 * restated as CUDA for one B300 (sm_103a): an LBVH over a triangle scene
 * rebuilt or refit from per-body rigid transforms (§IV-B-3 acceleration
 * structure; §IV-C per-body world matrices every frame), supersampled primary
 * visibility (§IV-B-2 multisampling), any-hit shadow rays per light (§IV-B-3),
 * Cook-Torrance GGX shading (§IV-B-1) and a box-filter resolve into a linear
 * HDR image.  No graphics API is involved.
 *
 * Conventions for every call:
 *  - Return FIRE_OK (0) or a negative FIRE_ERR_* code; fire_last_error()
 *    gives a thread-local message for the last failure.
 *  - "device" pointers are CUDA device memory of the current device (for
 *    example a torch tensor's data_ptr()); "host" pointers are ordinary host
 *    memory.  The caller owns every buffer it passes in; the library never
 *    frees or retains caller pointers beyond the call, except that device
 *    work enqueued by the call reads/writes them asynchronously on `stream`.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls enqueue
 *    work and return without synchronising, except where stated.
 *  - Errors found on the device (traversal stack overflow, iteration cap) set
 *    a sticky per-scene error word that fire_sync_status() reports; bad input
 *    is rejected on the host (or by a counting kernel) and never traps on the
 *    device.
 *  - A scene handle must not be used from two host threads at once.
 */
#ifndef FIRE_H
#define FIRE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FIRE_OK 0
#define FIRE_ERR_INVALID_ARG (-1)
#define FIRE_ERR_OOM (-2)
#define FIRE_ERR_CUDA (-3)
#define FIRE_ERR_STACK_OVERFLOW (-4)
#define FIRE_ERR_TIMEOUT (-5)
#define FIRE_ERR_NOT_BUILT (-6)

typedef struct fire_scene_s* fire_scene; /* opaque, library-owned */

/* glTF metallic-roughness material (§IV-B-1): linear albedo in [0,1],
 * roughness in (0,1] (alpha = roughness^2 in the GGX term), metallic in [0,1]. */
typedef struct {
  float albedo[3];
  float roughness;
  float metallic;
} fire_material;

/* Pinhole camera: forward = normalize(target - pos), right = normalize(forward x up),
 * true up = right x forward; vfov_deg is the vertical field of view; image row 0
 * is the top.  spp is 1 (pixel centre) or 4 (rotated grid, offsets
 * (-1/8,-3/8), (3/8,-1/8), (-3/8,1/8), (1/8,3/8) pixels). */
typedef struct {
  float pos[3];
  float target[3];
  float up[3];
  float vfov_deg;
  int32_t width;
  int32_t height;
  int32_t spp;
} fire_camera;

/* Light (§IV-B-3 Fig. 5: several omnidirectional lights).  type 0: point light
 * at v with irradiance I/d^2; type 1: directional light, v = direction towards
 * the light (normalised by the library), irradiance I. */
typedef struct {
  int32_t type;
  float v[3];
  float intensity;
} fire_light;

/* Render options; a zeroed struct (or NULL) selects the defaults. */
typedef struct {
  int32_t row_begin;     /* render rows [row_begin, row_end) only; 0,0 = all rows.
                            Other rows of out_rgba are left untouched. */
  int32_t row_end;
  int32_t block_threads; /* threads per block of the batch kernels, a multiple of
                            32 up to 128 (0 = default); fire_render uses 128 */
  int32_t blocks_per_sm; /* persistent grid = SMs x blocks_per_sm (0 = default).
                            fire_render: applies to its primary pass only -- the
                            pass that a refit of the next frame on another stream
                            overlaps, so fewer blocks leave it room; the shadow
                            and resolve passes always run at full occupancy.
                            fire_render_batch: all of its kernels. */
  int32_t stack_depth;   /* traversal stack entries (0 = sufficient for the tree) */
  int32_t flags;         /* FIRE_RENDER_* bits, 0 by default */
} fire_render_opts;

/* Test hook: accept a stack_depth below the tree height.  A ray whose stack
 * would overflow drops the deepest pending subtree (its result may then be
 * wrong) and sets FIRE_ERR_STACK_OVERFLOW in the scene's error word; no
 * access ever leaves the stack. */
#define FIRE_RENDER_ALLOW_SHALLOW_STACK 1

/* Primary visibility method (the result is the same either way, bit for
 * bit: the nearest hit with the (t, original index) tie-break).  By default
 * fire_render traverses the tree (FIRE_RENDER_TRACE_PRIMARY states it).
 * FIRE_RENDER_RASTER_PRIMARY rasterises instead, like the paper's main pass
 * (§IV-A-1): one pass over the triangles, each testing the samples of its
 * conservative screen footprint with the same ray-triangle test, nearest
 * hit kept per sample by a 64-bit atomic minimum; it needs 24 B per sample
 * of extra scratch (allocated on first use) and hands a frame back to
 * traversal, on the device, when a footprint cannot be bounded (geometry
 * touching the camera, a full work list).  The two flags exclude each
 * other. */
#define FIRE_RENDER_TRACE_PRIMARY 2
#define FIRE_RENDER_RASTER_PRIMARY 4

/* One G-buffer record per sample, sample id = (y*W + x)*spp + k:
 * prim = original triangle index of the nearest hit (-1 = miss), t = hit
 * distance along the unit ray, vis = bit j set if light j was cast
 * (n.l > 0, n the shading normal) and unoccluded, bit 8+j set if light j
 * was cast. */
typedef struct {
  int32_t prim;
  float t;
  uint32_t vis;
  uint32_t pad;
} fire_gbuffer_rec;

/* ---------------------------------------------------------------- scenes */

/* Create a scene from a rest-pose triangle mesh (§IV-A-1 resource containers;
 * vertex pulling: flat vertex and index buffers).
 *   verts_xyzw [nv*4] device float  rest positions (w ignored)
 *   tri_idx    [nt*3] device uint32 vertex indices, each < nv
 *   tri_mat    [nt]   device uint32 material index, each < nmat
 *   vert_body  [nv]   device uint16 rigid body of each vertex, each < nbody
 *   mats       [nmat] host fire_material
 * The library copies all geometry (the caller may free its buffers after the
 * call returns; the copy is ordered on `stream`).  Out-of-range indices or
 * non-finite positions -> FIRE_ERR_INVALID_ARG (checked by a counting kernel;
 * this call synchronises `stream` once).  nt = 0 is a valid empty scene. */
int fire_scene_create(const float* verts_xyzw, int64_t nv, const uint32_t* tri_idx, int64_t nt,
                      const uint32_t* tri_mat, const uint16_t* vert_body,
                      const fire_material* mats, int32_t nmat, int32_t nbody, void* stream,
                      fire_scene* out);

/* Release all device memory of the scene (synchronises the device). */
int fire_scene_destroy(fire_scene s);

/* Replace the materials (host array of the same length nmat). */
int fire_scene_set_materials(fire_scene s, const fire_material* mats, int32_t nmat);

/* As fire_scene_set_materials; with FIRE_MATERIALS_SRGB_ALBEDO the albedo
 * values are sRGB-encoded (as glTF-like assets store colours) and are
 * decoded to linear on the device before shading (§IV-A-1: colour inputs are
 * converted from sRGB to linear): c / 12.92 for c <= 0.04045, else
 * ((c + 0.055) / 1.055)^2.4.  Roughness and metallic are not colours and are
 * kept.  Unknown flag bits -> FIRE_ERR_INVALID_ARG.  (fire_shade and
 * fire_shade_backward take their material table as an argument: it is
 * linear.) */
#define FIRE_MATERIALS_SRGB_ALBEDO 1
int fire_scene_set_materials_ex(fire_scene s, const fire_material* mats, int32_t nmat, int32_t flags);

/* Smooth shading (§IV-A-1: the main pass shades with the meshes' per-vertex
 * normal attribute).  normals: [nv*4] floats, rest-pose normal of each
 * vertex in xyz (w ignored), host or device memory (on_device != 0; host
 * values must be finite, else FIRE_ERR_INVALID_ARG); copied.  NULL returns
 * the scene to flat shading.  At a hit with barycentrics (u, v) (from the
 * same FP32 triangle test that found it) the shading normal is
 *   n_s = normalize(R (w0 n0 + u n1 + v n2)), w0 = (1 - u) - v,
 * evaluated as fma(v, n2, fma(u, n1, w0 n0)) per component, R = rotation of
 * the vertex's body in the matrices of the frame being rendered; n_s is
 * negated if it points away from the ray's side of the triangle, and a zero
 * interpolated normal keeps the geometric one.  n_s replaces the geometric
 * normal in the shading (n.l, n.v, n.h) and in the decision to cast a
 * shadow ray (n_s . l > 0); the shadow-ray origin stays lifted along the
 * geometric normal.  Applies to fire_render, fire_render_batch, fire_shade
 * and the backward calls.  Replacing or clearing the normals synchronises
 * the device (renders in flight may read them). */
int fire_scene_set_normals(fire_scene s, const float* normals, int32_t on_device, void* stream);

/* Scene sizes: out[0] = nv, out[1] = nt, out[2] = nmat, out[3] = nbody,
 * out[4] = binary tree height (after a build), out[5] = device bytes held,
 * out[6] = 4-wide traversal nodes, out[7] = 4-wide tree depth. */
int fire_scene_info(fire_scene s, int64_t* out8);

/* Facts of the scene's last fire_render; waits for the stream it ran on.
 *   out4 host int64[4]: out[0] = 1 if its primary pass rasterised, 0 if it
 *   traversed; out[1] = raster fallback reasons (bits: 1 geometry next to
 *   the camera, 2 non-finite projection, 4 a raster work list full; any bit means
 *   the traversal produced the primary hits); out[2] = raster pieces
 *   queued; out[3] = shadow rays queued.
 * Before any render -> zeros. */
int fire_render_info(fire_scene s, int64_t* out4);

/* ------------------------------------------------------------------ LBVH */

/* Build the LBVH (§IV-B-3 acceleration-structure build, restated as Karras
 * 2012): transform every vertex by its body's row-major 3x4 world matrix
 * (x' = fma(m0,x, fma(m1,y, fma(m2,z, m3))) per row), Morton keys of
 * triangle-box centroids over the centroid bounds, stable radix sort,
 * radix-tree topology, bottom-up boxes.  With several rigid bodies the key
 * holds a body field (body = that of the triangle's first vertex, B = bits
 * of (nbody - 1), m = min(21, (63 - B) / 3) Morton bits per axis) between
 * the Morton code's top 4 bits per axis and the rest:
 *   key = coarse << (B + 3(m-4)) | body << 3(m-4) | fine,
 * so inside each of the 16^3 coarse cells a body's triangles form one
 * subtree (the paper's per-mesh bottom levels under a top level, §IV-B-3)
 * and a refit under rigid motion widens only the nodes of the coarse levels
 * by the bodies' drift.  One body: the plain 63-bit Morton code.
 *   body_xforms [nbody*12] float, device if xforms_on_device else host
 * Non-finite matrices -> FIRE_ERR_INVALID_ARG (host check only for host
 * matrices; device matrices are the caller's responsibility). */
int fire_bvh_build(fire_scene s, const float* body_xforms, int32_t xforms_on_device, void* stream);

/* Refit with the topology of the last build (§IV-B-3 step 4: new transforms
 * each frame): re-transform the vertices and recompute every box bottom-up
 * (by treelets: subtrees of at most 32 4-wide nodes cut at build, each
 * refit by one warp from shared memory, then the nodes above them; every
 * box is the exact min/max over its triangles' vertices).
 * Before any build -> FIRE_ERR_NOT_BUILT.
 *
 * Frame buffers: the per-frame data (48-B triangle records and the 4-wide
 * boxes, 48·nt + 128·n4 bytes) exists twice.  A refit writes the buffer the
 * last render did not read and makes it current; renders, shading and the
 * backward read the current buffer.  The library orders the calls with CUDA
 * events across streams (a refit waits for the last reader of the buffer it
 * overwrites; a render waits for the refit that wrote its buffer), so a
 * refit issued on its own stream overlaps the previous frame's render, like
 * the paper's asynchronous compute queue.  Supported overlap: one refit
 * stream and one stream of render/shade calls per scene.  (Measured best:
 * render calls on a high-priority stream, the refit on a normal one, and
 * fire_render_opts.blocks_per_sm = 7.) */
int fire_bvh_refit(fire_scene s, const float* body_xforms, int32_t xforms_on_device, void* stream);

/* ---------------------------------------------------------------- render */

/* Render one frame: primary rays (spp per pixel), any-hit shadow rays per
 * light from the hit point lifted by eps = 1e-4 x scene-box diagonal along the
 * normal (§IV-B-3), Cook-Torrance GGX + Lambert shading with E = I/d^2 (point)
 * or I (directional) (§IV-B-1), box-filter mean of the samples (§IV-B-2).
 *   cam         host fire_camera
 *   lights      host fire_light[nlights], 0 <= nlights <= 8
 *   opts        host, or NULL for defaults
 *   out_rgba    device float [H*W*4]: rgb = linear radiance, a = hit fraction
 *   gbuf        device fire_gbuffer_rec [H*W*spp] or NULL (written if given)
 * Before any build -> FIRE_ERR_NOT_BUILT. */
int fire_render(fire_scene s, const fire_camera* cam, const fire_light* lights, int32_t nlights,
                const fire_render_opts* opts, float* out_rgba, fire_gbuffer_rec* gbuf,
                void* stream);

/* Test hooks of fire_render_batch (with block_threads or blocks_per_sm set,
 * which skips the search): FIRE_BATCH_TILE(n), n = 1..3, forces the tile
 * shape n of fire_batch_last_tuning's list; FIRE_BATCH_GRAB2 makes a warp
 * grab 2 tasks per atomic.  No other flag bit is accepted by the batch. */
#define FIRE_BATCH_TILE(n) ((n) << 8)
#define FIRE_BATCH_GRAB2 1024

/* Render many cameras over many scenes with three launches for the whole
 * batch (primary rays of every camera, one shared shadow-ray queue, shading
 * and resolve), replayed as one CUDA graph while the batch's shape and
 * buffers are unchanged (descriptor changes are re-uploaded before replay).
 * Unless opts fixes threads / blocks per SM, the first call of each batch
 * shape times candidate configurations (fire_batch_last_tuning).
 * Batch-wide limit: sum of W*H*spp below 2^28, else FIRE_ERR_INVALID_ARG.
 *   scenes     host fire_scene[nscenes] (each built)
 *   cams       host fire_camera[ncams]; cam_scene host int32[ncams] (< nscenes)
 *   lights     host fire_light[light_off[nscenes]]; light_off host int32[nscenes+1]
 *              (scene i uses lights[light_off[i] .. light_off[i+1]), at most 8)
 *   outs       host array of ncams device float pointers, [H_i*W_i*4] each
 *   opts       host or NULL; block_threads/blocks_per_sm/stack_depth of 0 are
 *              chosen by the library's autotuner (timed once per batch shape)
 * Results equal ncams separate fire_render calls bit for bit. */
int fire_render_batch(const fire_scene* scenes, int32_t nscenes, const fire_camera* cams,
                      const int32_t* cam_scene, int32_t ncams, const fire_light* lights,
                      const int32_t* light_off, float* const* outs, const fire_render_opts* opts,
                      void* stream);

/* ---------------------------------------------------------------- display */

/* Display output stage of a rendered image (§IV-A-1: Reinhard tone mapping
 * c' / (1 + c') of c' = exposure * c per channel, then gamma correction, the
 * inverse of the sRGB-to-linear conversion (IEC 61966-2-1); §IV-B-2: FXAA,
 * Lottes' post-process that blends along luma edges), then 8-bit rounding.
 *   hdr_rgba     device float [H*W*4] as written by fire_render (alpha =
 *                coverage, quantised as is)
 *   exposure     > 0
 *   flags        FIRE_DISPLAY_FXAA or 0
 *   scratch_rgba device float [H*W*4] (the tone-mapped image before FXAA),
 *                required with FIRE_DISPLAY_FXAA, else may be NULL
 *   out_rgba8    device uint8 [H*W*4] sRGB-encoded rgb + coverage
 * Stateless; asynchronous on `stream`.  Non-finite pixels give unspecified
 * bytes. */
#define FIRE_DISPLAY_FXAA 1
int fire_display(const float* hdr_rgba, int32_t width, int32_t height, float exposure, int32_t flags,
                 float* scratch_rgba, uint8_t* out_rgba8, void* stream);

/* ------------------------------------------------------- differentiable */

/* Shade a G-buffer (from fire_render) with device-side parameters, holding
 * visibility fixed: params [nmat*5] device float (albedo rgb, roughness,
 * metallic per material), inten [nlights] device float (replaces the lights'
 * intensities).  Writes out_rgba like fire_render. */
int fire_shade(fire_scene s, const fire_gbuffer_rec* gbuf, const fire_camera* cam,
               const fire_light* lights, int32_t nlights, const float* params, const float* inten,
               float* out_rgba, void* stream);

/* Backward of fire_shade: given dL/d(out_rgba) [H*W*4] device float (alpha
 * ignored), ACCUMULATE dL/dparams into dparams [nmat*5] and dL/dinten into
 * dinten [nlights] (device float; zero them first for a plain gradient).
 * Recomputes every shading input from the G-buffer (no stored intermediates). */
int fire_shade_backward(fire_scene s, const fire_gbuffer_rec* gbuf, const fire_camera* cam,
                        const fire_light* lights, int32_t nlights, const float* params,
                        const float* inten, const float* dL_drgba, float* dparams, float* dinten,
                        void* stream);

/* Allocation-free variant of fire_shade_backward (the paper has no
 * counterpart; it is a service for callers that cannot call cudaMalloc while
 * they run, e.g. a frame loop whose device memory is fixed at start-up, or a
 * host that must not pay the device synchronisation an allocation can cause).
 * Same arguments, results and accumulate-into-outputs behaviour as
 * fire_shade_backward, within the same tolerance; unlike it, the call is not
 * timed by the stage profiler (fire_profile_*), whose events it would have to
 * create.  Its scratch (counters and the FP64 accumulator) is a fixed array
 * inside the library image, 33,024 B per GPU that loads the library, held
 * until the process exits.
 *  - nmat*5 + nlights must be <= 4096, else FIRE_ERR_INVALID_ARG.
 *  - The first call on a device looks up the array's device address (with
 *    that device current).  That first call may also make CUDA load the
 *    library's module on the device (lazy module loading is CUDA's default),
 *    and the driver then allocates the array and may synchronise: make one
 *    warm-up call at start-up, before the frame loop and before any stream
 *    capture.  After a cudaDeviceReset in the process the cached address is
 *    stale: do not call this entry point again in that process.
 *  - Every call shares the one array and clears it on `stream` before use:
 *    calls whose GPU work overlaps (other streams or host threads) race. */
int fire_shade_backward_noalloc(fire_scene s, const fire_gbuffer_rec* gbuf, const fire_camera* cam,
                                const fire_light* lights, int32_t nlights, const float* params,
                                const float* inten, const float* dL_drgba, float* dparams, float* dinten,
                                void* stream);

/* ------------------------------------------------------------- utilities */

/* Copy internal state to host memory for checks (synchronises `stream` = the
 * library's last used stream of this scene).  what:
 *  0 morton codes by original triangle  uint64[nt]
 *  1 sorted order (position -> triangle) uint32[nt]
 *  2 children in Karras numbering       int32[(nt-1)*2] (internal i < nt-1,
 *                                       leaf at sorted position p = nt-1+p)
 *  3 parent by Karras code              int32[2nt-1] (root -1)
 *  4 node boxes by Karras code          float[(2nt-1)*6] (lo xyz, hi xyz)
 *  5 triangle records in sorted order  float[nt*12]: v0 xyz, original index
 *                                       (bits), e1 = v1-v0 xyz, material (bits),
 *                                       e2 = v2-v0 xyz, 0
 *  6 centroid bounds                    float[6]
 *  7 4-wide nodes of the current buffer  128 B x (4-wide node count, fire_scene_info
 *                                       out[6]); two-level: the bottom levels
 * two-level scenes only (else FIRE_ERR_INVALID_ARG):
 *  8 bottom-level root of each body      int32[nbody] (-1: no triangles)
 *  9 top level of the current buffer    128 B x 1026 (4-wide nodes; leaf link
 *                                       ~entry; unused nodes undefined)
 * 10 its record                         16 B: float eps, float span, int32 nodes
 *                                       in use, int32 error (nonzero: not built)
 * 11 body matrices of the current buffer float[nbody*12]
 * 13 the top level's entries            int32[1024*2]: (bottom-level 4-wide
 *                                       node, body) in body order; (-1, -1)
 *                                       past the last
 * any scene:
 * 12 the last fire_render's shadow rays in the order its shadow pass takes
 *    them (light by light, each light's rays in task order)  float[n*8]:
 *    origin xyz, t_max, unit direction xyz, sample * 8 + light (int bits);
 *    n = fire_render_info out[3] (0 before any render)
 * bytes must equal the exact size; otherwise FIRE_ERR_INVALID_ARG. */
int fire_debug_dump(fire_scene s, int32_t what, void* host_dst, size_t bytes);

/* Two-level acceleration structure (§IV-B-3: a bottom level per mesh built
 * once, a top level over the instances rebuilt every frame).  enable = 1:
 * the next fire_bvh_build builds one bottom level per body over the REST
 * pose (an LBVH with body-prefixed keys: each body's subtree, collapsed into
 * its own 4-wide tree, never refit), cuts each body's bottom level into
 * subtrees -- the top level's entries, so that a body whose parts lie far
 * apart gets tight boxes: breadth first from the body's root, a node whose
 * members are all inner nodes is replaced by them while the body's entries
 * stay within its share (1024 / bodies with triangles, at most 64) -- and
 * builds a top level over the entries' world boxes (the 8 corners of the
 * entry's rest box through its body's matrix, widened by
 * 2^-10 (1 + largest |coordinate|)); each fire_bvh_refit then only rebuilds
 * the top level (one block) into the other frame buffer.  Rays meet a body's
 * triangles in the body's frame, o' = R^T (o - t), d' = R^T d (R, t: the
 * body's 3x4 matrix); hits rank by (t of that ray, original index); the hit
 * normal is R (e1 x e2) of the rest triangle; the shadow-ray lift is 1e-4 x
 * the diagonal of the union of the instances' world boxes.
 * Requires every triangle's three vertices in one body and nbody <= 1024
 * (else FIRE_ERR_INVALID_ARG); not available with smooth normals, the raster
 * primary pass or fire_render_batch (FIRE_ERR_INVALID_ARG).  A top level
 * deeper than 16 4-wide levels sets FIRE_ERR_STACK_OVERFLOW.  Changing the
 * mode synchronises the device and leaves the scene unbuilt
 * (FIRE_ERR_NOT_BUILT until the next fire_bvh_build). */
int fire_scene_set_two_level(fire_scene s, int32_t enable);

/* Check of the traversal on the host (test hook; synchronises the device):
 * the scene's current structures (the 4-wide tree and its triangle records,
 * or the two-level structure) are copied to host memory and the traversal
 * code of the render kernels, compiled for the host, runs the n rays o3/d3
 * (host float[n*3]; the direction need not be unit).  any = 0: nearest hit
 * over (0, inf) -> prim (original index or -1) and t; any = 1: any hit in
 * (0, tmax[i]) other than triangle skip[i] (skip may be NULL) -> hit[i].
 * Every load is checked to lie inside the copied arrays and be aligned for
 * its width.  err_out: the traversal's error bits (1 stack, 2 iteration cap,
 * 4 a link outside the structure) | 0x100 if any load failed the check.
 * Outputs may be NULL. */
int fire_debug_trace_host(fire_scene s, const float* o3, const float* d3, const float* tmax, const int32_t* skip,
                          int64_t n, int32_t any, int32_t* prim, float* t, uint8_t* hit, uint32_t* err_out);

/* Traversal work and memory demand (measurement aid; synchronises the
 * device): the rays of fire_debug_trace_host, run the same way, in groups
 * of `group` consecutive rays (32: the rays a warp of the primary or shadow
 * pass takes together; the last group may be shorter).  A node step is one
 * fetch of a 4-wide node (7 x 16 B of its 128 B), a triangle test one fetch
 * of a 48-B record.  out8 (host int64[8]): [0] rays, [1] node steps, [2]
 * triangle tests, [3] the sum over groups of the distinct nodes the group
 * fetched, [4] of the distinct triangle records, [5] groups, [6] loads that
 * failed the check (0), [7] the traversal's error bits.  Demand bytes of a
 * group = distinct nodes x 128 + distinct records x 48: what its warp asks
 * of L2, once per node and record, when L1 keeps nothing between warps.
 * steps (host int32[n], may be NULL): each ray's node steps.
 * group < 1 -> FIRE_ERR_INVALID_ARG. */
int fire_debug_trace_stats(fire_scene s, const float* o3, const float* d3, const float* tmax, const int32_t* skip,
                           int64_t n, int32_t any, int32_t group, int64_t* out8, int32_t* steps);

/* Synchronise `stream`, then return and clear the scene's sticky device error
 * (FIRE_OK, FIRE_ERR_STACK_OVERFLOW or FIRE_ERR_TIMEOUT). */
int fire_sync_status(fire_scene s, void* stream);

/* Test hook: cap traversal loop iterations per ray (0 = no cap beyond the
 * library's safety bound).  A ray that hits the cap stops early and sets
 * FIRE_ERR_TIMEOUT in the scene's error word. */
int fire_debug_set_iteration_cap(fire_scene s, int64_t cap);

/* Test hook: make the next device allocation of this thread fail (n-th
 * allocation from now, 1 = next), to exercise FIRE_ERR_OOM paths. 0 = off. */
int fire_debug_fail_alloc(int32_t nth);

/* Stage timing with CUDA events recorded on the launching stream around each
 * stage of the scene's calls (off by default; negligible cost when on).
 * Stages: 0 refit, 1 primary pass (raster or traversal), 2 shadow rays,
 * 3 build (up to the binary tree; the 4-wide collapse is not included),
 * 4 G-buffer shading, 5 shading backward, 6 shading + resolve, 7 shadow
 * queue ordering (between 1 and 2: the rays put in task order).
 * fire_profile_read synchronises the pending events and returns, per stage,
 * the summed milliseconds and the number of kernel launches since the last
 * read (then resets). */
int fire_profile_enable(fire_scene s, int32_t enable);
int fire_profile_read(fire_scene s, double* ms8, int64_t* launches8);

/* Configuration of the last fire_render_batch launch: out4 = threads per
 * block, blocks per SM (0 = occupancy limit), stack depth, 1 if the autotuner
 * ran during that call. */
int fire_batch_last_config(int32_t* out4);

/* Measurement aid (the paper has no counterpart): one launch of
 * (SMs x 4) blocks of 256 threads that reads the `bytes` at `buf` `reps`
 * times with 16-B loads cached in L2 only (not L1) and folds them into
 * `sink` (device uint32[sink_words], sink_words >= 4 x SMs; its contents
 * have no meaning).  Timed by the caller with events on `stream`: bytes x
 * reps / time is the L2 read bandwidth for a buffer that fits in L2, the
 * DRAM read bandwidth for one that does not.  buf must be 16-B aligned and
 * bytes a positive multiple of 16, reps >= 1, else FIRE_ERR_INVALID_ARG. */
int fire_probe_read(const void* buf, int64_t bytes, int32_t reps, uint32_t* sink, int32_t sink_words,
                    void* stream);

/* The autotuner's record for the configuration of the last fire_render_batch
 * launch.  out8: threads per block, blocks per SM (0 = occupancy limit),
 * stack depth, task width in pixels at 1 spp, at 4 spp (a task is 32 / 8
 * pixels), tasks a warp grabs per atomic, candidates timed (0 if the caller
 * fixed the configuration), 1 if the search ran during that call.  ms2:
 * the best and the worst candidate's time (ms; 0 if none was timed).  The
 * search is coordinate-wise: threads x blocks per SM, then the tile shape
 * (8x4 / 4x2, 4x8 / 2x4, 16x2 / 8x1 pixels at 1 / 4 spp), then 2 tasks per
 * grab, then twice the stack the trees need. */
int fire_batch_last_tuning(int32_t* out8, float* ms2);

/* Thread-local message of the last failed call ("" if none). */
const char* fire_last_error(void);

/* Library version string. */
const char* fire_version(void);

#ifdef __cplusplus
}
#endif
#endif /* FIRE_H */
