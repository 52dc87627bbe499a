/* CPU oracle for the renderer hot path -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded C++ restatement of what the paper's per-frame
 * path computes (rigid-body pose update §IV-C, acceleration structure §IV-B-3,
 * visibility + PBR shading §IV-B-1, ray-traced hard shadows §IV-B-3,
 * multisample resolve §IV-B-2).  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header or
 * constant with the CUDA library.
 *
 * Pins: every function below is checked in tests/ against closed forms,
 * brute force or an independent construction (see the test files).
 * Parity unpinned: tree quality (node visits per ray) is only reported.
 */
#ifndef FIRE_ORACLE_H
#define FIRE_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { float albedo[3], roughness, metallic; } orc_material;
typedef struct { float pos[3], target[3], up[3], vfov_deg; int32_t width, height, spp; } orc_camera;
typedef struct { int32_t type; float v[3]; float intensity; } orc_light;

typedef struct orc_scene orc_scene;

orc_scene* orc_scene_new(const float* verts4, int64_t nv, const uint32_t* idx, int64_t nt,
                         const uint32_t* tri_mat, const uint16_t* vert_body,
                         const orc_material* mats, int32_t nmat, int32_t nbody);
void orc_scene_free(orc_scene* s);
int32_t orc_set_materials(orc_scene* s, const orc_material* mats, int32_t nmat);
/* Materials whose albedo is sRGB-encoded: decoded to linear (orc_srgb_decode)
 * once, then used as by orc_set_materials. */
int32_t orc_set_materials_srgb(orc_scene* s, const orc_material* mats, int32_t nmat);
float orc_srgb_decode(float c);

/* Smooth shading (§IV-A-1 per-vertex normals): rest-pose vertex normals
 * [nv*4] (xyz, w unused), interpolated with the hit's barycentrics, turned by
 * the body's rotation, normalised and put on the facing side of the
 * geometric normal; NULL = flat (geometric) normals.  orc_shading_normal
 * gives that normal for the ray (o, d) meeting triangle prim (world frame of
 * the last update). */
int32_t orc_set_normals(orc_scene* s, const float* nrm4);
void orc_shading_normal(const orc_scene* s, int32_t prim, const float* o, const float* d, float* n3);

/* Transform vertices by the per-body 3x4 row-major matrices; build the LBVH
 * (rebuild != 0 or first call) or refit it with the topology kept. */
int32_t orc_update(orc_scene* s, const float* xforms, int32_t rebuild);

/* Two-level mode (§IV-B-3 per-mesh bottom level + per-frame top level): each
 * body's triangles stay in rest coordinates and rays meet them in the body's
 * frame (object ray = R^T (o - t), R^T d); nearest hits rank by the object-
 * space t.  Every triangle's vertices must share one body, else -1.  Trace,
 * occlusion, rendering and the shading frame follow the mode. */
int32_t orc_set_two_level(orc_scene* s, int32_t enable);

/* what: 0 world verts [nv*3] f32; 1 morton codes by original tri [nt] u64;
 * 2 sorted order [nt] u32; 3 children [(nt-1)*2] i32 (Karras codes: internal
 * i < nt-1, leaf = nt-1+sorted position); 4 parent [2nt-1] i32 (root -1);
 * 5 node boxes [(2nt-1)*6] f32 (lo xyz, hi xyz) by Karras code;
 * 6 centroid bounds [6] f32; 7 scene box [6] f32 */
int32_t orc_get(const orc_scene* s, int32_t what, void* dst);

/* Nearest hit over [tmin, inf): prim = original triangle index or -1;
 * t2 = second-nearest hit distance over distinct triangles (inf if none). */
void orc_trace(const orc_scene* s, const float* o, const float* d, int64_t n, float tmin,
               int32_t use_bvh, int32_t* prim, float* t, float* u, float* v, float* t2);
/* Any hit with 0 < t < tmax, skipping triangle `skip` (or -1). out = 1 if occluded. */
void orc_occluded(const orc_scene* s, const float* o, const float* d, const float* tmax,
                  const int32_t* skip, int64_t n, int32_t use_bvh, uint8_t* out);

/* Primary ray of sample (x, y, k) of the camera. */
void orc_camera_ray(const orc_camera* c, int32_t x, int32_t y, int32_t k, float* o3, float* d3);

/* Render the listed samples (sample id = (y*W + x)*spp + k).  Per sample:
 * prim, t, t2, vis (bit j = light j cast and unoccluded; bit 8+j = light j cast),
 * radiance rgb. */
void orc_render_samples(const orc_scene* s, const orc_camera* c, const orc_light* L, int32_t nl,
                        const int64_t* ids, int64_t n, int32_t use_bvh,
                        int32_t* prim, float* t, float* t2, uint16_t* vis, float* rgb);
/* Render image rows [row0, row1) into rgba (row-major [H][W][4] of the full image). */
void orc_render_rows(const orc_scene* s, const orc_camera* c, const orc_light* L, int32_t nl,
                     int32_t row0, int32_t row1, int32_t use_bvh, float* rgba);

/* BRDF of the paper's Cook-Torrance variant (+ Lambert diffuse), per channel.
 * kmode 0: k = (r+1)^2/8, kmode 1: k = r^2/2. */
void orc_brdf_f32(const float* n, const float* v, const float* l, const orc_material* m,
                  float* f_rgb);
void orc_brdf_f64(const double* n, const double* v, const double* l, const double* albedo,
                  double rough, double metal, int32_t kmode, double* fd_rgb, double* fs_rgb);
double orc_ggx_d(double nh, double alpha);
double orc_schlick_f(double vh, double f0);
double orc_smith_g(double nl, double nv, double rough, int32_t kmode);

/* FP64 shading of fixed per-sample geometry (visibility held fixed) for the
 * gradient checks.  prim/t/vis come from orc_render_samples over all samples.
 * params: [nmat*5] (albedo rgb, roughness, metallic), inten: [nl].
 * orc_shade_f64 writes the rgb image [H*W*3]; orc_grad_f64 takes dL/dimage
 * [H*W*3] and writes dL/dparams [nmat*5] and dL/dinten [nl]. */
void orc_shade_f64(const orc_scene* s, const orc_camera* c, const orc_light* L, int32_t nl,
                   const int32_t* prim, const float* t, const uint16_t* vis,
                   const double* params, const double* inten, double* img);
void orc_grad_f64(const orc_scene* s, const orc_camera* c, const orc_light* L, int32_t nl,
                  const int32_t* prim, const float* t, const uint16_t* vis,
                  const double* params, const double* inten, const double* dimg,
                  double* dparams, double* dinten);

/* orc_shade_f64 with the hit frame recomputed in FP64 from the camera ray
 * and the world triangle (t, p, n, po, v, l, h, 1/d^2 all FP64; visibility
 * from vis).  Flat normals and single-level scenes only: -1 otherwise. */
int32_t orc_shade_f64_fresh(const orc_scene* s, const orc_camera* c, const orc_light* L, int32_t nl,
                            const int32_t* prim, const uint16_t* vis, const double* params,
                            const double* inten, double* img);

/* Shadow-ray offset epsilon = 1e-4 * scene-box diagonal. */
float orc_shadow_eps(const orc_scene* s);

/* Display output stage (§IV-A-1 Reinhard + gamma correction, §IV-B-2 FXAA):
 * hdr [H*W*4] linear rgb + coverage -> out [H*W*4] bytes (sRGB-encoded rgb,
 * coverage); gamma_out (optional, [H*W*4]) receives the tone-mapped,
 * encoded image before FXAA.  orc_srgb_encode / orc_root12_pow5 expose the
 * encode curve and its r^(5/12) for the pins. */
void orc_display(const float* hdr, int32_t W, int32_t H, float exposure, int32_t fxaa, float* gamma_out,
                 uint8_t* out);
float orc_srgb_encode(float r);
float orc_root12_pow5(float r);

#ifdef __cplusplus
}
#endif
#endif
