"""ctypes binding of libfire.so (include/fire.h): argument marshalling only.

Every step of the renderer runs in the library's CUDA kernels; this module
turns torch tensors into device pointers, Python records into the C structs,
and negative return codes into exceptions.  There is no CPU path: if the
library or a GPU is missing, calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfire.so")

FIRE_OK = 0
ERRORS = {-1: "FIRE_ERR_INVALID_ARG", -2: "FIRE_ERR_OOM", -3: "FIRE_ERR_CUDA",
          -4: "FIRE_ERR_STACK_OVERFLOW", -5: "FIRE_ERR_TIMEOUT", -6: "FIRE_ERR_NOT_BUILT"}

DUMP = {"morton": 0, "order": 1, "children": 2, "parent": 3, "boxes": 4, "tris": 5,
        "centroid_bounds": 6, "nodes4": 7, "blas_root": 8, "tlas": 9, "tlas_info": 10, "body_xforms": 11,
        "shadow_rays": 12, "top_entries": 13}

EXPORTS = ["fire_scene_create", "fire_scene_destroy", "fire_scene_set_materials", "fire_scene_info",
           "fire_bvh_build", "fire_bvh_refit", "fire_render", "fire_render_batch", "fire_shade",
           "fire_shade_backward", "fire_debug_dump", "fire_sync_status",
           "fire_debug_set_iteration_cap", "fire_debug_fail_alloc", "fire_batch_last_config",
           "fire_profile_enable", "fire_profile_read", "fire_shade_backward_noalloc", "fire_render_info",
           "fire_display", "fire_scene_set_materials_ex", "fire_scene_set_normals", "fire_probe_read",
           "fire_scene_set_two_level", "fire_debug_trace_host", "fire_batch_last_tuning", "fire_last_error",
           "fire_version", "fire_debug_trace_stats"]

STAGES = ["refit", "primary", "shadow", "build", "shade_gbuf", "backward", "resolve", "queue"]


class FireError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Material(C.Structure):
    _fields_ = [("albedo", C.c_float * 3), ("roughness", C.c_float), ("metallic", C.c_float)]


class Camera(C.Structure):
    _fields_ = [("pos", C.c_float * 3), ("target", C.c_float * 3), ("up", C.c_float * 3),
                ("vfov_deg", C.c_float), ("width", C.c_int32), ("height", C.c_int32), ("spp", C.c_int32)]


class Light(C.Structure):
    _fields_ = [("type", C.c_int32), ("v", C.c_float * 3), ("intensity", C.c_float)]


class RenderOpts(C.Structure):
    _fields_ = [("row_begin", C.c_int32), ("row_end", C.c_int32), ("block_threads", C.c_int32),
                ("blocks_per_sm", C.c_int32), ("stack_depth", C.c_int32), ("flags", C.c_int32)]


GBUF_REC_BYTES = 16
MAX_TOP_ENTRIES = 1024  # top-level entries of a two-level scene (its dump holds this many + 2 nodes)

_lib = None


def lib():
    """Load libfire.so (built by _build.build()); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libfire.so not built ({LIB_PATH}); run paper_2410_05095_b300._build.build()")
        L = C.CDLL(LIB_PATH)
        P, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
        sig = {
            "fire_scene_create": [P, i64, P, i64, P, P, P, i32, i32, P, P],
            "fire_scene_destroy": [P],
            "fire_scene_set_materials": [P, P, i32],
            "fire_scene_info": [P, P],
            "fire_bvh_build": [P, P, i32, P],
            "fire_bvh_refit": [P, P, i32, P],
            "fire_render": [P, P, P, i32, P, P, P, P],
            "fire_render_batch": [P, i32, P, P, i32, P, P, P, P, P],
            "fire_shade": [P, P, P, P, i32, P, P, P, P],
            "fire_shade_backward": [P, P, P, P, i32, P, P, P, P, P, P],
            "fire_debug_dump": [P, i32, P, C.c_size_t],
            "fire_sync_status": [P, P],
            "fire_debug_set_iteration_cap": [P, i64],
            "fire_debug_fail_alloc": [i32],
            "fire_batch_last_config": [P],
            "fire_profile_enable": [P, i32],
            "fire_profile_read": [P, P, P],
            "fire_shade_backward_noalloc": [P, P, P, P, i32, P, P, P, P, P, P],
            "fire_render_info": [P, P],
            "fire_display": [P, i32, i32, C.c_float, i32, P, P, P],
            "fire_scene_set_materials_ex": [P, P, i32, i32],
            "fire_scene_set_normals": [P, P, i32, P],
            "fire_probe_read": [P, i64, i32, P, i32, P],
            "fire_scene_set_two_level": [P, i32],
            "fire_debug_trace_host": [P, P, P, P, P, i64, i32, P, P, P, P],
            "fire_debug_trace_stats": [P, P, P, P, P, i64, i32, i32, P, P],
            "fire_batch_last_tuning": [P, P],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        L.fire_last_error.restype = C.c_char_p
        L.fire_last_error.argtypes = []
        L.fire_version.restype = C.c_char_p
        L.fire_version.argtypes = []
        _lib = L
    return _lib


def _check(code: int):
    if code != FIRE_OK:
        raise FireError(code, lib().fire_last_error().decode())


def _ptr(t) -> C.c_void_p:
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return C.c_void_p(t.data_ptr())
    return t.ctypes.data_as(C.c_void_p)


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def make_camera(cam) -> Camera:
    c = Camera()
    c.pos[:] = [float(v) for v in cam.pos]
    c.target[:] = [float(v) for v in cam.target]
    c.up[:] = [float(v) for v in cam.up]
    c.vfov_deg, c.width, c.height, c.spp = float(cam.vfov_deg), int(cam.width), int(cam.height), int(cam.spp)
    return c


def make_lights(lights):
    arr = (Light * max(1, len(lights)))()
    for i, l in enumerate(lights):
        arr[i].type = int(l.type)
        arr[i].v[:] = [float(v) for v in l.v]
        arr[i].intensity = float(l.intensity)
    return arr


def make_materials(mats: np.ndarray):
    arr = (Material * len(mats))()
    for i, m in enumerate(mats):
        arr[i].albedo[:] = [float(a) for a in m["albedo"]]
        arr[i].roughness = float(m["roughness"])
        arr[i].metallic = float(m["metallic"])
    return arr


def make_opts(**kw) -> RenderOpts:
    o = RenderOpts()
    for k, v in kw.items():
        setattr(o, k, int(v))
    return o


class Scene:
    """A library-owned scene (fire_scene).  Inputs are copied at creation."""

    def __init__(self, verts, idx, tri_mat, vert_body, mats: np.ndarray, nbody: int, stream=None):
        """verts [nv,4] f32, idx [nt,3] u32-as-int32, tri_mat [nt] i32, vert_body [nv] i16/u16:
        torch CUDA tensors (or numpy arrays, copied by the library from host)."""
        self.h = C.c_void_p()
        self.nv, self.nt = int(verts.shape[0]), int(idx.shape[0])
        self.nmat, self.nbody = len(mats), int(nbody)
        self._mats = make_materials(mats)
        _check(lib().fire_scene_create(_ptr(verts), self.nv, _ptr(idx), self.nt, _ptr(tri_mat),
                                       _ptr(vert_body), C.cast(self._mats, C.c_void_p), self.nmat,
                                       self.nbody, _stream(stream), C.byref(self.h)))

    @classmethod
    def from_numpy(cls, scene, device="cuda", stream=None):
        """Upload a scenegen.Scene's arrays to the GPU, then create the scene."""
        import torch
        t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a).view(dt)).to(device)
        return cls(t(scene.verts, np.float32), t(scene.idx, np.int32), t(scene.tri_mat, np.int32),
                   t(scene.vert_body, np.int16), scene.mats, scene.nbody, stream)

    def destroy(self):
        if self.h:
            _check(lib().fire_scene_destroy(self.h))
            self.h = C.c_void_p()

    def __del__(self):
        try:
            if self.h and _lib is not None:
                lib().fire_scene_destroy(self.h)
                self.h = C.c_void_p()
        except Exception:
            pass

    def set_materials(self, mats: np.ndarray, srgb: bool = False):
        """Replace the materials; srgb=True: albedo is sRGB-encoded (decoded on the device)."""
        self._mats = make_materials(mats)
        _check(lib().fire_scene_set_materials_ex(self.h, C.cast(self._mats, C.c_void_p), len(mats),
                                                 1 if srgb else 0))

    def set_normals(self, normals, stream=None):
        """Rest-pose vertex normals [nv, 4] (numpy host array or CUDA tensor) for
        smooth shading; None returns to flat shading (see include/fire.h)."""
        if normals is None:
            _check(lib().fire_scene_set_normals(self.h, None, 0, _stream(stream)))
            return
        dev = hasattr(normals, "is_cuda") and normals.is_cuda
        if dev:
            assert normals.dtype.itemsize == 4 and normals.numel() == 4 * self.nv and normals.is_contiguous()
            x = normals
        else:
            x = np.ascontiguousarray(np.asarray(normals, np.float32).reshape(self.nv, 4))
        _check(lib().fire_scene_set_normals(self.h, _ptr(x), int(dev), _stream(stream)))

    def info(self) -> dict:
        out = (C.c_int64 * 8)()
        _check(lib().fire_scene_info(self.h, out))
        return dict(nv=out[0], nt=out[1], nmat=out[2], nbody=out[3], height=out[4], bytes=out[5],
                    n4=out[6], depth4=out[7])

    def render_info(self) -> dict:
        """Facts of the last render (waits for it): primary method, raster
        fallback reasons, raster pieces queued, shadow rays queued."""
        out = (C.c_int64 * 4)()
        _check(lib().fire_render_info(self.h, out))
        return dict(raster=bool(out[0]), fallback=out[1], pieces=out[2], shadow_rays=out[3])

    def build(self, xforms, stream=None):
        """xforms: [nbody,12] f32 -- a CUDA tensor (device) or numpy/CPU tensor (host)."""
        dev = hasattr(xforms, "is_cuda") and xforms.is_cuda
        x = xforms if dev else np.ascontiguousarray(np.asarray(xforms, np.float32))
        _check(lib().fire_bvh_build(self.h, _ptr(x), int(dev), _stream(stream)))

    def refit(self, xforms, stream=None):
        dev = hasattr(xforms, "is_cuda") and xforms.is_cuda
        x = xforms if dev else np.ascontiguousarray(np.asarray(xforms, np.float32))
        _check(lib().fire_bvh_refit(self.h, _ptr(x), int(dev), _stream(stream)))

    def render(self, cam, lights, out=None, gbuf=None, opts: RenderOpts | None = None, stream=None):
        """Render into out ([H,W,4] f32 CUDA tensor, allocated if None); gbuf:
        optional [H*W*spp, 4] int32 CUDA tensor (fire_gbuffer_rec records)."""
        import torch
        if out is None:
            out = torch.zeros((cam.height, cam.width, 4), dtype=torch.float32, device="cuda")
        c, L = make_camera(cam), make_lights(lights)
        _check(lib().fire_render(self.h, C.byref(c), C.cast(L, C.c_void_p), len(lights),
                                 C.byref(opts) if opts is not None else None, _ptr(out), _ptr(gbuf),
                                 _stream(stream)))
        return out

    def shade(self, gbuf, cam, lights, params, inten, out=None, stream=None):
        import torch
        if out is None:
            out = torch.zeros((cam.height, cam.width, 4), dtype=torch.float32, device="cuda")
        c, L = make_camera(cam), make_lights(lights)
        _check(lib().fire_shade(self.h, _ptr(gbuf), C.byref(c), C.cast(L, C.c_void_p), len(lights),
                                _ptr(params), _ptr(inten), _ptr(out), _stream(stream)))
        return out

    def shade_backward(self, gbuf, cam, lights, params, inten, dL, dparams, dinten, stream=None):
        c, L = make_camera(cam), make_lights(lights)
        _check(lib().fire_shade_backward(self.h, _ptr(gbuf), C.byref(c), C.cast(L, C.c_void_p), len(lights),
                                         _ptr(params), _ptr(inten), _ptr(dL), _ptr(dparams), _ptr(dinten),
                                         _stream(stream)))

    def shade_backward_noalloc(self, gbuf, cam, lights, params, inten, dL, dparams, dinten, stream=None):
        """fire_shade_backward without any allocation (scratch in a fixed
        library array; see include/fire.h)."""
        c, L = make_camera(cam), make_lights(lights)
        _check(lib().fire_shade_backward_noalloc(self.h, _ptr(gbuf), C.byref(c), C.cast(L, C.c_void_p),
                                                 len(lights), _ptr(params), _ptr(inten), _ptr(dL),
                                                 _ptr(dparams), _ptr(dinten), _stream(stream)))

    def set_two_level(self, enable: bool = True):
        """Two-level acceleration structure (bottom level per body at rest,
        top level rebuilt every frame); takes effect at the next build."""
        _check(lib().fire_scene_set_two_level(self.h, int(bool(enable))))

    def trace_host(self, o, d, tmax=None, skip=None, any_hit=False):
        """Host emulation of the traversal (fire_debug_trace_host): returns
        (prim, t, hit, error bits) for rays o, d [n, 3]."""
        o = np.ascontiguousarray(o, np.float32)
        d = np.ascontiguousarray(d, np.float32)
        n = len(o)
        prim, t = np.zeros(n, np.int32), np.zeros(n, np.float32)
        hit = np.zeros(n, np.uint8)
        err = C.c_uint32(0)
        tm = None if tmax is None else np.ascontiguousarray(tmax, np.float32)
        sk = None if skip is None else np.ascontiguousarray(skip, np.int32)
        _check(lib().fire_debug_trace_host(self.h, _ptr(o), _ptr(d), _ptr(tm), _ptr(sk), n, int(bool(any_hit)),
                                           _ptr(prim), _ptr(t), _ptr(hit), C.byref(err)))
        return prim, t, hit.astype(bool), int(err.value)

    def trace_stats(self, o, d, tmax=None, skip=None, any_hit=False, group=32, per_ray=False) -> dict:
        """Traversal work and demand of rays o, d [n, 3] in groups of `group`
        (fire_debug_trace_stats); per_ray: also each ray's node steps."""
        o = np.ascontiguousarray(o, np.float32)
        d = np.ascontiguousarray(d, np.float32)
        tm = None if tmax is None else np.ascontiguousarray(tmax, np.float32)
        sk = None if skip is None else np.ascontiguousarray(skip, np.int32)
        out = np.zeros(8, np.int64)
        steps = np.zeros(len(o), np.int32) if per_ray else None
        _check(lib().fire_debug_trace_stats(self.h, _ptr(o), _ptr(d), _ptr(tm), _ptr(sk), len(o),
                                            int(bool(any_hit)), int(group), _ptr(out), _ptr(steps)))
        keys = ("rays", "node_steps", "tri_tests", "group_nodes", "group_tris", "groups", "bad_loads", "err")
        res = dict(zip(keys, (int(x) for x in out)))
        if per_ray:
            res["steps"] = steps
        return res

    def dump(self, what: str) -> np.ndarray:
        T = self.nt
        nb = self.nbody
        shapes = {"morton": (np.uint64, (T,)), "order": (np.uint32, (T,)),
                  "children": (np.int32, (max(T - 1, 0), 2)), "parent": (np.int32, (max(2 * T - 1, 0),)),
                  "boxes": (np.float32, (max(2 * T - 1, 0), 6)), "tris": (np.float32, (T, 12)),
                  "centroid_bounds": (np.float32, (6,)), "nodes4": (np.float32, (self.info()["n4"], 32)),
                  "blas_root": (np.int32, (nb,)), "tlas": (np.float32, (MAX_TOP_ENTRIES + 2, 32)),
                  "tlas_info": (np.float32, (4,)), "body_xforms": (np.float32, (nb, 12)),
                  "top_entries": (np.int32, (MAX_TOP_ENTRIES, 2))}
        if what == "shadow_rays":
            shapes[what] = (np.float32, (self.render_info()["shadow_rays"], 8))
        dt, shp = shapes[what]
        out = np.zeros(shp, dt)
        _check(lib().fire_debug_dump(self.h, DUMP[what], _ptr(out), out.nbytes))
        return out

    def sync_status(self, stream=None) -> int:
        """Synchronise and return (and clear) the sticky device error code (0 = OK)."""
        return int(lib().fire_sync_status(self.h, _stream(stream)))

    def set_iteration_cap(self, cap: int):
        _check(lib().fire_debug_set_iteration_cap(self.h, int(cap)))

    def profile(self, enable: bool = True):
        _check(lib().fire_profile_enable(self.h, int(enable)))

    def profile_read(self) -> dict:
        """{stage: (milliseconds, launches)} since the last read (synchronises)."""
        ms, n = (C.c_double * 8)(), (C.c_int64 * 8)()
        _check(lib().fire_profile_read(self.h, ms, n))
        return {name: (ms[i], n[i]) for i, name in enumerate(STAGES)}


def display(hdr, exposure: float = 1.0, fxaa: bool = True, out=None, scratch=None, stream=None):
    """Display stage of an [H, W, 4] float CUDA image from render(): Reinhard
    tone map, sRGB encode, optional FXAA -> [H, W, 4] uint8 CUDA tensor."""
    import torch
    H, W = int(hdr.shape[0]), int(hdr.shape[1])
    if out is None:
        out = torch.empty((H, W, 4), dtype=torch.uint8, device=hdr.device)
    if fxaa and scratch is None:
        scratch = torch.empty((H, W, 4), dtype=torch.float32, device=hdr.device)
    _check(lib().fire_display(_ptr(hdr), W, H, float(exposure), 1 if fxaa else 0, _ptr(scratch) if fxaa else None,
                              _ptr(out), _stream(stream)))
    return out


def render_batch(scenes, cams, cam_scene, lights_per_scene, outs, opts: RenderOpts | None = None, stream=None):
    """One persistent launch (graph-replayed) for all cameras."""
    n = len(scenes)
    hs = (C.c_void_p * n)(*[s.h.value for s in scenes])
    cs = (Camera * len(cams))(*[make_camera(c) for c in cams])
    csc = (C.c_int32 * len(cams))(*cam_scene)
    flat = [l for ls in lights_per_scene for l in ls]
    L = make_lights(flat)
    off = [0]
    for ls in lights_per_scene:
        off.append(off[-1] + len(ls))
    lo = (C.c_int32 * (n + 1))(*off)
    op = (C.c_void_p * len(outs))(*[o.data_ptr() for o in outs])
    _check(lib().fire_render_batch(hs, n, cs, csc, len(cams), C.cast(L, C.c_void_p), lo, op,
                                   C.byref(opts) if opts is not None else None, _stream(stream)))


def batch_last_config() -> dict:
    out = (C.c_int32 * 4)()
    _check(lib().fire_batch_last_config(out))
    return dict(threads=out[0], blocks_per_sm=out[1], stack=out[2], tuned=out[3])


def batch_last_tuning() -> dict:
    """The autotuner's record for the last batch launch (fire_batch_last_tuning)."""
    out = (C.c_int32 * 8)()
    ms = (C.c_float * 2)()
    _check(lib().fire_batch_last_tuning(out, ms))
    return dict(threads=out[0], blocks_per_sm=out[1], stack=out[2], tile_w_1spp=out[3], tile_w_4spp=out[4],
                grab=out[5], tried=out[6], tuned_now=bool(out[7]), best_ms=ms[0], worst_ms=ms[1])


def fail_next_alloc(nth: int = 1):
    _check(lib().fire_debug_fail_alloc(nth))


def version() -> str:
    return lib().fire_version().decode()


def probe_read(buf, reps: int, sink, stream=None):
    """fire_probe_read over a contiguous device tensor `buf` (all of its
    bytes, `reps` times); `sink` is a device int32/uint32 tensor of at least
    4 words per SM."""
    _check(lib().fire_probe_read(_ptr(buf), buf.numel() * buf.element_size(), int(reps), _ptr(sink),
                                 int(sink.numel()), _stream(stream)))
