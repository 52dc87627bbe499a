"""CPU oracle for the renderer hot path -- TEST INFRASTRUCTURE ONLY.

Only tests/, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
(and its ``--impl reference`` arm) may import this package.  The product
library never does: it shares no code with the oracle, and the oracle shares
none with it.

The oracle is ``fire_oracle.cpp``: a plain single-threaded C++17 restatement
of the paper's per-frame path (§IV-C pose update, §IV-B-3 acceleration
structure and shadow rays, §IV-B-1 Cook-Torrance shading, §IV-B-2 multisample
resolve).  This module compiles it with g++ and wraps its C API with ctypes
and numpy.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fire_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle (g++ -O2 -ffp-contract=off: no implicit FMA)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "fire_oracle.h"))):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-Wall", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


class Material(C.Structure):
    _fields_ = [("albedo", C.c_float * 3), ("roughness", C.c_float), ("metallic", C.c_float)]


class Camera(C.Structure):
    _fields_ = [("pos", C.c_float * 3), ("target", C.c_float * 3), ("up", C.c_float * 3),
                ("vfov_deg", C.c_float), ("width", C.c_int32), ("height", C.c_int32),
                ("spp", C.c_int32)]


class Light(C.Structure):
    _fields_ = [("type", C.c_int32), ("v", C.c_float * 3), ("intensity", C.c_float)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        P = C.c_void_p
        i64, i32 = C.c_int64, C.c_int32
        L.orc_scene_new.restype = P
        L.orc_scene_new.argtypes = [P, i64, P, i64, P, P, P, i32, i32]
        L.orc_scene_free.argtypes = [P]
        L.orc_set_materials.argtypes = [P, P, i32]
        L.orc_update.argtypes = [P, P, i32]
        L.orc_get.argtypes = [P, i32, P]
        L.orc_trace.argtypes = [P, P, P, i64, C.c_float, i32, P, P, P, P, P]
        L.orc_occluded.argtypes = [P, P, P, P, P, i64, i32, P]
        L.orc_camera_ray.argtypes = [P, i32, i32, i32, P, P]
        L.orc_render_samples.argtypes = [P, P, P, i32, P, i64, i32, P, P, P, P, P]
        L.orc_render_rows.argtypes = [P, P, P, i32, i32, i32, i32, P]
        L.orc_brdf_f32.argtypes = [P, P, P, P, P]
        L.orc_brdf_f64.argtypes = [P, P, P, P, C.c_double, C.c_double, i32, P, P]
        L.orc_ggx_d.restype = C.c_double
        L.orc_ggx_d.argtypes = [C.c_double, C.c_double]
        L.orc_schlick_f.restype = C.c_double
        L.orc_schlick_f.argtypes = [C.c_double, C.c_double]
        L.orc_smith_g.restype = C.c_double
        L.orc_smith_g.argtypes = [C.c_double, C.c_double, C.c_double, i32]
        L.orc_shade_f64.argtypes = [P, P, P, i32, P, P, P, P, P, P]
        L.orc_grad_f64.argtypes = [P, P, P, i32, P, P, P, P, P, P, P, P]
        L.orc_shade_f64_fresh.argtypes = [P, P, P, i32, P, P, P, P, P]
        L.orc_shade_f64_fresh.restype = i32
        L.orc_shadow_eps.restype = C.c_float
        L.orc_shadow_eps.argtypes = [P]
        L.orc_display.argtypes = [P, i32, i32, C.c_float, i32, P, P]
        L.orc_set_two_level.argtypes = [P, i32]
        L.orc_srgb_encode.restype = C.c_float
        L.orc_srgb_encode.argtypes = [C.c_float]
        L.orc_root12_pow5.restype = C.c_float
        L.orc_root12_pow5.argtypes = [C.c_float]
        L.orc_set_materials_srgb.argtypes = [P, P, i32]
        L.orc_srgb_decode.restype = C.c_float
        L.orc_srgb_decode.argtypes = [C.c_float]
        L.orc_set_normals.argtypes = [P, P]
        L.orc_shading_normal.argtypes = [P, i32, P, P, P]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def make_camera(cam) -> Camera:
    c = Camera()
    c.pos[:] = list(cam.pos)
    c.target[:] = list(cam.target)
    c.up[:] = list(cam.up)
    c.vfov_deg, c.width, c.height, c.spp = cam.vfov_deg, cam.width, cam.height, cam.spp
    return c


def make_lights(lights):
    arr = (Light * max(1, len(lights)))()
    for i, l in enumerate(lights):
        arr[i].type = l.type
        arr[i].v[:] = list(l.v)
        arr[i].intensity = l.intensity
    return arr


def make_materials(mats: np.ndarray):
    arr = (Material * len(mats))()
    for i, m in enumerate(mats):
        arr[i].albedo[:] = [float(a) for a in m["albedo"]]
        arr[i].roughness = float(m["roughness"])
        arr[i].metallic = float(m["metallic"])
    return arr


class OracleScene:
    """One scene held by the oracle (rest pose, LBVH, per-frame state)."""

    def __init__(self, scene):
        self.scene = scene
        self._keep = [np.ascontiguousarray(scene.verts, np.float32),
                      np.ascontiguousarray(scene.idx, np.uint32),
                      np.ascontiguousarray(scene.tri_mat, np.uint32),
                      np.ascontiguousarray(scene.vert_body, np.uint16)]
        self.mats = make_materials(scene.mats)
        v, i, m, b = self._keep
        self.h = lib().orc_scene_new(_p(v), scene.nv, _p(i), scene.nt, _p(m), _p(b),
                                     C.cast(self.mats, C.c_void_p), len(scene.mats), scene.nbody)
        if not self.h:
            raise ValueError("oracle rejected the scene")
        self.nt, self.nv = scene.nt, scene.nv

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_scene_free(self.h)
            self.h = None

    def set_materials(self, mats: np.ndarray):
        self.mats = make_materials(mats)
        assert lib().orc_set_materials(self.h, C.cast(self.mats, C.c_void_p), len(mats)) == 0

    def set_materials_srgb(self, mats: np.ndarray):
        """Materials whose albedo is sRGB-encoded (decoded once to linear)."""
        self.mats = make_materials(mats)
        assert lib().orc_set_materials_srgb(self.h, C.cast(self.mats, C.c_void_p), len(mats)) == 0

    def set_normals(self, normals):
        """Rest-pose vertex normals [nv, 4] (smooth shading); None = flat."""
        if normals is None:
            self._nrm = None
            lib().orc_set_normals(self.h, None)
            return
        self._nrm = np.ascontiguousarray(normals, np.float32).reshape(self.nv, 4)
        lib().orc_set_normals(self.h, _p(self._nrm))

    def shading_normal(self, prim: int, o, d) -> np.ndarray:
        """Shading normal of the ray (o, d) meeting triangle prim."""
        o = np.ascontiguousarray(o, np.float32)
        d = np.ascontiguousarray(d, np.float32)
        n = np.zeros(3, np.float32)
        lib().orc_shading_normal(self.h, int(prim), _p(o), _p(d), _p(n))
        return n

    def update(self, xforms: np.ndarray, rebuild: bool = False):
        x = np.ascontiguousarray(xforms, np.float32).reshape(-1)
        lib().orc_update(self.h, _p(x), int(rebuild))

    def set_two_level(self, enable: bool = True):
        """Two-level mode: bodies as instances of rest-space geometry."""
        if lib().orc_set_two_level(self.h, int(bool(enable))) != 0:
            raise ValueError("two-level mode needs every triangle's vertices in one body")

    def get(self, what: str) -> np.ndarray:
        T = self.nt
        spec = {"world": (0, np.float32, (self.nv, 3)), "morton": (1, np.uint64, (T,)),
                "order": (2, np.uint32, (T,)), "children": (3, np.int32, (max(T - 1, 0), 2)),
                "parent": (4, np.int32, (max(2 * T - 1, 0),)),
                "boxes": (5, np.float32, (max(2 * T - 1, 0), 6)),
                "centroid_bounds": (6, np.float32, (6,)), "scene_box": (7, np.float32, (6,))}[what]
        out = np.zeros(spec[2], dtype=spec[1])
        lib().orc_get(self.h, spec[0], _p(out))
        return out

    def trace(self, o, d, tmin=0.0, bvh=True, want_t2=False):
        o = np.ascontiguousarray(o, np.float32)
        d = np.ascontiguousarray(d, np.float32)
        n = len(o)
        prim = np.zeros(n, np.int32)
        t, u, v = np.zeros(n, np.float32), np.zeros(n, np.float32), np.zeros(n, np.float32)
        t2 = np.zeros(n, np.float32) if want_t2 else None
        lib().orc_trace(self.h, _p(o), _p(d), n, tmin, int(bvh), _p(prim), _p(t), _p(u), _p(v),
                        _p(t2) if want_t2 else None)
        return (prim, t, u, v, t2) if want_t2 else (prim, t, u, v)

    def occluded(self, o, d, tmax, skip=None, bvh=True):
        o = np.ascontiguousarray(o, np.float32)
        d = np.ascontiguousarray(d, np.float32)
        tmax = np.ascontiguousarray(tmax, np.float32)
        n = len(o)
        sk = None if skip is None else np.ascontiguousarray(skip, np.int32)
        out = np.zeros(n, np.uint8)
        lib().orc_occluded(self.h, _p(o), _p(d), _p(tmax), _p(sk) if sk is not None else None, n,
                           int(bvh), _p(out))
        return out.astype(bool)

    def render_samples(self, cam, lights, ids, bvh=True, want_t2=True):
        c, L = make_camera(cam), make_lights(lights)
        ids = np.ascontiguousarray(ids, np.int64)
        n = len(ids)
        prim, t = np.zeros(n, np.int32), np.zeros(n, np.float32)
        t2 = np.zeros(n, np.float32)
        vis, rgb = np.zeros(n, np.uint16), np.zeros((n, 3), np.float32)
        lib().orc_render_samples(self.h, C.byref(c), C.cast(L, C.c_void_p), len(lights), _p(ids), n,
                                 int(bvh), _p(prim), _p(t), _p(t2) if want_t2 else None, _p(vis), _p(rgb))
        return dict(prim=prim, t=t, t2=t2, vis=vis, rgb=rgb)

    def render_rows(self, cam, lights, row0=0, row1=None, bvh=True, out=None):
        c, L = make_camera(cam), make_lights(lights)
        if out is None:
            out = np.zeros((cam.height, cam.width, 4), np.float32)
        row1 = cam.height if row1 is None else row1
        lib().orc_render_rows(self.h, C.byref(c), C.cast(L, C.c_void_p), len(lights), row0, row1,
                              int(bvh), _p(out))
        return out

    def render_image(self, cam, lights, bvh=True, threads: int = 1):
        """Full image; rows split over `threads` Python threads (ctypes drops the GIL)."""
        out = np.zeros((cam.height, cam.width, 4), np.float32)
        if threads <= 1:
            return self.render_rows(cam, lights, 0, cam.height, bvh, out)
        from concurrent.futures import ThreadPoolExecutor
        bands = np.linspace(0, cam.height, threads * 4 + 1).astype(int)
        with ThreadPoolExecutor(threads) as ex:
            list(ex.map(lambda i: self.render_rows(cam, lights, bands[i], bands[i + 1], bvh, out),
                        range(len(bands) - 1)))
        return out

    def render_all_samples(self, cam, lights, bvh=True, threads: int = 1, want_t2=True):
        n = cam.width * cam.height * cam.spp
        ids = np.arange(n, dtype=np.int64)
        if threads <= 1:
            return self.render_samples(cam, lights, ids, bvh, want_t2)
        from concurrent.futures import ThreadPoolExecutor
        chunks = np.array_split(ids, threads * 4)
        with ThreadPoolExecutor(threads) as ex:
            parts = list(ex.map(lambda c: self.render_samples(cam, lights, c, bvh, want_t2), chunks))
        return {k: np.concatenate([p[k] for p in parts]) for k in parts[0]}

    def shadow_eps(self) -> float:
        return float(lib().orc_shadow_eps(self.h))

    # -- FP64 twin (gradient checks) ------------------------------------------
    def shade_f64(self, cam, lights, samples, params, inten):
        c, L = make_camera(cam), make_lights(lights)
        params = np.ascontiguousarray(params, np.float64).reshape(-1)
        inten = np.ascontiguousarray(inten, np.float64)
        img = np.zeros((cam.height, cam.width, 3), np.float64)
        lib().orc_shade_f64(self.h, C.byref(c), C.cast(L, C.c_void_p), len(lights),
                            _p(samples["prim"]), _p(samples["t"]), _p(samples["vis"]),
                            _p(params), _p(inten), _p(img))
        return img

    def shade_f64_fresh(self, cam, lights, samples, params, inten):
        """shade_f64 with the hit frame recomputed in FP64 from the camera ray
        and the world triangle (flat normals, single-level scenes)."""
        c, L = make_camera(cam), make_lights(lights)
        params = np.ascontiguousarray(params, np.float64).reshape(-1)
        inten = np.ascontiguousarray(inten, np.float64)
        img = np.zeros((cam.height, cam.width, 3), np.float64)
        r = lib().orc_shade_f64_fresh(self.h, C.byref(c), C.cast(L, C.c_void_p), len(lights),
                                      _p(samples["prim"]), _p(samples["vis"]), _p(params), _p(inten), _p(img))
        if r != 0:
            raise ValueError("FP64 frame from scratch: flat normals and single-level scenes only")
        return img

    def grad_f64(self, cam, lights, samples, params, inten, dimg):
        c, L = make_camera(cam), make_lights(lights)
        params = np.ascontiguousarray(params, np.float64).reshape(-1)
        inten = np.ascontiguousarray(inten, np.float64)
        dimg = np.ascontiguousarray(dimg, np.float64)
        dp = np.zeros(params.shape, np.float64)
        di = np.zeros(len(lights), np.float64)
        lib().orc_grad_f64(self.h, C.byref(c), C.cast(L, C.c_void_p), len(lights),
                           _p(samples["prim"]), _p(samples["t"]), _p(samples["vis"]),
                           _p(params), _p(inten), _p(dimg), _p(dp), _p(di))
        return dp.reshape(-1, 5), di


def camera_ray(cam, x, y, k):
    c = make_camera(cam)
    o, d = np.zeros(3, np.float32), np.zeros(3, np.float32)
    lib().orc_camera_ray(C.byref(c), x, y, k, _p(o), _p(d))
    return o, d


def brdf_f32(n, v, l, mat):
    m = Material()
    m.albedo[:] = [float(a) for a in mat["albedo"]]
    m.roughness, m.metallic = float(mat["roughness"]), float(mat["metallic"])
    f = np.zeros(3, np.float32)
    n, v, l = (np.ascontiguousarray(x, np.float32) for x in (n, v, l))
    lib().orc_brdf_f32(_p(n), _p(v), _p(l), C.byref(m), _p(f))
    return f


def brdf_f64(n, v, l, albedo, rough, metal, kmode=0):
    n, v, l, a = (np.ascontiguousarray(x, np.float64) for x in (n, v, l, albedo))
    fd, fs = np.zeros(3), np.zeros(3)
    lib().orc_brdf_f64(_p(n), _p(v), _p(l), _p(a), rough, metal, kmode, _p(fd), _p(fs))
    return fd, fs


def ggx_d(nh, alpha):
    return lib().orc_ggx_d(nh, alpha)


def schlick_f(vh, f0):
    return lib().orc_schlick_f(vh, f0)


def smith_g(nl, nv, rough, kmode=0):
    return lib().orc_smith_g(nl, nv, rough, kmode)


def params_of(mats: np.ndarray) -> np.ndarray:
    """[nmat, 5] float64: albedo rgb, roughness, metallic."""
    p = np.zeros((len(mats), 5))
    for i, m in enumerate(mats):
        p[i, :3] = m["albedo"]
        p[i, 3] = m["roughness"]
        p[i, 4] = m["metallic"]
    return p


def display(hdr: np.ndarray, exposure: float = 1.0, fxaa: bool = True, want_gamma: bool = False):
    """Display stage of an [H, W, 4] linear HDR image (rgb + coverage):
    Reinhard tone map, sRGB encode, optional FXAA, 8-bit quantisation.
    Returns [H, W, 4] uint8 (and the pre-FXAA gamma-space float image)."""
    h = np.ascontiguousarray(hdr, np.float32)
    H, W = h.shape[:2]
    out = np.zeros((H, W, 4), np.uint8)
    g = np.zeros((H, W, 4), np.float32) if want_gamma else None
    lib().orc_display(_p(h), W, H, float(exposure), int(bool(fxaa)), _p(g) if want_gamma else None, _p(out))
    return (out, g) if want_gamma else out


def srgb_encode(r: float) -> float:
    return float(lib().orc_srgb_encode(float(r)))


def root12_pow5(r: float) -> float:
    return float(lib().orc_root12_pow5(float(r)))


def srgb_decode(c: float) -> float:
    return float(lib().orc_srgb_decode(float(c)))
