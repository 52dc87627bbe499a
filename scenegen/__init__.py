"""Seeded synthetic inputs shaped like the paper's scenes (§V: scenes duplicated
to grow the triangle count; §IV-C: per-body world matrices every frame).

This module only *generates inputs*: meshes (icospheres + a heightfield
terrain), per-mesh materials, cameras, lights and rigid-body world matrices.
It holds none of the renderer's arithmetic (no transforms of vertices, no
LBVH, no intersection, no shading), so both the CUDA path and the CPU oracle
may consume what it produces.

Every random number comes from one xoshiro256** stream seeded through
splitmix64 (both published generators, written out here), with
u = (x >> 40) * 2**-24, so results never depend on a library's
distributions.  Seed = 2410 * 100 + workload index.

Workloads (every sphere is the 5,120-triangle icosphere, 20 * 4^4, and the
terrain a 256x256-cell heightfield; with the stated sphere counts the
headline frame then has the paper's ">7M" triangles):
  tiny41k    8 icospheres (5,120 tris) + 2-tri ground quad = 40,962 tris, 256x256, 1 spp, 1 light
  mid1m      200 icospheres + 256x256-cell terrain = 1,155,072 tris, 1280x720, 4 spp, 3 lights
  frame7m    1,400 icospheres + 256x256 terrain = 7,299,072 tris, 1920x1080, 4 spp, 2 lights,
             64 rigid bodies moved every frame
  batch16    16 scenes, T log-uniform in [20k, 2M], 64 cameras, 1 spp
  grad500k   72 icospheres + 256x256 terrain = 499,712 tris, 32 materials, 512x512, 1 spp
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MASK64 = (1 << 64) - 1
SEED_BASE = 2410 * 100


# ----------------------------------------------------------------------------
# Random numbers: splitmix64 (seeding) + xoshiro256** (stream)
# ----------------------------------------------------------------------------
def _rotl(x: int, k: int) -> int:
    return ((x << k) | (x >> (64 - k))) & MASK64


class Rng:
    """xoshiro256** (Blackman & Vigna 2018) seeded with splitmix64."""

    def __init__(self, seed: int):
        z = seed & MASK64
        s = []
        for _ in range(4):
            z = (z + 0x9E3779B97F4A7C15) & MASK64
            x = z
            x = ((x ^ (x >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
            x = ((x ^ (x >> 27)) * 0x94D049BB133111EB) & MASK64
            s.append(x ^ (x >> 31))
        self.s = s

    def next_u64(self) -> int:
        s0, s1, s2, s3 = self.s
        result = (_rotl((s1 * 5) & MASK64, 7) * 9) & MASK64
        t = (s1 << 17) & MASK64
        s2 ^= s0
        s3 ^= s1
        s1 ^= s2
        s0 ^= s3
        s2 ^= t
        s3 = _rotl(s3, 45)
        self.s = [s0, s1, s2, s3]
        return result

    def u(self) -> float:
        """Uniform in [0, 1) with 24 random bits (exact in float32)."""
        return (self.next_u64() >> 40) * (1.0 / 16777216.0)

    def uniform(self, a: float, b: float) -> float:
        return a + (b - a) * self.u()

    def unit_vector(self) -> np.ndarray:
        z = 2.0 * self.u() - 1.0
        phi = 2.0 * math.pi * self.u()
        r = math.sqrt(max(0.0, 1.0 - z * z))
        return np.array([r * math.cos(phi), r * math.sin(phi), z])


# ----------------------------------------------------------------------------
# Geometry generators
# ----------------------------------------------------------------------------
_ICO_CACHE: dict[int, tuple[np.ndarray, np.ndarray]] = {}


def icosphere(level: int) -> tuple[np.ndarray, np.ndarray]:
    """Unit icosphere: golden-ratio icosahedron, `level` 1-to-4 subdivisions.

    Face (a,b,c) -> (a,ab,ca), (b,bc,ab), (c,ca,bc), (ab,bc,ca); midpoints are
    normalised and shared through an edge map.  Level 4 = 5,120 triangles and
    2,562 vertices.  Returns float64 vertices [V,3] and int64 faces [F,3].
    """
    if level in _ICO_CACHE:
        return _ICO_CACHE[level]
    p = (1.0 + math.sqrt(5.0)) / 2.0
    verts = [(-1, p, 0), (1, p, 0), (-1, -p, 0), (1, -p, 0),
             (0, -1, p), (0, 1, p), (0, -1, -p), (0, 1, -p),
             (p, 0, -1), (p, 0, 1), (-p, 0, -1), (-p, 0, 1)]
    verts = [np.array(v, dtype=np.float64) / math.sqrt(1 + p * p) for v in verts]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
             (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
             (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
             (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(level):
        edge: dict[tuple[int, int], int] = {}

        def mid(a: int, b: int) -> int:
            key = (a, b) if a < b else (b, a)
            if key not in edge:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                edge[key] = len(verts) - 1
            return edge[key]

        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    out = (np.array(verts, dtype=np.float64), np.array(faces, dtype=np.int64))
    _ICO_CACHE[level] = out
    return out


def value_noise_heights(rng: Rng, x: np.ndarray, z: np.ndarray, octaves: int = 4,
                        amplitude: float = 2.0) -> np.ndarray:
    """h = amplitude * sum_o 0.5^o vn_o(2^o * 0.25 * (x, z)) / sum_o 0.5^o.

    vn_o is bilinear value noise with smoothstep weights over seeded lattice
    values in [0, 1), drawn in (octave, i, j) order over the lattice cells
    that cover |coordinate| <= 12.
    """
    h = np.zeros_like(x, dtype=np.float64)
    wsum = 0.0
    for o in range(octaves):
        f = (2.0 ** o) * 0.25
        L = int(math.ceil(12.0 * f)) + 1
        n = 2 * L + 2
        lat = np.array([[rng.u() for _ in range(n)] for _ in range(n)], dtype=np.float64)
        px, pz = x * f + L, z * f + L
        ix, iz = np.floor(px).astype(np.int64), np.floor(pz).astype(np.int64)
        fx, fz = px - ix, pz - iz
        sx, sz = fx * fx * (3 - 2 * fx), fz * fz * (3 - 2 * fz)
        a = lat[ix, iz] * (1 - sx) + lat[ix + 1, iz] * sx
        b = lat[ix, iz + 1] * (1 - sx) + lat[ix + 1, iz + 1] * sx
        w = 0.5 ** o
        h += w * (a * (1 - sz) + b * sz)
        wsum += w
    return amplitude * h / wsum


def terrain(rng: Rng, cells: int, half: float = 12.0, y_offset: float = -2.0):
    """Heightfield over [-half, half]^2 (x, z) with y = h(x, z) + y_offset.

    Each cell (i, j) is split along its (i,j)-(i+1,j+1) diagonal into two
    triangles.  Returns float64 verts [(cells+1)^2, 3], int64 faces [2 cells^2, 3].
    """
    g = cells
    t = np.linspace(-half, half, g + 1)
    X, Z = np.meshgrid(t, t, indexing="ij")
    Y = value_noise_heights(rng, X, Z) + y_offset
    verts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    i, j = np.meshgrid(np.arange(g), np.arange(g), indexing="ij")
    a = (i * (g + 1) + j).ravel()
    b = ((i + 1) * (g + 1) + j).ravel()
    c = ((i + 1) * (g + 1) + j + 1).ravel()
    d = (i * (g + 1) + j + 1).ravel()
    faces = np.concatenate([np.stack([a, b, c], 1), np.stack([a, c, d], 1)], axis=0)
    # interleave the two triangles of each cell so neighbours stay adjacent
    faces = faces.reshape(2, g * g, 3).transpose(1, 0, 2).reshape(-1, 3)
    return verts, faces


# ----------------------------------------------------------------------------
# Scene container (the arrays fire_scene_create takes)
# ----------------------------------------------------------------------------
MATERIAL_DTYPE = np.dtype([("albedo", np.float32, 3), ("roughness", np.float32),
                           ("metallic", np.float32)])


@dataclass
class Scene:
    verts: np.ndarray      # float32 [V, 4] rest pose (w = 1)
    idx: np.ndarray        # uint32  [T, 3]
    tri_mat: np.ndarray    # uint32  [T]
    vert_body: np.ndarray  # uint16  [V]
    mats: np.ndarray       # MATERIAL_DTYPE [nmat]
    nbody: int
    mesh_tri_start: list = field(default_factory=list)

    @property
    def nt(self) -> int:
        return int(self.idx.shape[0])

    @property
    def nv(self) -> int:
        return int(self.verts.shape[0])

    def identity_xforms(self) -> np.ndarray:
        x = np.zeros((self.nbody, 12), dtype=np.float32)
        x[:, 0] = x[:, 5] = x[:, 10] = 1.0
        return x


def vertex_normals(scene: Scene) -> np.ndarray:
    """Per-vertex rest-pose normals, as a glTF-like asset carries them: the
    area-weighted mean of the incident faces' normals (sum of the faces'
    unnormalised cross products in FP64, normalised).  float32 [V, 4], w = 0;
    a vertex with no face (or a zero sum) gets (0, 1, 0)."""
    v = scene.verts[:, :3].astype(np.float64)
    f = scene.idx.astype(np.int64)
    fn = np.cross(v[f[:, 1]] - v[f[:, 0]], v[f[:, 2]] - v[f[:, 0]])
    acc = np.zeros_like(v)
    for k in range(3):
        np.add.at(acc, f[:, k], fn)
    ln = np.linalg.norm(acc, axis=1)
    out = np.zeros((len(v), 4), dtype=np.float32)
    ok = ln > 0
    out[ok, :3] = acc[ok] / ln[ok, None]
    out[~ok, 1] = 1.0
    return out


def random_materials(rng: Rng, nmat: int) -> np.ndarray:
    m = np.zeros(nmat, dtype=MATERIAL_DTYPE)
    for i in range(nmat):
        m[i]["albedo"] = [rng.uniform(0.05, 0.95) for _ in range(3)]
        m[i]["roughness"] = rng.uniform(0.05, 1.0)
        m[i]["metallic"] = 1.0 if rng.u() < 0.3 else 0.0
    return m


def assemble(meshes, nmat: int, mats: np.ndarray, mesh_body=None, nbody: int = 1) -> Scene:
    """Concatenate (verts, faces) meshes; mesh m gets material m mod nmat."""
    vs, fs, tm, vb, starts = [], [], [], [], []
    voff = toff = 0
    for m, (v, f) in enumerate(meshes):
        vs.append(v)
        fs.append(f + voff)
        tm.append(np.full(len(f), m % nmat, dtype=np.uint32))
        body = 0 if mesh_body is None else mesh_body[m]
        vb.append(np.full(len(v), body, dtype=np.uint16))
        starts.append(toff)
        voff += len(v)
        toff += len(f)
    V = np.concatenate(vs).astype(np.float32)
    verts = np.ones((len(V), 4), dtype=np.float32)
    verts[:, :3] = V
    return Scene(verts=verts, idx=np.concatenate(fs).astype(np.uint32),
                 tri_mat=np.concatenate(tm), vert_body=np.concatenate(vb),
                 mats=mats, nbody=nbody, mesh_tri_start=starts)


def _kd_labels(cs, nbody: int):
    """Order sphere ids so that the runs of ids forming body b (ids i with
    floor(nbody*i/n) == b) are spatially compact: recursive median splits of
    the (x, z) centres along the longer extent, with the split counts taken
    from the body boundaries."""
    n = len(cs)
    start = [(b * n + nbody - 1) // nbody for b in range(nbody + 1)]  # first id of body b

    def rec(ids, b0, b1):
        if b1 - b0 <= 1 or len(ids) <= 1:  # (fewer spheres than bodies: empty bodies)
            return list(ids)
        mid = (b0 + b1) // 2
        cnt = start[mid] - start[b0]
        pts = np.array([cs[i] for i in ids])
        ax = 0 if np.ptp(pts[:, 0]) >= np.ptp(pts[:, 2]) else 2
        srt = sorted(ids, key=lambda i: (cs[i][ax], i))
        return rec(srt[:cnt], b0, mid) + rec(srt[cnt:], mid, b1)

    return rec(list(range(n)), 0, nbody)


def _spheres(rng: Rng, n: int, cxz: float, cy: tuple, radius: tuple, level: int = 4,
             nbody: int = 0):
    """n icospheres with centres uniform in [-cxz,cxz]^2 (x,z) x cy (y) and
    radii uniform in `radius`.  nbody > 0: number the spheres so that each
    run of consecutive ids that forms one rigid body (sphere i -> body
    floor(nbody*i/n)) is a spatially compact cluster (the draws themselves
    are unchanged)."""
    uv, uf = icosphere(level)
    cs, rs = [], []
    for _ in range(n):
        cs.append(np.array([rng.uniform(-cxz, cxz), rng.uniform(*cy), rng.uniform(-cxz, cxz)]))
        rs.append(rng.uniform(*radius))
    order = _kd_labels(cs, nbody) if nbody else range(n)
    return [(uv * rs[i] + cs[i], uf) for i in order]


# ----------------------------------------------------------------------------
# Cameras and lights (plain records; field order = fire_camera / fire_light)
# ----------------------------------------------------------------------------
@dataclass
class Camera:
    pos: tuple
    target: tuple
    up: tuple
    vfov_deg: float
    width: int
    height: int
    spp: int


@dataclass
class Light:
    type: int          # 0 = point (v = position), 1 = directional (v = direction to the light)
    v: tuple
    intensity: float


LIGHTS_MAIN = [Light(0, (0.0, 10.0, 0.0), 100.0),
               Light(0, (-8.0, 12.0, -6.0), 150.0),
               Light(1, tuple((np.array([0.3, 1.0, 0.5]) / np.linalg.norm([0.3, 1.0, 0.5])).tolist()), 2.0)]


def orbit_camera(rng: Rng, width: int, height: int, spp: int, radius: float = 12.0) -> Camera:
    d = rng.unit_vector()
    pos = tuple((d * radius).tolist())
    up = (0.0, 1.0, 0.0) if abs(d[1]) < 0.999 else (0.0, 0.0, 1.0)
    return Camera(pos, (0.0, 0.0, 0.0), up, 60.0, width, height, spp)


# ----------------------------------------------------------------------------
# Workloads
# ----------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    scene: Scene
    camera: Camera
    lights: list
    frames: int = 1
    motion: "RigidMotion | None" = None


def scene_icospheres_terrain(rng: Rng, nspheres: int, cells: int, nmat: int,
                             nbody_spheres: int = 0) -> Scene:
    mats = random_materials(rng, nmat)
    tv, tf = terrain(rng, cells)
    sph = _spheres(rng, nspheres, 10.0, (0.5, 3.0), (0.3, 1.0), nbody=nbody_spheres)
    meshes = [(tv, tf)] + sph
    if nbody_spheres:
        mesh_body = [nbody_spheres] + [(nbody_spheres * i) // nspheres for i in range(nspheres)]
        return assemble(meshes, nmat, mats, mesh_body, nbody_spheres + 1)
    return assemble(meshes, nmat, mats)


def workload_tiny41k(width: int = 256, height: int = 256) -> Workload:
    rng = Rng(SEED_BASE + 0)
    mats = random_materials(rng, 9)
    ground = (np.array([[-15.0, 0, -15.0], [15.0, 0, -15.0], [15.0, 0, 15.0], [-15.0, 0, 15.0]]),
              np.array([[0, 1, 2], [0, 2, 3]]))
    meshes = [ground] + _spheres(rng, 8, 5.0, (0.5, 3.0), (0.3, 1.0))
    scene = assemble(meshes, 9, mats)
    cam = Camera((0.0, 4.0, 12.0), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 60.0, width, height, 1)
    return Workload("tiny41k", scene, cam, [LIGHTS_MAIN[0]])


def workload_mid1m(width: int = 1280, height: int = 720, spp: int = 4) -> Workload:
    rng = Rng(SEED_BASE + 1)
    scene = scene_icospheres_terrain(rng, 200, 256, 32)
    cam = Camera((0.0, 10.0, 22.0), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 60.0, width, height, spp)
    return Workload("mid1m", scene, cam, LIGHTS_MAIN[:3])


def workload_frame7m(width: int = 1920, height: int = 1080, spp: int = 4,
                     nspheres: int = 1400, cells: int = 256) -> Workload:
    rng = Rng(SEED_BASE + 2)
    scene = scene_icospheres_terrain(rng, nspheres, cells, 32, nbody_spheres=64)
    cam = Camera((0.0, 10.0, 22.0), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 60.0, width, height, spp)
    return Workload("frame7m", scene, cam, LIGHTS_MAIN[:2], frames=100,
                    motion=RigidMotion(scene, Rng(SEED_BASE + 2 + 1000)))


def workload_grad500k(width: int = 512, height: int = 512) -> Workload:
    rng = Rng(SEED_BASE + 4)
    scene = scene_icospheres_terrain(rng, 72, 256, 32)
    cam = Camera((0.0, 10.0, 22.0), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 60.0, width, height, 1)
    return Workload("grad500k", scene, cam, LIGHTS_MAIN[:2])


def batch16(nscenes: int = 16, ncams_per: int = 4, tmin: float = 20e3, tmax: float = 2e6,
            seed_offset: int = 3):
    """Scenes of uneven size (target T log-uniform in [tmin, tmax], rounded to
    whole spheres inside that range), four orbit cameras each, 1-3 lights
    each, 1 spp."""
    rng = Rng(SEED_BASE + seed_offset)
    res = [(128, 128), (256, 256), (320, 240), (640, 480)]
    scenes, cams, cam_scene, lights = [], [], [], []
    for s in range(nscenes):
        T = math.exp(rng.uniform(math.log(tmin), math.log(tmax)))
        g = 64 if T < 200e3 else (128 if T < 800e3 else 256)
        n = max(1, int(round((T - 2 * g * g) / 5120.0)))
        # whole spheres: keep the total inside [tmin, tmax]
        while 2 * g * g + 5120 * n < tmin:
            n += 1
        while 2 * g * g + 5120 * n > tmax and n > 1:
            n -= 1
        scenes.append(scene_icospheres_terrain(rng, n, g, 32))
        nl = 1 + int(rng.u() * 3)
        lights.append(LIGHTS_MAIN[:nl])
        for _ in range(ncams_per):
            w, h = res[int(rng.u() * 4)]
            cams.append(orbit_camera(rng, w, h, 1))
            cam_scene.append(s)
    return scenes, cams, cam_scene, lights


# ----------------------------------------------------------------------------
# Rigid-body motion (the simulator's per-step world matrices, §IV-C)
# ----------------------------------------------------------------------------
class RigidMotion:
    """Bodies are runs of consecutive spheres, numbered by a k-d partition of
    their centres (compact clusters, like the rigid parts of a simulated
    scene).  Per frame, body b < nbody-1 gets a random delta: axis uniform on S^2,
    angle uniform in [0, 2 deg], translation of uniform direction and
    magnitude uniform in [0, 0.05].  The delta rotates about the body's
    current pivot (its rest-pose AABB centre mapped by the current matrix).
    Matrices are composed in float64 and handed out as absolute row-major
    3x4 float32 world matrices.  The last body (terrain) stays identity."""

    def __init__(self, scene: Scene, rng: Rng, max_deg: float = 2.0, max_t: float = 0.05):
        self.rng, self.max_deg, self.max_t = rng, max_deg, max_t
        self.nbody = scene.nbody
        self.W = np.tile(np.eye(4), (self.nbody, 1, 1))
        P = scene.verts[:, :3].astype(np.float64)
        self.pivot = np.zeros((self.nbody, 3))
        for b in range(self.nbody):
            sel = P[scene.vert_body == b]
            if len(sel):
                self.pivot[b] = 0.5 * (sel.min(0) + sel.max(0))
        self.frame = 0

    def xforms(self) -> np.ndarray:
        return self.W[:, :3, :4].reshape(self.nbody, 12).astype(np.float32)

    def step(self) -> np.ndarray:
        """Advance one frame and return the new absolute matrices."""
        for b in range(self.nbody - 1):
            axis = self.rng.unit_vector()
            ang = math.radians(self.max_deg) * self.rng.u()
            tdir = self.rng.unit_vector()
            tmag = self.max_t * self.rng.u()
            K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
            R = np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * (K @ K)
            p = self.W[b, :3, :3] @ self.pivot[b] + self.W[b, :3, 3]
            D = np.eye(4)
            D[:3, :3] = R
            D[:3, 3] = p - R @ p + tdir * tmag
            self.W[b] = D @ self.W[b]
        self.frame += 1
        return self.xforms()


WORKLOADS = {"tiny41k": workload_tiny41k, "mid1m": workload_mid1m,
             "frame7m": workload_frame7m, "grad500k": workload_grad500k}


def perturbed_params(mats: np.ndarray, intensities, seed: int = SEED_BASE + 40):
    """Start point of the shading optimisation: albedo +-0.2, roughness +-0.3,
    intensity x U[0.5, 2], clamped (albedo [0.01, 0.99], roughness [0.05, 1])."""
    rng = Rng(seed)
    m = mats.copy()
    for i in range(len(m)):
        m[i]["albedo"] = np.clip([a + rng.uniform(-0.2, 0.2) for a in m[i]["albedo"]], 0.01, 0.99)
        m[i]["roughness"] = np.clip(m[i]["roughness"] + rng.uniform(-0.3, 0.3), 0.05, 1.0)
    inten = np.array([I * rng.uniform(0.5, 2.0) for I in intensities], dtype=np.float32)
    return m, inten


def random_rays(rng: Rng, n: int, lo, hi, target_lo=None, target_hi=None):
    """Rays with origins uniform in box [lo, hi] aimed at points uniform in
    [target_lo, target_hi] (default: the same box).  float32 [n,3] each; the
    direction is left unnormalised."""
    lo, hi = np.asarray(lo, np.float64), np.asarray(hi, np.float64)
    tlo = lo if target_lo is None else np.asarray(target_lo, np.float64)
    thi = hi if target_hi is None else np.asarray(target_hi, np.float64)
    o = np.array([[rng.uniform(lo[a], hi[a]) for a in range(3)] for _ in range(n)])
    t = np.array([[rng.uniform(tlo[a], thi[a]) for a in range(3)] for _ in range(n)])
    return o.astype(np.float32), (t - o).astype(np.float32)


def random_soup(rng: Rng, n: int, extent: float = 1.0, size: float = 0.3):
    """n random triangles in [-extent, extent]^3 with edges up to `size`."""
    c = np.array([[rng.uniform(-extent, extent) for _ in range(3)] for _ in range(n)])
    v = np.zeros((3 * n, 4), dtype=np.float32)
    for i in range(n):
        for k in range(3):
            v[3 * i + k, :3] = c[i] + np.array([rng.uniform(-size, size) for _ in range(3)])
            v[3 * i + k, 3] = 1.0
    idx = np.arange(3 * n, dtype=np.uint32).reshape(n, 3)
    return v, idx
