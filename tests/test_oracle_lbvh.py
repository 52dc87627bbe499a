"""Pins for the oracle's pose update and LBVH (transform, Morton codes, sort,
radix-tree topology, refit) against closed forms, hand-derived codes and the
defining invariants of a Karras radix tree -- none of them re-type the
oracle's own formulas."""
import os

import numpy as np
import pytest

import oracle
import scenegen as sg

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _scene_from_tris(tris: np.ndarray, nbody: int = 1, vbody=None) -> sg.Scene:
    tris = np.asarray(tris, np.float32).reshape(-1, 3, 3)
    T = len(tris)
    verts = np.ones((3 * T, 4), np.float32)
    verts[:, :3] = tris.reshape(-1, 3)
    mats = sg.random_materials(sg.Rng(7), 1)
    vb = np.zeros(3 * T, np.uint16) if vbody is None else np.asarray(vbody, np.uint16)
    return sg.Scene(verts=verts, idx=np.arange(3 * T, dtype=np.uint32).reshape(T, 3),
                    tri_mat=np.zeros(T, np.uint32), vert_body=vb, mats=mats, nbody=nbody)


def _point_tri(c, d=0.25):
    c = np.asarray(c, np.float64)
    return np.stack([c - d, c, c + d])


def test_morton_hand_codes():
    """Centroids at lo / mid / hi of the bounds give the hand-derived codes
    of tests/golden/morton_corners.txt (§IV-B-3 acceleration structure;
    LBVH codes are the Morton order of triangle centroids)."""
    pos = {"lo": 0.0, "mid": 4.0, "hi": 8.0}
    rows = []
    for line in open(os.path.join(GOLDEN, "morton_corners.txt")):
        if line.strip() and not line.startswith("#"):
            *p, code = line.split()
            rows.append(([pos[a] for a in p], int(code, 16)))
    tris = [_point_tri([0, 0, 0]), _point_tri([8, 8, 8])] + [_point_tri(p) for p, _ in rows]
    S = oracle.OracleScene(_scene_from_tris(np.array(tris)))
    S.update(np.eye(3, 4, dtype=np.float32).reshape(1, 12), rebuild=True)
    codes = S.get("morton")
    assert list(S.get("centroid_bounds")) == [0, 0, 0, 8, 8, 8]
    for i, (_, want) in enumerate(rows):
        assert int(codes[2 + i]) == want, (i, hex(int(codes[2 + i])), hex(want))


def test_morton_body_prefix_hand_codes():
    """Scenes of several rigid bodies: keys carry the body id above the Morton
    bits (tests/golden/morton_body_prefix.txt, derived from the key layout in
    plain integer arithmetic); the body is that of the triangle's first
    vertex."""
    pos = {"lo": 0.0, "mid": 4.0, "hi": 8.0}
    rows = {}
    for line in open(os.path.join(GOLDEN, "morton_body_prefix.txt")):
        if line.strip() and not line.startswith("#"):
            nb, body, x, y, z, key = line.split()
            rows.setdefault(int(nb), []).append((int(body), [pos[x], pos[y], pos[z]], int(key, 16)))
    assert sorted(rows) == [2, 3, 65, 1025, 65536]
    for nbody, cases in rows.items():
        tris = [_point_tri([0, 0, 0]), _point_tri([8, 8, 8])] + [_point_tri(p) for _, p, _ in cases]
        vb = np.repeat([0, 0] + [b for b, _, _ in cases], 3).astype(np.uint16)
        S = oracle.OracleScene(_scene_from_tris(np.array(tris), nbody=nbody, vbody=vb))
        S.update(np.tile(np.eye(3, 4, dtype=np.float32).reshape(1, 12), (nbody, 1)), rebuild=True)
        codes = S.get("morton")
        assert list(S.get("centroid_bounds")) == [0, 0, 0, 8, 8, 8]
        for i, (_, _, want) in enumerate(cases):
            assert int(codes[2 + i]) == want, (nbody, i, hex(int(codes[2 + i])), hex(want))
    # a triangle whose vertices belong to different bodies takes its first
    # vertex's (nbody 3: B = 2, m = 20, the body field at bits 48..49)
    tris = [_point_tri([0, 0, 0]), _point_tri([8, 8, 8]), _point_tri([8, 8, 8])]
    vb = np.array([0, 0, 0, 1, 1, 1, 2, 0, 1], np.uint16)
    S = oracle.OracleScene(_scene_from_tris(np.array(tris), nbody=3, vbody=vb))
    S.update(np.tile(np.eye(3, 4, dtype=np.float32).reshape(1, 12), (3, 1)), rebuild=True)
    assert [(int(c) >> 48) & 3 for c in S.get("morton")] == [0, 1, 2]


def _split_key(key: int, B: int, m: int, c: int = 4):
    """(coarse cell, body, plain m-bit Morton code) of a key with a body field."""
    f = 3 * (m - c)
    fine = key & ((1 << f) - 1)
    body = (key >> f) & ((1 << B) - 1)
    coarse = key >> (B + f)
    return coarse, body, (coarse << f) | fine


def test_each_body_is_one_subtree_per_coarse_cell():
    """With a body field below the coarse cell bits, the triangles of one
    body inside one coarse cell (1/16 of the bounds per axis) are
    consecutive in the sorted order and are exactly the leaves of one node
    of the radix tree (checked on a soup of interleaved bodies whose boxes
    overlap); cells come in Morton order, bodies in id order inside a cell."""
    rng = sg.Rng(321)
    nbody, n = 7, 700
    tris = []
    for _ in range(n):
        c = np.array([rng.uniform(-3, 3) for _ in range(3)])
        tris.append(np.stack([c, c + [0.2, 0.0, 0.05], c + [0.0, 0.15, 0.1]]))
    body_of_tri = np.array([int(rng.u() * nbody) for _ in range(n)])
    vb = np.repeat(body_of_tri, 3).astype(np.uint16)
    S = oracle.OracleScene(_scene_from_tris(np.array(tris), nbody=nbody, vbody=vb))
    S.update(np.tile(np.eye(3, 4, dtype=np.float32).reshape(1, 12), (nbody, 1)), rebuild=True)
    order, children, keys = S.get("order"), S.get("children"), S.get("morton")
    B, m = 3, 20
    parts = [_split_key(int(keys[t]), B, m) for t in order]
    assert [p[1] for p in parts] == body_of_tri[order].tolist()
    cell_body = [(p[0], p[1]) for p in parts]
    assert cell_body == sorted(cell_body)  # cells in order, bodies in id order inside a cell
    T = n
    leaves = {}

    def rec(code):
        if code >= T - 1:
            leaves[code] = {code - (T - 1)}
            return leaves[code]
        a, b = int(children[code][0]), int(children[code][1])
        leaves[code] = rec(a) | rec(b)
        return leaves[code]

    import sys
    sys.setrecursionlimit(10000)
    rec(0)
    covers = set(frozenset(v) for v in leaves.values())
    groups = {}
    for p, cb in enumerate(cell_body):
        groups.setdefault(cb, []).append(p)
    assert len(groups) > nbody  # bodies do span several cells
    for cb, ps in groups.items():
        assert ps == list(range(ps[0], ps[-1] + 1)) and frozenset(ps) in covers, cb


def _deinterleave(code: int, m: int = 21):
    q = [0, 0, 0]
    for k in range(m):
        for a in range(3):
            q[a] |= ((code >> (3 * k + 2 - a)) & 1) << k
    return q


def test_morton_decodes_to_quantised_centroid(tiny41k):
    """Every code de-interleaves to per-axis integers q with
    q <= x < q + 1 for x = 2^21 (c-lo)/(hi-lo) in exact arithmetic, up to the
    roundings of the FP32 quantiser (a few 2^-24 relative, plus the FP32
    centroid), and bit 63 is never set."""
    sc = tiny41k.scene
    S = oracle.OracleScene(sc)
    S.update(sc.identity_xforms(), rebuild=True)
    codes = S.get("morton")
    world = S.get("world").astype(np.float64)
    tri = world[sc.idx.astype(np.int64)]
    c = 0.5 * (tri.min(1) + tri.max(1))
    lo, hi = c.min(0), c.max(0)
    rng = np.random.default_rng(0)
    for i in rng.choice(sc.nt, 400, replace=False):
        code = int(codes[i])
        assert code >> 63 == 0
        q = _deinterleave(code)
        for a in range(3):
            x = (c[i, a] - lo[a]) / (hi[a] - lo[a]) * 2 ** 21
            assert q[a] <= 2 ** 21 - 1
            tol = 5 * 2.0 ** -24 * x + 0.1
            assert q[a] - tol <= x and (x < q[a] + 1 + tol or q[a] == 2 ** 21 - 1), (i, a, x, q[a])


def test_body_keys_decode_to_body_and_quantised_centroid():
    """Moving workload (65 bodies: B = 7 body bits, m = 18 bits per axis):
    each key's body field is the body of the triangle's first vertex and its
    coarse and fine bits together de-interleave to q <= 2^m (c - lo)/(hi - lo)
    < q + 1, up to the FP32 quantiser's roundings."""
    w = sg.workload_frame7m(nspheres=40, cells=16)
    sc = w.scene
    assert sc.nbody == 65
    B, m = 7, 18
    S = oracle.OracleScene(sc)
    xf = w.motion.xforms()
    S.update(xf, rebuild=True)
    codes = S.get("morton")
    world = S.get("world").astype(np.float64)
    tri = world[sc.idx.astype(np.int64)]
    c = 0.5 * (tri.min(1) + tri.max(1))
    lo, hi = c.min(0), c.max(0)
    body = sc.vert_body[sc.idx[:, 0]].astype(np.int64)
    rng = np.random.default_rng(1)
    for i in rng.choice(sc.nt, 500, replace=False):
        key = int(codes[i])
        _, b, code = _split_key(key, B, m)
        assert b == body[i] and key >> 63 == 0
        q = _deinterleave(code, m)
        for a in range(3):
            x = (c[i, a] - lo[a]) / (hi[a] - lo[a]) * 2 ** m
            tol = 5 * 2.0 ** -24 * x + 0.1
            assert q[a] - tol <= x and (x < q[a] + 1 + tol or q[a] == 2 ** m - 1), (i, a, x, q[a])


def test_sort_is_stable_permutation(tiny41k):
    sc = tiny41k.scene
    S = oracle.OracleScene(sc)
    S.update(sc.identity_xforms(), rebuild=True)
    codes, order = S.get("morton"), S.get("order")
    assert sorted(order.tolist()) == list(range(sc.nt))
    k = codes[order]
    assert np.all(k[1:] >= k[:-1])
    eq = k[1:] == k[:-1]
    assert np.all(order[1:][eq] > order[:-1][eq])  # equal keys keep original order


def _delta(keys, i, j):
    if j < 0 or j >= len(keys):
        return -1
    a, b = int(keys[i]), int(keys[j])
    if a != b:
        return 64 - (a ^ b).bit_length()
    return 64 + 32 - (int(i) ^ int(j)).bit_length()


def check_radix_tree(keys, children, parent):
    """The defining properties of the Karras radix tree over sorted keys:
    node i covers a contiguous range [f, l] with i in {f, l}; its children are
    numbered s and s+1 (leaf T-1+p for a one-key range); the split s is where
    the highest differing bit of the range changes (delta(s, s+1) =
    delta(f, l) < delta within each half); every node but the root has
    exactly one parent."""
    T = len(keys)
    if T < 2:
        return
    rng_of = {}

    def rec(code):
        if code >= T - 1:
            p = code - (T - 1)
            rng_of[code] = (p, p)
            return p, p
        a, b = int(children[code][0]), int(children[code][1])
        fa, la = rec(a)
        fb, lb = rec(b)
        assert la + 1 == fb, "children ranges must be adjacent"
        rng_of[code] = (fa, lb)
        return fa, lb

    import sys
    sys.setrecursionlimit(10000)
    f, l = rec(0)
    assert (f, l) == (0, T - 1)
    seen = np.zeros(2 * T - 1, int)
    for i in range(T - 1):
        f, l = rng_of[i]
        assert i in (f, l)
        a, b = int(children[i][0]), int(children[i][1])
        s = rng_of[a][1]
        assert (a == s) if a < T - 1 else (a - (T - 1) == s and s == f)
        assert (b == s + 1) if b < T - 1 else (b - (T - 1) == s + 1 and s + 1 == l)
        d = _delta(keys, f, l)
        assert _delta(keys, s, s + 1) == d
        if s > f:
            assert _delta(keys, f, s) > d
        if s + 1 < l:
            assert _delta(keys, s + 1, l) > d
        seen[a] += 1
        seen[b] += 1
        assert parent[a] == i and parent[b] == i
    assert seen[0] == 0 and np.all(seen[1:] == 1)
    assert parent[0] == -1


@pytest.mark.parametrize("n,dups", [(2, False), (3, False), (17, False), (200, False), (300, True)])
def test_topology_invariants_random(n, dups):
    rng = sg.Rng(100 + n)
    cs = []
    for _ in range(n):
        if dups:
            # few distinct centroids -> many equal Morton codes (index-augmented split)
            cs.append([float(int(rng.u() * 3)) for _ in range(3)])
        else:
            cs.append([rng.uniform(-4, 4) for _ in range(3)])
    S = oracle.OracleScene(_scene_from_tris(np.array([_point_tri(c, 0.125) for c in cs])))
    S.update(np.eye(3, 4, dtype=np.float32).reshape(1, 12), rebuild=True)
    keys = S.get("morton")[S.get("order")]
    if dups:
        assert len(np.unique(keys)) < n // 4
    check_radix_tree(keys, S.get("children"), S.get("parent"))


def test_topology_invariants_scene(tiny41k):
    sc = tiny41k.scene
    S = oracle.OracleScene(sc)
    S.update(sc.identity_xforms(), rebuild=True)
    check_radix_tree(S.get("morton")[S.get("order")], S.get("children"), S.get("parent"))


def test_single_and_two_triangles():
    S = oracle.OracleScene(_scene_from_tris(np.array([_point_tri([1, 2, 3])])))
    S.update(np.eye(3, 4, dtype=np.float32).reshape(1, 12), rebuild=True)
    assert S.get("children").shape == (0, 2)
    assert list(S.get("parent")) == [-1]
    box = S.get("boxes")[0]
    assert list(box) == [0.75, 1.75, 2.75, 1.25, 2.25, 3.25]
    S = oracle.OracleScene(_scene_from_tris(np.array([_point_tri([1, 2, 3]), _point_tri([0, 0, 0])])))
    S.update(np.eye(3, 4, dtype=np.float32).reshape(1, 12), rebuild=True)
    assert S.get("order").tolist() == [1, 0]
    assert S.get("children").tolist() == [[1, 2]]


def test_refit_boxes_are_exact_subtree_bounds(tiny41k):
    """Every node's box equals min/max over the vertices of the triangles it
    covers (exact: min/max never round), before and after a rigid motion."""
    sc = tiny41k.scene
    S = oracle.OracleScene(sc)
    S.update(sc.identity_xforms(), rebuild=True)
    order = S.get("order")
    T = sc.nt
    for frame in range(2):
        world = S.get("world")
        tri = world[sc.idx.astype(np.int64)][order]  # sorted position order
        tmin, tmax = tri.min(1), tri.max(1)
        boxes, children = S.get("boxes"), S.get("children")
        # ranges by recursion over the child array
        stack, rng_of = [0], {}
        lo_of = {}

        def leaf_range(code):
            while code < T - 1:
                code = children[code][0]
            return code - (T - 1)

        def leaf_range_r(code):
            while code < T - 1:
                code = children[code][1]
            return code - (T - 1)

        rs = np.random.default_rng(frame)
        for code in list(rs.choice(T - 1, 300, replace=False)) + list(T - 1 + rs.choice(T, 100)):
            f, l = leaf_range(code), leaf_range_r(code)
            want = np.concatenate([tmin[f:l + 1].min(0), tmax[f:l + 1].max(0)])
            assert np.array_equal(boxes[code], want), code
        # move: a refit keeps the topology
        x = sc.identity_xforms()
        x[0, 3] = 0.5
        x[0, 0], x[0, 2], x[0, 8], x[0, 10] = 0.8, 0.6, -0.6, 0.8
        S.update(x, rebuild=False)
        assert np.array_equal(S.get("order"), order)


def test_transform_identity_and_rigid():
    """Identity matrices reproduce the rest pose exactly; a rotation +
    translation matches the float64 product to within the rounding of a
    three-term FP32 multiply-add chain."""
    rng = sg.Rng(5)
    n = 200
    v = np.array([[rng.uniform(-10, 10) for _ in range(3)] for _ in range(n)])
    tris = v.reshape(-1, 1, 3).repeat(3, 1)[: n // 2 * 0 + n]
    vb = np.array([i % 3 for i in range(3 * n)], np.uint16)
    S = oracle.OracleScene(_scene_from_tris(tris, nbody=3, vbody=vb))
    I = np.tile(np.eye(3, 4, dtype=np.float32).reshape(1, 12), (3, 1))
    S.update(I, rebuild=True)
    rest = np.repeat(v.astype(np.float32), 3, axis=0)
    assert np.array_equal(S.get("world"), rest)
    X = np.zeros((3, 12), np.float32)
    for b in range(3):
        ax = np.array([rng.uniform(-1, 1) for _ in range(3)])
        ax /= np.linalg.norm(ax)
        ang = rng.uniform(0, 3)
        K = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
        R = np.eye(3) + np.sin(ang) * K + (1 - np.cos(ang)) * K @ K
        M = np.concatenate([R, np.array([[rng.uniform(-5, 5)] for _ in range(3)])], 1)
        X[b] = M.astype(np.float32).reshape(12)
    S.update(X, rebuild=False)
    w = S.get("world").astype(np.float64)
    M64 = X.astype(np.float64).reshape(3, 3, 4)
    r64 = rest.astype(np.float64)
    exact = np.einsum("vij,vj->vi", M64[vb][:, :, :3], r64) + M64[vb][:, :, 3]
    scale = np.einsum("vij,vj->vi", np.abs(M64[vb][:, :, :3]), np.abs(r64)) + np.abs(M64[vb][:, :, 3])
    assert np.all(np.abs(w - exact) <= 4 * 2.0 ** -24 * scale)
