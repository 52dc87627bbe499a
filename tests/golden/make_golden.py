"""Writes the closed-form fixtures of this folder (pure Python arithmetic;
no renderer code is called).

morton_body_prefix.txt -- see body_key_rows().

brdf_normal_incidence.txt -- §IV-B-1 Cook-Torrance variant at l = v = n:
  h = n, so n.h = v.h = n.l = n.v = 1; D = 1/(pi a^2) with a = r^2 (GGX);
  F = F0 (Schlick at normal incidence); G = 1 (Schlick-GGX at x = 1);
  f_s = F0 / (4 pi a^2); f_d = (1 - F0)(1 - m) albedo / pi (Lambert),
  F0 = 0.04 (1 - m) + albedo m (metallic-roughness workflow).
"""
import math
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def brdf_rows():
    rows = []
    for alb in (0.05, 0.5, 0.95):
        for r in (0.05, 0.3, 1.0):
            for m in (0.0, 1.0):
                f0 = 0.04 * (1 - m) + alb * m
                a = r * r
                fs = f0 / (4 * math.pi * a * a)
                fd = (1 - f0) * (1 - m) * alb / math.pi
                rows.append((alb, r, m, fd, fs))
    return rows


def body_key_rows():
    """Morton keys with a body field, of centroids at lo / mid / hi of the
    bounds [0, 8]^3 (§IV-C rigid bodies; the LBVH key layout of the
    acceleration structure): B = bits of (nbody - 1), m = min(21, (63 - B)
    // 3) bits per axis; per axis q = 0 at lo, 2^(m-1) at mid ((c - lo) 2^m /
    (hi - lo) is exactly 2^(m-1)), 2^m - 1 at hi (clamped); x -> bit 3k+2,
    y -> 3k+1, z -> 3k; the top c = 4 bits of each q (coarse) above the body,
    the rest (fine) below it:
      key = coarse << (B + 3(m-4)) | body << 3(m-4) | fine."""
    rows = []
    c = 4
    for nbody in (2, 3, 65, 1025, 65536):
        B = (nbody - 1).bit_length()
        m = min(21, (63 - B) // 3)
        q = {"lo": 0, "mid": 1 << (m - 1), "hi": (1 << m) - 1}
        for body, pt in ((0, ("hi", "hi", "hi")), (nbody - 1, ("lo", "lo", "lo")), (nbody - 1, ("hi", "mid", "lo")),
                         (nbody // 2, ("mid", "mid", "mid")), (1, ("lo", "hi", "mid"))):
            coarse = fine = 0
            for k in range(m):
                bits = [(q[pt[a]] >> k) & 1 for a in range(3)]  # x, y, z
                for a in range(3):
                    if k >= m - c:
                        coarse |= bits[a] << (3 * (k - (m - c)) + 2 - a)
                    else:
                        fine |= bits[a] << (3 * k + 2 - a)
            f = 3 * (m - c)
            rows.append((nbody, body, pt, (coarse << (B + f)) | (body << f) | fine))
    return rows


def main():
    with open(os.path.join(HERE, "brdf_normal_incidence.txt"), "w") as f:
        f.write("# l = v = n: f_d = (1-F0)(1-m) albedo/pi, f_s = F0/(4 pi r^4), F0 = 0.04(1-m) + albedo m\n")
        f.write("# (Cook-Torrance variant of §IV-B-1; written by make_golden.py)\n")
        f.write("# albedo roughness metallic f_d f_s\n")
        for row in brdf_rows():
            f.write(" ".join(repr(float(x)) for x in row) + "\n")
    with open(os.path.join(HERE, "morton_body_prefix.txt"), "w") as f:
        f.write("# Morton keys with a body field: B = bits of (nbody-1), m = min(21, (63-B)//3) bits per axis,\n")
        f.write("# key = coarse << (B + 3(m-4)) | body << 3(m-4) | fine, coarse/fine = the top 4 / the other\n")
        f.write("# bits of each axis, interleaved (x -> 3k+2, y -> 3k+1, z -> 3k); centroid bounds [0,8]^3,\n")
        f.write("# q = 0 at lo, 2^(m-1) at mid, 2^m - 1 at hi.  (Written by make_golden.py.)\n")
        f.write("# nbody body x y z key\n")
        for nbody, body, pt, key in body_key_rows():
            f.write(f"{nbody} {body} {pt[0]} {pt[1]} {pt[2]} {key:#018x}\n")


if __name__ == "__main__":
    main()
