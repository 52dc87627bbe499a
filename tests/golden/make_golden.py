"""Writes the closed-form fixtures of this folder (pure Python arithmetic;
no renderer code is called).

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


def main():
    with open(os.path.join(HERE, "brdf_normal_incidence.txt"), "w") as f:
        f.write("# l = v = n: f_d = (1-F0)(1-m) albedo/pi, f_s = F0/(4 pi r^4), F0 = 0.04(1-m) + albedo m\n")
        f.write("# (Cook-Torrance variant of §IV-B-1; written by make_golden.py)\n")
        f.write("# albedo roughness metallic f_d f_s\n")
        for row in brdf_rows():
            f.write(" ".join(repr(float(x)) for x in row) + "\n")


if __name__ == "__main__":
    main()
