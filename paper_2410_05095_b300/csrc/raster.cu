// Primary visibility by triangle-parallel rasterisation with the ray test as
// the coverage test -- the paper's main pass is a rasteriser (§IV-A-1, MSAA
// §IV-B-2); here it computes exactly the nearest ray hit of every sample:
//   k_rclear  sample keys := "no hit", sample ray directions (the camera's
//             own cam_dir values), raster counters := 0, frame constants
//   k_rsetup  one thread per triangle: conservative screen footprint (pixel
//             box, and edge lines for well-conditioned triangles); boxes of
//             up to kSmallSamples samples are tested by the thread itself,
//             larger ones are cut into pieces of <= kPieceSamples samples
//             and queued
//   k_rgraze  the triangles k_rsetup deferred (nearly edge-on or slivers:
//             footprint from their box), one thread each, same steps
//   k_rbig    one warp per queued piece, 32 samples at a time
// Every candidate sample runs the same Moller-Trumbore test (same ray, same
// operands) as the traversal; an accepted hit updates the sample's 64-bit
// key (t bits << 32 | original index) with atomicMin, which is the
// traversal's (t, original index) minimum.  The footprint is conservative,
// so the key of each sample equals the traversal's result; the G-buffer and
// shadow queue are then written by the traversal's own kernel tail
// (k_primary in key mode).
// Cases the footprint cannot bound -- geometry within a tiny ball around the
// camera, non-finite projections, a full piece queue -- set a flag, and the
// frame's primary pass falls back to traversal on the device.  Parts of a
// triangle with Z < zn outside that ball lie outside the view frustum (the
// ball's radius is zn * 1.01 * sqrt(1 + tan_x^2 + tan_y^2)), so clipping
// them away loses no sample.
#include <algorithm>

#include "trace_device.cuh"

namespace fire {

namespace {

constexpr int kSmallSamples = 256;    // boxes up to this many samples: tested by their thread
constexpr int kPieceSamples = 4096;   // queued pieces hold at most this many samples
constexpr int kPieceW = 64;           // piece width in pixels

__device__ __forceinline__ void raster_fallback(uint32_t* ctrl, uint32_t why) { atomicOr(ctrl + kCtrlRasterFlag, why); }

// Conservative screen footprint of one triangle, in pixel coordinates
// (sample k of pixel x sits at x + 0.5 + ox_k).
struct Footprint {
  float lx, hx, ly, hy;  // box, margin included
  float m;               // margin (pixels)
  bool edges;            // edge lines valid (e_j(p) >= -m for every candidate)
  float ea[3], eb[3], ec[3];
};

// 0: footprint filled; -1: nothing of the triangle can be hit; -2: needs the
// box bound and defer_box was set; > 0: fallback reason bits.
__device__ __forceinline__ int footprint(const CamParams& c, float4 A, float4 B, float4 C, float zn, float rn,
                                         float slack, bool defer_box, Footprint& F) {
  const float3 o = f3(c.ox, c.oy, c.oz);
  const float3 q[3] = {sub3(xyz(A), o), add3(sub3(xyz(A), o), xyz(B)), add3(sub3(xyz(A), o), xyz(C))};
  const float3 qlo = f3(fmin3f(q[0].x, q[1].x, q[2].x), fmin3f(q[0].y, q[1].y, q[2].y), fmin3f(q[0].z, q[1].z, q[2].z));
  const float3 qhi = f3(fmax3f(q[0].x, q[1].x, q[2].x), fmax3f(q[0].y, q[1].y, q[2].y), fmax3f(q[0].z, q[1].z, q[2].z));
  // geometry inside the ball |q| <= rn may be hit at Z < zn: no footprint for it
  {
    const float bx = fmaxf(fmaxf(qlo.x, -qhi.x), 0.0f), by = fmaxf(fmaxf(qlo.y, -qhi.y), 0.0f),
                bz = fmaxf(fmaxf(qlo.z, -qhi.z), 0.0f);
    if (bx * bx + by * by + bz * bz <= rn * rn) return 1;
  }
  const float3 cr = f3(c.rx, c.ry, c.rz), cu = f3(c.ux, c.uy, c.uz), cf = f3(c.fx, c.fy, c.fz);
  float sx0 = inf_f(), sx1 = -inf_f(), sy0 = inf_f(), sy1 = -inf_f(), zmin = inf_f();
  bool bad = false;
  auto add = [&](float x, float y, float z) {
    const float iz = __fdividef(1.0f, z);
    float sx = x * iz, sy = y * iz;
    bad |= !(fabsf(sx) < 1e30f && fabsf(sy) < 1e30f);
    sx0 = fminf(sx0, sx);
    sx1 = fmaxf(sx1, sx);
    sy0 = fminf(sy0, sy);
    sy1 = fmaxf(sy1, sy);
    zmin = fminf(zmin, z);
  };
  // conditioning of the triangle test for rays from the camera:
  // |det| / (|d| |e1| |e2|) ~ |N.q0| / (|q0| |e1| |e2|)
  const float3 N = cross3(xyz(B), xyz(C));
  const float cond = fabsf(dot3(N, q[0])) * rsqrtf(fmaxf(dot3(q[0], q[0]), 1e-30f)) *
                     rsqrtf(fmaxf(dot3(xyz(B), xyz(B)), 1e-30f)) * rsqrtf(fmaxf(dot3(xyz(C), xyz(C)), 1e-30f));
  const bool good = cond >= 1e-2f;
  if (!good && defer_box) return -2;
  float X[3] = {0, 0, 0}, Y[3] = {0, 0, 0}, Z[3] = {0, 0, 0};
  if (good) {
    // well conditioned: the test accepts only next to the triangle itself;
    // clip it against Z >= zn and project s = (X/Z, Y/Z)
#pragma unroll
    for (int v = 0; v < 3; ++v) {
      X[v] = dot3(q[v], cr);
      Y[v] = dot3(q[v], cu);
      Z[v] = dot3(q[v], cf);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int b = a == 2 ? 0 : a + 1;
      const bool ina = Z[a] >= zn, inb = Z[b] >= zn;
      if (ina) add(X[a], Y[a], Z[a]);
      if (ina != inb) {
        float f = __fdividef(zn - Z[a], Z[b] - Z[a]);
        add(X[a] + f * (X[b] - X[a]), Y[a] + f * (Y[b] - Y[a]), zn);
      }
    }
  } else {
    // nearly edge-on or sliver: bound by the triangle's box, which the
    // traversal's leaf test requires the ray to cross; the box is clipped
    // against Z >= zn (its corners in front + its edges' crossings)
    float BX[8], BY[8], BZ[8];
#pragma unroll
    for (int v = 0; v < 8; ++v) {
      const float3 p = f3((v & 1) ? qhi.x : qlo.x, (v & 2) ? qhi.y : qlo.y, (v & 4) ? qhi.z : qlo.z);
      BX[v] = dot3(p, cr);
      BY[v] = dot3(p, cu);
      BZ[v] = dot3(p, cf);
      if (BZ[v] >= zn) add(BX[v], BY[v], BZ[v]);
    }
#pragma unroll
    for (int v = 0; v < 8; ++v)
#pragma unroll
      for (int bit = 1; bit < 8; bit <<= 1) {
        const int w = v | bit;
        if (w == v) continue;
        if ((BZ[v] >= zn) != (BZ[w] >= zn)) {
          float f = __fdividef(zn - BZ[v], BZ[w] - BZ[v]);
          add(BX[v] + f * (BX[w] - BX[v]), BY[v] + f * (BY[w] - BY[v]), zn);
        }
      }
  }
  if (bad) return 2;
  if (!(zmin < inf_f())) return -1;  // wholly behind the clip plane
  // margin (pixels): rounding of the projection and of the triangle test,
  // which grow as Z shrinks relative to |q|, plus the traversal's box slack
  // pixel coordinates: px = sx * kx + hw, py = hh - sy * ky
  const float hw = 0.5f * (float)c.W, hh = 0.5f * (float)c.H;
  const float kx = __fdividef(hw, c.sxs), ky = __fdividef(hh, c.sys);
  const float qm = fmaxf(fabsf(qlo.x), fabsf(qhi.x)) + fmaxf(fabsf(qlo.y), fabsf(qhi.y)) +
                   fmaxf(fabsf(qlo.z), fabsf(qhi.z));
  const float smax = fmaxf(fmaxf(fabsf(sx0), fabsf(sx1)), fmaxf(fabsf(sy0), fabsf(sy1)));
  F.m = 0.01f + __fdividef(1e-5f * qm * (1.0f + smax) + slack, zmin) * fmaxf(kx, ky);
  F.lx = fmaf(sx0, kx, hw) - F.m;
  F.hx = fmaf(sx1, kx, hw) + F.m;
  F.ly = fmaf(-sy1, ky, hh) - F.m;
  F.hy = fmaf(-sy0, ky, hh) + F.m;
  // edge lines of the projected triangle (all three vertices in front)
  F.edges = good && Z[0] >= zn && Z[1] >= zn && Z[2] >= zn;
  if (F.edges) {
    float px[3], py[3];
#pragma unroll
    for (int v = 0; v < 3; ++v) {
      const float iz = __fdividef(1.0f, Z[v]);
      px[v] = fmaf(X[v] * iz, kx, hw);
      py[v] = fmaf(-(Y[v] * iz), ky, hh);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int b = a == 2 ? 0 : a + 1, e = a == 0 ? 2 : a - 1;
      const float na = -(py[b] - py[a]), nb = px[b] - px[a];
      const float len2 = na * na + nb * nb;
      const float side = na * (px[e] - px[a]) + nb * (py[e] - py[a]);
      if (!(len2 > 0.0f) || !(fabsf(side) > 1e-3f * len2)) {
        F.edges = false;  // degenerate projection: box only
        break;
      }
      const float s = (side > 0.0f ? 1.0f : -1.0f) * rsqrtf(len2);
      F.ea[a] = na * s;
      F.eb[a] = nb * s;
      F.ec[a] = -(F.ea[a] * px[a] + F.eb[a] * py[a]);
    }
  }
  return 0;
}

__device__ __forceinline__ bool inside(const Footprint& F, float sxp, float syp) {
  if (sxp < F.lx || sxp > F.hx || syp < F.ly || syp > F.hy) return false;
  if (F.edges) {
#pragma unroll
    for (int a = 0; a < 3; ++a)
      if (fmaf(F.ea[a], sxp, fmaf(F.eb[a], syp, F.ec[a])) < -F.m) return false;
  }
  return true;
}

__device__ __forceinline__ void raster_sample(const RasterArgs& r, float3 o, float4 A, float4 B, float4 C,
                                              int64_t sid) {
  float t;
  const float4 d4 = __ldg(r.dirs + sid);
  if (mt_t(o, f3(d4.x, d4.y, d4.z), A, B, C, t) && t > 0.0f && t < inf_f()) {
    const unsigned long long key =
        ((unsigned long long)__float_as_uint(t) << 32) | (unsigned long long)(uint32_t)__float_as_int(A.w);
    if (key < __ldcg(r.keys + sid)) atomicMin(r.keys + sid, key);
  }
}

__device__ __forceinline__ void frame_constants(const RasterArgs& r, float& zn, float& rn, float& slack) {
  zn = __uint_as_float(r.ctrl[kCtrlRasterParams]);
  rn = __uint_as_float(r.ctrl[kCtrlRasterParams + 1]);
  slack = __uint_as_float(r.ctrl[kCtrlRasterParams + 2]);
}

// Also zeroes the raster counters and stores the frame's constants:
//   zn    = 2^-14 x scene-box diagonal (clip plane distance)
//   rn    = zn x 1.01 x sqrt(1 + tan_x^2 + tan_y^2) (fallback ball radius)
//   slack = 2^-17 x (largest |coordinate| of the scene box + largest |o|),
//           above the traversal's box-test slack of 2^-19 (M + |o_a|)
__global__ void __launch_bounds__(256) k_rclear(RasterArgs r) {
  const CamParams& c = r.cam;
  if (blockIdx.x == 0 && threadIdx.x < 4) r.ctrl[kCtrlRasterPieces + threadIdx.x] = 0u;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    float zn = 1e-20f, span = 0.0f;
    if (r.nt > 0) {
      float3 lo, hi;
      root_box(r.nodes4, lo, hi);
      const float3 ext = sub3(hi, lo);
      zn = fmaxf(sqrtf(dot3(ext, ext)) * 0x1p-14f, 1e-20f);
      span = scene_span(r.nodes4, r.nt);
    }
    const float rn = zn * 1.01f * sqrtf(1.0f + c.sxs * c.sxs + c.sys * c.sys);
    const float om = fmax3f(fabsf(c.ox), fabsf(c.oy), fabsf(c.oz));
    r.ctrl[kCtrlRasterParams] = __float_as_uint(zn);
    r.ctrl[kCtrlRasterParams + 1] = __float_as_uint(rn);
    r.ctrl[kCtrlRasterParams + 2] = __float_as_uint((span + om) * 0x1p-17f);
  }
  const int64_t first = (int64_t)r.row_begin * c.W * c.spp;
  const int64_t n = (int64_t)(r.row_end - r.row_begin) * c.W * c.spp;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t sid = first + i;
    const int k = (int)(sid % c.spp);
    const int64_t p = sid / c.spp;
    const float3 d = cam_dir(c, (int)(p % c.W), (int)(p / c.W), k);
    r.dirs[sid] = make_float4(d.x, d.y, d.z, 0.0f);
    r.keys[sid] = ~0ull;
  }
}

// One triangle: footprint, then its samples (small boxes) or queued pieces.
// defer: triangles that need the box bound (nearly edge-on, slivers) go to
// a list for k_rgraze instead, so that their longer setup does not hold up
// the other 31 lanes of the warp.
__device__ __forceinline__ void raster_triangle(const RasterArgs& r, int64_t i, bool defer) {
  const CamParams& c = r.cam;
  float zn, rn, slack;
  frame_constants(r, zn, rn, slack);
  const float4 A = __ldg(r.tris + 3 * i), B = __ldg(r.tris + 3 * i + 1), C = __ldg(r.tris + 3 * i + 2);
  Footprint F;
  const int st = footprint(c, A, B, C, zn, rn, slack, defer, F);
  if (st == -2) {
    const uint32_t slot = atomicAdd(r.ctrl + kCtrlRasterGraze, 1u);
    if (slot < r.cap_graze) r.graze[slot] = (int32_t)i;
    else raster_fallback(r.ctrl, 4u);
    return;
  }
  if (st != 0) {
    if (st > 0) raster_fallback(r.ctrl, (uint32_t)st);
    return;
  }
  // pixel box: candidates of pixel x have x + 0.5 + ox_k in [lx, hx], |ox_k| <= omax
  const float omax = c.spp == 4 ? 0.375f : 0.0f;
  const float xa = fmaxf(ceilf(F.lx - 0.5f - omax), 0.0f);
  const float xb = fminf(floorf(F.hx - 0.5f + omax), (float)(c.W - 1));
  const float ya = fmaxf(ceilf(F.ly - 0.5f - omax), (float)r.row_begin);
  const float yb = fminf(floorf(F.hy - 0.5f + omax), (float)(r.row_end - 1));
  if (!(xa <= xb && ya <= yb)) return;
  const int x0 = (int)xa, x1 = (int)xb, y0 = (int)ya, y1 = (int)yb;
  const int64_t n = (int64_t)(x1 - x0 + 1) * (y1 - y0 + 1) * c.spp;
  if (n <= kSmallSamples) {
    const float3 o = f3(c.ox, c.oy, c.oz);
    // per sample row (pixel row y, sample k): the x interval where the box
    // and the three edge half-planes (margin m) hold
    float ia[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) ia[a] = F.edges && F.ea[a] != 0.0f ? __fdividef(1.0f, F.ea[a]) : 0.0f;
    for (int y = y0; y <= y1; ++y)
      for (int k = 0; k < c.spp; ++k) {
        float ox, oy;
        spp_offset(c.spp, k, ox, oy);
        const float sy = (float)y + (0.5f + oy);
        if (sy < F.ly || sy > F.hy) continue;
        float lo = F.lx, hi = F.hx;
        if (F.edges) {
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            // ea * sx >= rhs
            const float rhs = -F.m - fmaf(F.eb[a], sy, F.ec[a]);
            if (F.ea[a] > 0.0f) lo = fmaxf(lo, rhs * ia[a] - 1e-3f);
            else if (F.ea[a] < 0.0f) hi = fminf(hi, rhs * ia[a] + 1e-3f);
            else if (rhs > 1e-3f) hi = -inf_f();
          }
        }
        const int xa2 = max(x0, (int)ceilf(fmaxf(lo - (0.5f + ox), -1.0f)));
        const int xb2 = min(x1, (int)floorf(fminf(hi - (0.5f + ox), (float)c.W)));
        for (int x = xa2; x <= xb2; ++x) raster_sample(r, o, A, B, C, ((int64_t)y * c.W + x) * c.spp + k);
      }
    return;
  }
  // queue pieces of at most kPieceW x ph pixels (<= kPieceSamples samples)
  const int ph = max(1, kPieceSamples / (kPieceW * c.spp));
  for (int py = y0; py <= y1; py += ph)
    for (int px = x0; px <= x1; px += kPieceW) {
      uint32_t slot = atomicAdd(r.ctrl + kCtrlRasterPieces, 1u);
      if (slot >= r.cap_pieces) {
        raster_fallback(r.ctrl, 4u);
        return;
      }
      const int qx1 = min(px + kPieceW - 1, x1), qy1 = min(py + ph - 1, y1);
      r.pieces[slot] = make_int4((int)i, px | (qx1 << 16), py | (qy1 << 16), 0);
    }
}

__global__ void __launch_bounds__(256) k_rsetup(RasterArgs r) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < r.nt) raster_triangle(r, i, true);
}

// The deferred triangles of k_rsetup, one thread each.
__global__ void __launch_bounds__(128) k_rgraze(RasterArgs r) {
  const uint32_t n = min(r.ctrl[kCtrlRasterGraze], (uint32_t)r.cap_graze);
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
    raster_triangle(r, r.graze[j], false);
}

__global__ void __launch_bounds__(128) k_rbig(RasterArgs r) {
  const int lane = threadIdx.x & 31;
  const uint32_t npieces = min(r.ctrl[kCtrlRasterPieces], (uint32_t)r.cap_pieces);
  const CamParams& c = r.cam;
  const int spp = c.spp;
  const float3 o = f3(c.ox, c.oy, c.oz);
  float zn, rn, slack;
  frame_constants(r, zn, rn, slack);
  while (true) {
    uint32_t e = 0;
    if (lane == 0) e = atomicAdd(r.ctrl + kCtrlRasterCursor, 1u);
    e = __shfl_sync(kFull, e, 0);
    if (e >= npieces) return;
    const int4 P = r.pieces[e];
    const int64_t ti = P.x;
    const float4 A = __ldg(r.tris + 3 * ti), B = __ldg(r.tris + 3 * ti + 1), C = __ldg(r.tris + 3 * ti + 2);
    Footprint F;
    if (footprint(c, A, B, C, zn, rn, slack, false, F) != 0) continue;  // queued only with a footprint
    const int x0 = P.y & 0xffff, x1 = (P.y >> 16) & 0xffff, y0 = P.z & 0xffff, y1 = (P.z >> 16) & 0xffff;
    const int w = x1 - x0 + 1;
    const int n = w * (y1 - y0 + 1) * spp;
    for (int j = lane; j < n; j += 32) {
      const int k = spp == 4 ? (j & 3) : 0;
      const int p = spp == 4 ? (j >> 2) : j;
      const int py = p / w;
      const int x = x0 + (p - py * w), y = y0 + py;
      float ox, oy;
      spp_offset(spp, k, ox, oy);
      if (!inside(F, (float)x + (0.5f + ox), (float)y + (0.5f + oy))) continue;
      raster_sample(r, o, A, B, C, ((int64_t)y * c.W + x) * spp + k);
    }
  }
}

}  // namespace

int raster_primary(fire_scene_s* s, const RasterArgs& r, cudaStream_t st) {
  const int64_t n = (int64_t)(r.row_end - r.row_begin) * r.cam.W * r.cam.spp;
  const int sms = sm_count();
  int gclear = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * 8, (n + 255) / 256));
  k_rclear<<<gclear, 256, 0, st>>>(r);
  if (r.nt > 0) {
    k_rsetup<<<(unsigned)((r.nt + 255) / 256), 256, 0, st>>>(r);
    k_rgraze<<<sms * 4, 128, 0, st>>>(r);
    static int occ = 0;
    if (occ == 0) {
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_rbig, 128, 0) != cudaSuccess || occ < 1) occ = 1;
    }
    k_rbig<<<sms * occ, 128, 0, st>>>(r);
  }
  (void)s;
  return cuda_check(cudaGetLastError(), "raster kernels");
}

}  // namespace fire
