// Display output stage of the resolved linear HDR image: Reinhard tone
// mapping and gamma correction (§IV-A-1: colours above 1 are mapped into
// [0, 1), then the sRGB-to-linear conversion is inverted) and FXAA (§IV-B-2),
// then 8-bit quantisation.
//   k_tonemap  per pixel: c' = e c; r = c' / (1 + c'); sRGB encode
//              (IEC 61966-2-1: 12.92 r below 0.0031308, else
//              1.055 r^(1/2.4) - 0.055); bytes directly when FXAA is off,
//              else the gamma-space image into the caller's scratch
//   k_fxaa     per pixel, from the scratch image (clamp-to-edge fetches,
//              bilinear taps): Lottes' FXAA in its simple form -- edge
//              direction perpendicular to the luma gradient of the four
//              diagonal neighbours, scaled and clamped to 8 pixels, two
//              blends along it, the wider one unless its luma leaves the
//              neighbourhood's range
// r^(1/2.4) = (r^(1/12))^5 with r = m 2^-k, m in [1, 2): m^(1/12) by three
// Newton steps on t^12 = m from the chord start, times 2^(-k/12) (constants
// rounded from FP64 on the host).  FP32 throughout (-fmad=false, IEEE
// division), so the bytes are a pure function of the input.
#include <cmath>

#include "fire_internal.cuh"

namespace fire {
namespace {

struct DisplayConsts {
  float tab[12];  // 2^(-k/12)
  float chord;    // 2^(1/12) - 1
  float exposure;
  int W, H;
};

__device__ __forceinline__ float root12_pow5(const DisplayConsts& C, float r) {  // r^(5/12), r in [2^-9, 1)
  int e = 0;
  float m = frexpf(r, &e) * 2.0f;  // r = m 2^(e-1), m in [1, 2)
  const int k = 1 - e;
  float t = 1.0f + (m - 1.0f) * C.chord;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float t2 = t * t, t4 = t2 * t2, t8 = t4 * t4, t11 = (t8 * t2) * t;
    t = (11.0f * t + m / t11) / 12.0f;
  }
  const float u = t * C.tab[min(max(k, 0), 11)];
  const float u2 = u * u;
  return (u2 * u2) * u;
}

__device__ __forceinline__ float tonemap(const DisplayConsts& C, float c) {
  const float cc = C.exposure * c;
  const float r = cc / (1.0f + cc);
  if (r <= 0.0031308f) return 12.92f * r;
  return 1.055f * root12_pow5(C, r) - 0.055f;
}

__device__ __forceinline__ unsigned quant(float v) {
  return (unsigned)(int)floorf(fminf(fmaxf(v, 0.0f), 1.0f) * 255.0f + 0.5f);
}

__device__ __forceinline__ uint32_t pack(unsigned r, unsigned g, unsigned b, unsigned a) {
  return r | (g << 8) | (b << 16) | (a << 24);
}

__global__ void __launch_bounds__(256) k_tonemap(DisplayConsts C, const float4* __restrict__ hdr,
                                                 float4* __restrict__ gamma, uint32_t* __restrict__ out) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= (int64_t)C.W * C.H) return;
  const float4 h = hdr[p];
  const float4 g = make_float4(tonemap(C, h.x), tonemap(C, h.y), tonemap(C, h.z), h.w);
  if (gamma) gamma[p] = g;
  else out[p] = pack(quant(g.x), quant(g.y), quant(g.z), quant(g.w));
}

__device__ __forceinline__ float luma(float4 c) { return (0.299f * c.x + 0.587f * c.y) + 0.114f * c.z; }

__device__ __forceinline__ float4 fetch(const float4* __restrict__ g, int W, int H, int i, int j) {
  i = min(max(i, 0), W - 1);
  j = min(max(j, 0), H - 1);
  return __ldg(g + (int64_t)j * W + i);
}

__device__ __forceinline__ float4 tap(const float4* __restrict__ g, int W, int H, float px, float py) {
  const float u = px - 0.5f, v = py - 0.5f;
  const float fi = floorf(u), fj = floorf(v);
  const float fu = u - fi, fv = v - fj;
  const int i0 = (int)fi, j0 = (int)fj;
  const float4 c00 = fetch(g, W, H, i0, j0), c10 = fetch(g, W, H, i0 + 1, j0);
  const float4 c01 = fetch(g, W, H, i0, j0 + 1), c11 = fetch(g, W, H, i0 + 1, j0 + 1);
  float4 r;
  float top = c00.x + (c10.x - c00.x) * fu, bot = c01.x + (c11.x - c01.x) * fu;
  r.x = top + (bot - top) * fv;
  top = c00.y + (c10.y - c00.y) * fu;
  bot = c01.y + (c11.y - c01.y) * fu;
  r.y = top + (bot - top) * fv;
  top = c00.z + (c10.z - c00.z) * fu;
  bot = c01.z + (c11.z - c01.z) * fu;
  r.z = top + (bot - top) * fv;
  r.w = 0.0f;
  return r;
}

__global__ void __launch_bounds__(256) k_fxaa(DisplayConsts C, const float4* __restrict__ g,
                                              uint32_t* __restrict__ out) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= (int64_t)C.W * C.H) return;
  const int W = C.W, H = C.H;
  const int x = (int)(p % W), y = (int)(p / W);
  const float4 M = __ldg(g + p);
  const float lM = luma(M), lNW = luma(fetch(g, W, H, x - 1, y - 1)), lNE = luma(fetch(g, W, H, x + 1, y - 1)),
              lSW = luma(fetch(g, W, H, x - 1, y + 1)), lSE = luma(fetch(g, W, H, x + 1, y + 1));
  const float lmin = fminf(lM, fminf(fminf(lNW, lNE), fminf(lSW, lSE)));
  const float lmax = fmaxf(lM, fmaxf(fmaxf(lNW, lNE), fmaxf(lSW, lSE)));
  float dx = -((lSW + lSE) - (lNW + lNE));
  float dy = (lNE + lSE) - (lNW + lSW);
  const float reduce = fmaxf((((lNW + lNE) + lSW) + lSE) * (0.25f * 0.125f), 1.0f / 128.0f);
  const float rcp = 1.0f / (fminf(fabsf(dx), fabsf(dy)) + reduce);
  dx = fminf(fmaxf(dx * rcp, -8.0f), 8.0f);
  dy = fminf(fmaxf(dy * rcp, -8.0f), 8.0f);
  const float px = (float)x + 0.5f, py = (float)y + 0.5f;
  const float k1 = 1.0f / 3.0f - 0.5f, k2 = 2.0f / 3.0f - 0.5f;
  const float4 a1 = tap(g, W, H, px + dx * k1, py + dy * k1), a2 = tap(g, W, H, px + dx * k2, py + dy * k2);
  const float4 b1 = tap(g, W, H, px + dx * -0.5f, py + dy * -0.5f), b2 = tap(g, W, H, px + dx * 0.5f, py + dy * 0.5f);
  float4 A, B;
  A.x = 0.5f * (a1.x + a2.x);
  A.y = 0.5f * (a1.y + a2.y);
  A.z = 0.5f * (a1.z + a2.z);
  B.x = A.x * 0.5f + 0.25f * (b1.x + b2.x);
  B.y = A.y * 0.5f + 0.25f * (b1.y + b2.y);
  B.z = A.z * 0.5f + 0.25f * (b1.z + b2.z);
  const float lB = luma(B);
  const float4 c = (lB < lmin || lB > lmax) ? A : B;
  out[p] = pack(quant(c.x), quant(c.y), quant(c.z), quant(M.w));
}

// sRGB-encoded albedo to linear (IEC 61966-2-1 decode; §IV-A-1 converts
// sRGB colour inputs to linear before lighting): c / 12.92 at or below
// 0.04045, else ((c + 0.055) / 1.055)^2.4, on the three albedo entries of
// each 5-float material record.
__global__ void k_srgb_decode(float* mats, int nmat) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * nmat) return;
  float* p = mats + 5 * (i / 3) + i % 3;
  const float c = *p;
  *p = c <= 0.04045f ? c / 12.92f : powf((c + 0.055f) / 1.055f, 2.4f);
}

}  // namespace

int srgb_decode_materials(float* mats, int nmat, cudaStream_t st) {
  if (nmat <= 0) return FIRE_OK;
  k_srgb_decode<<<(3 * nmat + 255) / 256, 256, 0, st>>>(mats, nmat);
  return cuda_check(cudaGetLastError(), "sRGB decode");
}

int display_image(const float* hdr, int W, int H, float exposure, bool fxaa, float* scratch, uint8_t* out,
                  cudaStream_t st) {
  DisplayConsts C;
  for (int k = 0; k < 12; ++k) C.tab[k] = (float)std::pow(2.0, -k / 12.0);
  C.chord = (float)(std::pow(2.0, 1.0 / 12.0) - 1.0);
  C.exposure = exposure;
  C.W = W;
  C.H = H;
  const int64_t n = (int64_t)W * H;
  if (n == 0) return FIRE_OK;
  const unsigned grid = (unsigned)((n + 255) / 256);
  k_tonemap<<<grid, 256, 0, st>>>(C, reinterpret_cast<const float4*>(hdr),
                                  fxaa ? reinterpret_cast<float4*>(scratch) : nullptr,
                                  reinterpret_cast<uint32_t*>(out));
  if (fxaa)
    k_fxaa<<<grid, 256, 0, st>>>(C, reinterpret_cast<const float4*>(scratch), reinterpret_cast<uint32_t*>(out));
  return cuda_check(cudaGetLastError(), "display kernels");
}

}  // namespace fire
