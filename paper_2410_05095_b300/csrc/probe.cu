// Measurement aid (no counterpart in the paper): the read bandwidth of one
// persistent launch over a device buffer, used as the L2 peak beside which
// the traversal kernels' L2 traffic is reported.  A buffer that fits in L2,
// read `reps` times with 16-B loads cached in L2 only (ld.global.cg, so L1
// does not serve the repeats), measures the L2 read rate; a buffer larger
// than L2 measures DRAM.
#include <algorithm>

#include "fire_internal.cuh"

namespace fire {
namespace {

__global__ void __launch_bounds__(256) k_read_probe(const uint4* __restrict__ buf, int64_t n16, int reps,
                                                    uint32_t* __restrict__ sink) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t first = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  uint32_t acc = 0u;
  for (int r = 0; r < reps; ++r) {
    // a rotating start spreads the repeats over different L2 slices per warp
    const int64_t start = (first + (int64_t)r * 4096 * 32) % stride;
    for (int64_t i = start; i < n16; i += stride) {
      const uint4 v = __ldcg(buf + i);
      acc ^= v.x ^ v.y ^ v.z ^ v.w;
    }
  }
  // keep the loads: one word per thread block, never read for its value
  acc = __reduce_xor_sync(0xffffffffu, acc);
  if ((threadIdx.x & 31) == 0) atomicXor(sink + blockIdx.x, acc);
}

}  // namespace
}  // namespace fire

using namespace fire;

extern "C" int fire_probe_read(const void* buf, int64_t bytes, int32_t reps, uint32_t* sink, int32_t sink_words,
                               void* stream) {
  set_error(FIRE_OK, "");
  if (!buf || !sink || bytes < 16 || bytes % 16 != 0 || reps < 1 ||
      (reinterpret_cast<uintptr_t>(buf) & 15u) != 0)
    return set_error(FIRE_ERR_INVALID_ARG, "probe: buffer must be 16-B aligned, a multiple of 16 B, reps >= 1");
  const int grid = sm_count() * 4;
  if (sink_words < grid) return set_error(FIRE_ERR_INVALID_ARG, "probe: sink needs 4 words per SM");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  k_read_probe<<<grid, 256, 0, st>>>(static_cast<const uint4*>(buf), bytes / 16, reps, sink);
  return cuda_check(cudaGetLastError(), "k_read_probe");
}
