// Gaussian random starts for the adaptive setup, generated on the device with the
// counter-based Philox-4x32-10 generator (Salmon, Moraes, Dror, Shaw, SC'11) and the
// Box-Muller transform.  Element i of the stream (seed) is a pure function of (seed, i).
#include "kernels.h"

namespace wmg {

WMG_D void mulhilo32(uint32_t a, uint32_t b, uint32_t& hi, uint32_t& lo) {
  const uint64_t p = (uint64_t)a * b;
  hi = (uint32_t)(p >> 32);
  lo = (uint32_t)p;
}

// ten Philox rounds on the counter c with key k
WMG_D uint4 philox4x32_10(uint4 c, uint2 k) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t hi0, lo0, hi1, lo1;
    mulhilo32(M0, c.x, hi0, lo0);
    mulhilo32(M1, c.z, hi1, lo1);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += W0;
    k.y += W1;
  }
  return c;
}

// out[4 i .. 4 i + 3] = four N(0, 1) numbers from counter cbase + i (stream elements 4 (cbase + i) ..)
__global__ void k_gaussian(double* out, size_t n, uint64_t seed, size_t cbase) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (4 * i >= n) return;
  const size_t ci = cbase + i;
  const uint4 r = philox4x32_10(make_uint4((uint32_t)ci, (uint32_t)(ci >> 32), 0u, 0u),
                                make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
  // (0, 1] uniforms from the top 24 bits (exact in FP32); Box-Muller in FP32 arithmetic
  const float inv = 1.0f / 16777216.0f;
  const float u0 = (float)((r.x >> 8) + 1u) * inv, u1 = (float)((r.y >> 8) + 1u) * inv;
  const float u2 = (float)((r.z >> 8) + 1u) * inv, u3 = (float)((r.w >> 8) + 1u) * inv;
  const float a = sqrtf(-2.0f * logf(u0)), b = sqrtf(-2.0f * logf(u2));
  float s0, c0, s1, c1;
  sincospif(2.0f * u1, &s0, &c0);
  sincospif(2.0f * u3, &s1, &c1);
  const double z[4] = {a * c0, a * s0, b * c1, b * s1};
  for (int j = 0; j < 4 && 4 * i + j < n; ++j) out[4 * i + j] = z[j];
}

// out[j] = element first + j of the stream of `seed` (first a multiple of 4)
void gaussian_fill(double* out, size_t n, uint64_t seed, size_t first, cudaStream_t s) {
  const size_t threads = (n + 3) / 4;
  k_gaussian<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(out, n, seed, first / 4);
  count_launch();
}

}  // namespace wmg
