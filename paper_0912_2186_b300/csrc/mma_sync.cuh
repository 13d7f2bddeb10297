// Legacy warp-level tensor-core MMA (mma.sync m16n8k16, FP16 operands, FP32 accumulation) and
// the FP16 packing used by the coarse stencil kernels.
#pragma once
#include <cuda_fp16.h>

#include "wmg_common.cuh"

namespace wmg {

constexpr int kKPad = 8;  // halves of padding per staged column (bank-conflict-free B loads)

WMG_D uint32_t pack_half2(float lo, float hi) {
  __half2 h = __floats2half2_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&h);
}

// d (16x8, FP32) += a (16x16, FP16, fragment of this lane) * b (16x8, FP16, fragment b0, b1)
WMG_D void mma16816(float d[4], const uint4& a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b0), "r"(b1));
}

}  // namespace wmg
