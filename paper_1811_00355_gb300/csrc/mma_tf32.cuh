// Tensor-core helpers: mma.sync m16n8k8 with TF32 inputs and FP32
// accumulation, each FP32 operand split as x = hi + lo (both TF32) and the
// product taken as a_hi b_hi + a_hi b_lo + a_lo b_hi (the "3xTF32" scheme of
// Ootomo and Yokota, IJHPCA 2022), which keeps FP32 accuracy.
//
// Fragments (g = lane / 4, t = lane % 4):
//   A (16 x 8, row-major):  a0 (g, t), a1 (g + 8, t), a2 (g, t + 4), a3 (g + 8, t + 4)
//   B (8 x 8, k x n):       b0 (k = t, n = g), b1 (k = t + 4, n = g)
//   C (16 x 8):             c0 (g, 2t), c1 (g, 2t + 1), c2 (g + 8, 2t), c3 (g + 8, 2t + 1)
#pragma once

#include <cstdint>

namespace ddamg {

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void split(float x, uint32_t& hi, uint32_t& lo) {
  hi = to_tf32(x);
  lo = to_tf32(x - __uint_as_float(hi));
}
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
// an operand fragment split into TF32 parts
template <int N>
struct Split {
  uint32_t hi[N], lo[N];
};
template <int N>
__device__ __forceinline__ Split<N> split_frag(const float (&v)[N]) {
  Split<N> s;
#pragma unroll
  for (int e = 0; e < N; ++e) split(v[e], s.hi[e], s.lo[e]);
  return s;
}
// d += a b from split operands (small terms first)
__device__ __forceinline__ void mma3(float (&d)[4], const Split<4>& a, const Split<2>& b) {
  mma_tf32(d, a.lo, b.hi);
  mma_tf32(d, a.hi, b.lo);
  mma_tf32(d, a.hi, b.hi);
}

}  // namespace ddamg
