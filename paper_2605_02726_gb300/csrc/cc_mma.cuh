// Warp-level tensor-core helpers: mma.sync.m16n8k8 TF32 with a hi/lo split that keeps FP32-level
// accuracy, and the fragment conventions shared by the kernels that use them.
//
// Fragments of m16n8k8 (g = lane / 4, t = lane % 4):
//   A (16x8):  a0 = A[g][t], a1 = A[g+8][t], a2 = A[g][t+4], a3 = A[g+8][t+4]
//   B (8x8):   b0 = B[t][g], b1 = B[t+4][g]
//   C (16x8):  c0 = C[g][2t], c1 = C[g][2t+1], c2 = C[g+8][2t], c3 = C[g+8][2t+1]
#pragma once

#include <stdint.h>

namespace cc {
namespace {

// x = hi + lo: hi keeps the 10 explicit mantissa bits a TF32 operand carries, lo = x - hi is
// exact in FP32 and enters the MMA with its own low 13 bits ignored, an error of at most
// 2^-20 |x|.
__device__ __forceinline__ void split2(float x, uint32_t& hi, uint32_t& lo) {
    hi = __float_as_uint(x) & 0xffffe000u;
    lo = __float_as_uint(x - __uint_as_float(hi));
}
struct AFrag {
    uint32_t h[4], l[4];
};
__device__ __forceinline__ AFrag make_a(float a0, float a1, float a2, float a3) {
    AFrag f;
    split2(a0, f.h[0], f.l[0]);
    split2(a1, f.h[1], f.l[1]);
    split2(a2, f.h[2], f.l[2]);
    split2(a3, f.h[3], f.l[3]);
    return f;
}
__device__ __forceinline__ void mma1(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
// A * B at FP32 accuracy into two independent accumulator chains: dh += Ah Bh, dl += Al Bh + Ah Bl
// (the result is dh + dl); B from the per-lane fragment table entry (b0h, b1h, b0l, b1l).
__device__ __forceinline__ void mma3(float (&dh)[4], float (&dl)[4], const AFrag& a, const float4& b) {
    mma1(dh, a.h, __float_as_uint(b.x), __float_as_uint(b.y));
    mma1(dl, a.l, __float_as_uint(b.x), __float_as_uint(b.y));
    mma1(dl, a.h, __float_as_uint(b.z), __float_as_uint(b.w));
}
__device__ __forceinline__ void add4(float (&d)[4], const float (&e)[4]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) d[q] += e[q];
}
__device__ __forceinline__ void mma3b(float (&d)[4], const AFrag& a, const AFrag& b) {  // b.h[0..1], b.l[0..1]
    mma1(d, a.l, b.h[0], b.h[1]);
    mma1(d, a.h, b.l[0], b.l[1]);
    mma1(d, a.h, b.h[0], b.h[1]);
}
// ldmatrix of 32-bit values: a matrix "row" is 4 consecutive floats (16 bytes) of shared memory,
// and lane l receives float l % 4 of row l / 4 of each 8x4 matrix.  `row` is this lane's row
// address (16-byte aligned): lanes 8m..8m+7 address the rows of matrix m.
__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const float* row) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(row);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}
__device__ __forceinline__ void split_u(uint32_t x, uint32_t& hi, uint32_t& lo) { split2(__uint_as_float(x), hi, lo); }
// v[i] for a runtime i without a dynamically indexed (local-memory) array
template <int NV>
__device__ __forceinline__ float sel(const float (&v)[NV], int i) {
    float r = v[0];
#pragma unroll
    for (int j = 1; j < NV; ++j) r = i == j ? v[j] : r;
    return r;
}
// A fragment from an accumulator fragment (chunk permutation: slot t <- col 2t, slot t+4 <- col 2t+1)
__device__ __forceinline__ AFrag chain(const float (&c)[4]) { return make_a(c[0], c[2], c[1], c[3]); }


}  // namespace
}  // namespace cc
