// Element types of the tensor-core kernels and the packed FP32 helpers their
// epilogues share: two 16-bit elements of a 32-bit word <-> two floats, and
// two-lane FP32 add / multiply / fused multiply-add (f32x2, IEEE round to
// nearest per lane, the same results as the scalar operations).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "common.cuh"

namespace nvisr {
namespace {

template <int DT>
struct Elem;
template <>
struct Elem<DT_BF16> { using T = __nv_bfloat16; };
template <>
struct Elem<DT_F16> { using T = __half; };
template <>
struct Elem<DT_E4M3> { using T = __nv_fp8_e4m3; };
template <>
struct Elem<DT_F32> { using T = float; };

// Packed two-lane FP32 arithmetic (IEEE round-to-nearest per lane, as the scalar ops).
__device__ __forceinline__ void add_f32x2(float &a, float &b, float c, float d) {
    uint64_t x, y;
    asm("mov.b64 %0, {%1, %2};" : "=l"(x) : "f"(a), "f"(b));
    asm("mov.b64 %0, {%1, %2};" : "=l"(y) : "f"(c), "f"(d));
    asm("add.rn.f32x2 %0, %0, %1;" : "+l"(x) : "l"(y));
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(x));
}
__device__ __forceinline__ void fma_f32x2(float &a, float &b, float s0, float s1, float c0, float c1) {
    uint64_t x, y, z;
    asm("mov.b64 %0, {%1, %2};" : "=l"(x) : "f"(a), "f"(b));
    asm("mov.b64 %0, {%1, %2};" : "=l"(y) : "f"(s0), "f"(s1));
    asm("mov.b64 %0, {%1, %2};" : "=l"(z) : "f"(c0), "f"(c1));
    asm("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x) : "l"(y), "l"(z));
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(x));
}
__device__ __forceinline__ void mul_f32x2(float &a, float &b, float c, float d) {
    uint64_t x, y;
    asm("mov.b64 %0, {%1, %2};" : "=l"(x) : "f"(a), "f"(b));
    asm("mov.b64 %0, {%1, %2};" : "=l"(y) : "f"(c), "f"(d));
    asm("mul.rn.f32x2 %0, %0, %1;" : "+l"(x) : "l"(y));
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(x));
}
// Two 16-bit elements of one 32-bit word (element 0 in the low half) <-> two floats.
template <typename T>
__device__ __forceinline__ void unpack2(uint32_t w, float &lo, float &hi);
template <>
__device__ __forceinline__ void unpack2<__nv_bfloat16>(uint32_t w, float &lo, float &hi) {
    lo = __uint_as_float(w << 16);
    hi = __uint_as_float(w & 0xffff0000u);
}
template <>
__device__ __forceinline__ void unpack2<__half>(uint32_t w, float &lo, float &hi) {
    const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&w));
    lo = f.x;
    hi = f.y;
}
template <typename T>
__device__ __forceinline__ uint32_t pack2(float lo, float hi);
template <>
__device__ __forceinline__ uint32_t pack2<__nv_bfloat16>(float lo, float hi) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&h);
}
template <>
__device__ __forceinline__ uint32_t pack2<__half>(float lo, float hi) {
    const __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&h);
}

}  // namespace
}  // namespace nvisr
