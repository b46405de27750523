// Requantisation arithmetic shared by the separate requantise kernels and the
// requantise fused into the 2 x 2 shuffle tail, written with explicit roundings
// (__fmul_rn / __fadd_rn / __fmaf_rn) so that the compiler contracts nothing on
// its own: both paths give the same codes, sample for sample.
#pragma once

#include <cuda_runtime.h>

namespace nvisr {

// a * wa + b * wb (one rounding for b * wb, one fused multiply-add)
__device__ __forceinline__ float rq_blend(float a, float wa, float b, float wb) {
    return __fmaf_rn(a, wa, __fmul_rn(b, wb));
}

// bilinear blend of the corners (row 0: a00, a01; row 1: a10, a11) at fractions (lx, ly)
__device__ __forceinline__ float rq_bilerp(float a00, float a01, float a10, float a11, float lx, float ly) {
    const float top = rq_blend(a00, __fsub_rn(1.f, lx), a01, lx);
    const float bot = rq_blend(a10, __fsub_rn(1.f, lx), a11, lx);
    return rq_blend(top, __fsub_rn(1.f, ly), bot, ly);
}

// R'G'B' -> Y', Cb', Cr' with luma weights (kr, kg, kb) and chroma scales 1 / (2(1 - kb)),
// 1 / (2(1 - kr))
__device__ __forceinline__ void rq_ycc(float r, float g, float b, float kr, float kg, float kb, float cb_s, float cr_s,
                                       float &y, float &cb, float &cr) {
    y = __fmaf_rn(kb, b, __fmaf_rn(kg, g, __fmul_rn(kr, r)));
    cb = __fmul_rn(__fsub_rn(b, y), cb_s);
    cr = __fmul_rn(__fsub_rn(r, y), cr_s);
}

// code of a normalised value: v * mul + add, rounded half to even, clamped to [0, vmax]
__device__ __forceinline__ float rq_code(float v, float mul, float add, float vmax) {
    const float q = rintf(__fmaf_rn(v, mul, add));
    return fminf(fmaxf(q, 0.0f), vmax);
}

// mean of two values; [1 2 1] / 4 of three
__device__ __forceinline__ float rq_mean2(float a, float b) { return __fmul_rn(0.5f, __fadd_rn(a, b)); }
__device__ __forceinline__ float rq_121(float a, float b, float c) {
    return __fmul_rn(0.25f, __fadd_rn(__fadd_rn(a, __fmul_rn(2.0f, b)), c));
}

}  // namespace nvisr
