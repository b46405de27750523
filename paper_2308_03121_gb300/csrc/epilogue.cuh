// Epilogue helpers shared by the convolution kernels: activation and the
// network's skip path (upsampled input frame added to the final residual).
#pragma once

#include "common.cuh"

namespace nvisr {

static __device__ __forceinline__ float lrelu(float v) { return v >= 0.f ? v : 0.1f * v; }

// Skip value of planar float32 frame(s) at output (c, Y, X) for integer scale s.
static __device__ __forceinline__ float skip_value(const ConvArgs &a, int c, int Y, int X, int s, int H, int W) {
    if (a.skip_mode == 0 || a.nskip == 0) return 0.f;
    float acc = 0.f;
    for (int f = 0; f < a.nskip; ++f) {
        const float *p = a.skip_src[f] + (int64_t)c * a.skip_plane;
        float v;
        if (a.skip_mode == 1) {
            v = p[(int64_t)(Y / s) * a.skip_pitch + X / s];
        } else {
            const float inv = 1.0f / (float)s;
            float sy = fmaxf(((float)Y + 0.5f) * inv - 0.5f, 0.f);
            float sx = fmaxf(((float)X + 0.5f) * inv - 0.5f, 0.f);
            int y0 = min((int)sy, H - 1), x0 = min((int)sx, W - 1);
            int y1 = min(y0 + 1, H - 1), x1 = min(x0 + 1, W - 1);
            float ly = sy - (float)y0, lx = sx - (float)x0;
            const float *r0 = p + (int64_t)y0 * a.skip_pitch;
            const float *r1 = p + (int64_t)y1 * a.skip_pitch;
            float top = r0[x0] * (1.f - lx) + r0[x1] * lx;
            float bot = r1[x0] * (1.f - lx) + r1[x1] * lx;
            v = top * (1.f - ly) + bot * ly;
        }
        acc += v;
    }
    return a.nskip == 2 ? acc * 0.5f : acc;
}

}  // namespace nvisr
