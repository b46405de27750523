/*
 * FP64 oracle: direct convolution and modulated deformable convolution.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code with
 * the CUDA path.
 *
 * Both routines are the plain definitions, written as nested loops over the
 * output and the reduction, in double precision.  Tensors are planar
 * [channel][row][column], weights are [cout][cin][k][k] (PyTorch OIHW).
 *
 *  - nvo_conv2d: 2-D cross-correlation, stride 1, zero padding (k-1)/2, + bias
 *    (the convolutional layers of the enhancement networks NNVISR hosts,
 *    Section 3.1 "Network Integration").
 *  - nvo_dcn2d: modulated deformable convolution V2 with the operand layout of
 *    torchvision's deform_conv2d, which the paper's DCNv2 operator follows
 *    (Section 3.1): for output pixel p, tap k = (ky, kx), input channel c in
 *    offset group g = c / (cin / G):
 *        y[o,p] = b[o] + sum_{c,k} w[o,c,k] * m[g,k](p) * bilin(x_c, p + p_k + d[g,k](p))
 *    with p_k = (ky-1, kx-1), offsets d[g,k] = (off[2(gK+k)], off[2(gK+k)+1]) =
 *    (dy, dx), mask m[g,k] = mask[gK+k], and bilinear interpolation in which
 *    every corner outside the image contributes zero.
 *
 * Output windows: both routines compute output rows [r0, r1) and columns
 * [c0, c1) only (pass 0, h, 0, w for the whole image); the output array is
 * always the full [cout][h][w] array.
 */
#include <math.h>
#include <stddef.h>

void nvo_conv2d(const double *x, int cin, int h, int w,
                const double *wt, const double *bias, int cout, int k,
                double *y, int r0, int r1, int c0, int c1)
{
    const int pad = (k - 1) / 2;
#pragma omp parallel for collapse(2) schedule(dynamic, 1)
    for (int o = 0; o < cout; ++o) {
        for (int yy = r0; yy < r1; ++yy) {
            for (int xx = c0; xx < c1; ++xx) {
                double acc = bias ? bias[o] : 0.0;
                for (int c = 0; c < cin; ++c) {
                    for (int ky = 0; ky < k; ++ky) {
                        const int iy = yy + ky - pad;
                        if (iy < 0 || iy >= h) continue;
                        for (int kx = 0; kx < k; ++kx) {
                            const int ix = xx + kx - pad;
                            if (ix < 0 || ix >= w) continue;
                            acc += wt[(((size_t)o * cin + c) * k + ky) * k + kx] *
                                   x[((size_t)c * h + iy) * w + ix];
                        }
                    }
                }
                y[((size_t)o * h + yy) * w + xx] = acc;
            }
        }
    }
}

/* Bilinear sample of one plane at (sy, sx); corners outside the image add 0. */
static double bilinear_zero(const double *plane, int h, int w, double sy, double sx)
{
    const double fy = floor(sy), fx = floor(sx);
    const int y0 = (int)fy, x0 = (int)fx;
    const double ly = sy - fy, lx = sx - fx;
    double v = 0.0;
    for (int dy = 0; dy < 2; ++dy) {
        const int yy = y0 + dy;
        if (yy < 0 || yy >= h) continue;
        const double wy = dy ? ly : 1.0 - ly;
        for (int dx = 0; dx < 2; ++dx) {
            const int xx = x0 + dx;
            if (xx < 0 || xx >= w) continue;
            const double wx = dx ? lx : 1.0 - lx;
            v += wy * wx * plane[(size_t)yy * w + xx];
        }
    }
    return v;
}

void nvo_dcn2d(const double *x, int cin, int h, int w,
               const double *off, const double *mask, int groups,
               const double *wt, const double *bias, int cout,
               double *y, int r0, int r1, int c0, int c1)
{
    const size_t hw = (size_t)h * w;
    const int cpg = cin / groups;
#pragma omp parallel for collapse(2) schedule(dynamic, 1)
    for (int yy = r0; yy < r1; ++yy) {
        for (int xx = c0; xx < c1; ++xx) {
            const size_t p = (size_t)yy * w + xx;
            for (int o = 0; o < cout; ++o) {
                double acc = bias ? bias[o] : 0.0;
                for (int c = 0; c < cin; ++c) {
                    const int g = c / cpg;
                    for (int ky = 0; ky < 3; ++ky) {
                        for (int kx = 0; kx < 3; ++kx) {
                            const int kk = ky * 3 + kx;
                            const double dy = off[(size_t)(2 * (g * 9 + kk)) * hw + p];
                            const double dx = off[(size_t)(2 * (g * 9 + kk) + 1) * hw + p];
                            const double m = mask[(size_t)(g * 9 + kk) * hw + p];
                            const double v = bilinear_zero(x + (size_t)c * hw, h, w,
                                                           yy + ky - 1 + dy, xx + kx - 1 + dx);
                            acc += wt[(((size_t)o * cin + c) * 3 + ky) * 3 + kx] * m * v;
                        }
                    }
                }
                y[(size_t)o * hw + p] = acc;
            }
        }
    }
}

/* Number of OpenMP threads the routines above use (1 without OpenMP). */
#ifdef _OPENMP
#include <omp.h>
int nvo_threads(void) { return omp_get_max_threads(); }
#else
int nvo_threads(void) { return 1; }
#endif
