/*
 * conv_oracle.c -- plain FP64 3-D convolution (forward and both gradients) for checking the
 * surrogate's tensor-core kernels. TEST INFRASTRUCTURE ONLY (see rt_oracle.c).
 *
 * The surrogate is a stack of 3x3x3 convolutions with "same" zero padding and dilation d:
 *     y[b][o][z][y][x] = bias[o] + sum_{i, kz, ky, kx} w[o][i][kz][ky][kx]
 *                          * x[b][i][z + (kz-1) d][y + (ky-1) d][x + (kx-1) d]     (0 outside)
 * (cross-correlation, the convention of common deep-learning libraries). Layouts are plain
 * NCDHW, weights [c_out][c_in][3][3][3].
 */
#include <stdlib.h>

static double at(const double *x, int b, int c, int z, int y, int xx, int C, int D, int H, int W)
{
    if (z < 0 || z >= D || y < 0 || y >= H || xx < 0 || xx >= W) return 0.0;
    return x[((((long)b * C + c) * D + z) * H + y) * W + xx];
}

int oracle_conv3d_fwd(const double *x, const double *w, const double *bias, int B, int Ci, int Co,
                      int D, int H, int W, int dil, double *y)
{
    if (B < 0 || Ci < 1 || Co < 1 || D < 1 || H < 1 || W < 1 || dil < 1) return -1;
    for (int b = 0; b < B; ++b)
        for (int o = 0; o < Co; ++o)
            for (int z = 0; z < D; ++z)
                for (int yy = 0; yy < H; ++yy)
                    for (int xx = 0; xx < W; ++xx) {
                        double s = bias ? bias[o] : 0.0;
                        for (int i = 0; i < Ci; ++i)
                            for (int kz = 0; kz < 3; ++kz)
                                for (int ky = 0; ky < 3; ++ky)
                                    for (int kx = 0; kx < 3; ++kx)
                                        s += w[(((long)o * Ci + i) * 3 + kz) * 9 + ky * 3 + kx] *
                                             at(x, b, i, z + (kz - 1) * dil, yy + (ky - 1) * dil,
                                                xx + (kx - 1) * dil, Ci, D, H, W);
                        y[((((long)b * Co + o) * D + z) * H + yy) * W + xx] = s;
                    }
    return 0;
}

/* Gradients for dL/dy = gy: gx (may be NULL), gw and gbias (may be NULL), all OVERWRITTEN.
 *   gx[b][i][p]        = sum_{o,k} w[o][i][k] gy[b][o][p - (k-1) d]
 *   gw[o][i][k]        = sum_{b,p} gy[b][o][p] x[b][i][p + (k-1) d]
 *   gbias[o]           = sum_{b,p} gy[b][o][p]                                           */
int oracle_conv3d_bwd(const double *x, const double *w, const double *bias, int B, int Ci, int Co,
                      int D, int H, int W, int dil, const double *gy, double *gx, double *gw,
                      double *gbias)
{
    (void)bias;
    if (B < 0 || Ci < 1 || Co < 1 || D < 1 || H < 1 || W < 1 || dil < 1) return -1;
    const long nvox = (long)D * H * W;
    if (gx)
        for (long q = 0; q < (long)B * Ci * nvox; ++q) gx[q] = 0.0;
    if (gw)
        for (long q = 0; q < (long)Co * Ci * 27; ++q) gw[q] = 0.0;
    if (gbias)
        for (int o = 0; o < Co; ++o) gbias[o] = 0.0;
    for (int b = 0; b < B; ++b)
        for (int o = 0; o < Co; ++o)
            for (int z = 0; z < D; ++z)
                for (int yy = 0; yy < H; ++yy)
                    for (int xx = 0; xx < W; ++xx) {
                        const double g = gy[((((long)b * Co + o) * D + z) * H + yy) * W + xx];
                        if (gbias) gbias[o] += g;
                        for (int i = 0; i < Ci; ++i)
                            for (int kz = 0; kz < 3; ++kz)
                                for (int ky = 0; ky < 3; ++ky)
                                    for (int kx = 0; kx < 3; ++kx) {
                                        const int sz = z + (kz - 1) * dil, sy = yy + (ky - 1) * dil;
                                        const int sx = xx + (kx - 1) * dil;
                                        if (sz < 0 || sz >= D || sy < 0 || sy >= H || sx < 0 || sx >= W) continue;
                                        const long wi = (((long)o * Ci + i) * 3 + kz) * 9 + ky * 3 + kx;
                                        const long xi = ((((long)b * Ci + i) * D + sz) * H + sy) * W + sx;
                                        if (gw) gw[wi] += g * x[xi];
                                        if (gx) gx[xi] += g * w[wi];
                                    }
                    }
    return 0;
}
