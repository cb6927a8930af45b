// L1 + D-SSIM loss and its image gradient.
//
// Sec. 3.1: the optimiser "compares the result to the captured ground-truth
// images" with the configured loss.  L = w_l1 mean|x - y| + w_ssim (1 - mean
// SSIM), SSIM over an 11x11 Gaussian window (sigma 1.5, normalised), C1 =
// 0.01^2, C2 = 0.03^2, window sums with zero padding, means over every pixel,
// channel and view.
//
// Two tiled kernels, 32x32 outputs per block with a 5-pixel halo staged in
// shared memory and separable 11-tap sums:
//   k_ssim_fwd: the five window moments -> SSIM map value and its partials
//     dS/dmu_x, dS/dE[x^2], dS/dE[xy] (three maps), plus per-block sums of S
//     and |x - y|;
//   k_ssim_bwd: window sums of the three partial maps -> dL/dx, and (block 0)
//     a fixed-order FP64 reduction of the block sums into the loss.
#include <math.h>

#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int TW = 32;                 // output tile width / height
constexpr int HALO = 5;
constexpr int SW = TW + 2 * HALO;      // 42
constexpr float C1 = 0.0001f, C2 = 0.0009f;

struct Win { float g[11]; };

__global__ void __launch_bounds__(256)
k_ssim_fwd(const float* __restrict__ x, const float* __restrict__ y, int H, int W, Win win,
           float* __restrict__ dm0, float* __restrict__ dm1, float* __restrict__ dm2,
           float2* __restrict__ partial) {
    __shared__ float sx[SW][SW], sy[SW][SW];
    __shared__ float hs[5][SW][TW];
    const int plane = blockIdx.z;
    const int64_t HW = (int64_t)H * W;
    const float* xp = x + plane * HW;
    const float* yp = y + plane * HW;
    const int ox = blockIdx.x * TW, oy = blockIdx.y * TW;
    for (int i = threadIdx.x; i < SW * SW; i += 256) {
        const int r = i / SW, c = i % SW;
        const int gy = oy + r - HALO, gx = ox + c - HALO;
        const bool in = gy >= 0 && gy < H && gx >= 0 && gx < W;
        sx[r][c] = in ? xp[(int64_t)gy * W + gx] : 0.f;
        sy[r][c] = in ? yp[(int64_t)gy * W + gx] : 0.f;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < SW * TW; i += 256) {
        const int r = i / TW, c = i % TW;
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f, a4 = 0.f;
#pragma unroll
        for (int k = 0; k < 11; ++k) {
            const float w = win.g[k], xv = sx[r][c + k], yv = sy[r][c + k];
            a0 += w * xv; a1 += w * yv; a2 += w * xv * xv; a3 += w * yv * yv; a4 += w * xv * yv;
        }
        hs[0][r][c] = a0; hs[1][r][c] = a1; hs[2][r][c] = a2; hs[3][r][c] = a3; hs[4][r][c] = a4;
    }
    __syncthreads();
    float ssum = 0.f, l1 = 0.f;
    for (int i = threadIdx.x; i < TW * TW; i += 256) {
        const int r = i / TW, c = i % TW;
        const int gy = oy + r, gx = ox + c;
        if (gy >= H || gx >= W) continue;
        float mx = 0.f, my = 0.f, exx = 0.f, eyy = 0.f, exy = 0.f;
#pragma unroll
        for (int k = 0; k < 11; ++k) {
            const float w = win.g[k];
            mx += w * hs[0][r + k][c]; my += w * hs[1][r + k][c];
            exx += w * hs[2][r + k][c]; eyy += w * hs[3][r + k][c]; exy += w * hs[4][r + k][c];
        }
        const float sxx = exx - mx * mx, syy = eyy - my * my, sxy = exy - mx * my;
        const float n1 = 2.f * mx * my + C1, n2 = 2.f * sxy + C2;
        const float d1 = mx * mx + my * my + C1, d2 = sxx + syy + C2;
        const float S = (n1 * n2) / (d1 * d2);
        const int64_t p = plane * HW + (int64_t)gy * W + gx;
        dm0[p] = S * (2.f * my / n1 - 2.f * my / n2 - 2.f * mx / d1 + 2.f * mx / d2);
        dm1[p] = -S / d2;
        dm2[p] = 2.f * S / n2;
        ssum += S;
        l1 += fabsf(sx[r + HALO][c + HALO] - sy[r + HALO][c + HALO]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ssum += __shfl_xor_sync(0xFFFFFFFFu, ssum, o);
        l1 += __shfl_xor_sync(0xFFFFFFFFu, l1, o);
    }
    __shared__ float2 ws[8];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = make_float2(ssum, l1);
    __syncthreads();
    if (threadIdx.x == 0) {
        float2 t = make_float2(0.f, 0.f);
        for (int w = 0; w < 8; ++w) { t.x += ws[w].x; t.y += ws[w].y; }
        partial[((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(256)
k_ssim_bwd(const float* __restrict__ x, const float* __restrict__ y, int H, int W, Win win,
           const float* __restrict__ dm0, const float* __restrict__ dm1, const float* __restrict__ dm2,
           float inv_m, float w_l1, float w_ssim, float* __restrict__ dx,
           const float2* __restrict__ partial, int64_t n_partial, double m_total, float* __restrict__ d_loss) {
    __shared__ float sm[3][SW][SW];
    __shared__ float hs[3][SW][TW];
    const int plane = blockIdx.z;
    const int64_t HW = (int64_t)H * W;
    const int ox = blockIdx.x * TW, oy = blockIdx.y * TW;
    for (int i = threadIdx.x; i < SW * SW; i += 256) {
        const int r = i / SW, c = i % SW;
        const int gy = oy + r - HALO, gx = ox + c - HALO;
        const bool in = gy >= 0 && gy < H && gx >= 0 && gx < W;
        const int64_t p = plane * HW + (int64_t)gy * W + gx;
        sm[0][r][c] = in ? dm0[p] : 0.f;
        sm[1][r][c] = in ? dm1[p] : 0.f;
        sm[2][r][c] = in ? dm2[p] : 0.f;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < SW * TW; i += 256) {
        const int r = i / TW, c = i % TW;
        float a0 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll
        for (int k = 0; k < 11; ++k) {
            const float w = win.g[k];
            a0 += w * sm[0][r][c + k]; a1 += w * sm[1][r][c + k]; a2 += w * sm[2][r][c + k];
        }
        hs[0][r][c] = a0; hs[1][r][c] = a1; hs[2][r][c] = a2;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < TW * TW; i += 256) {
        const int r = i / TW, c = i % TW;
        const int gy = oy + r, gx = ox + c;
        if (gy >= H || gx >= W) continue;
        float a0 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll
        for (int k = 0; k < 11; ++k) {
            const float w = win.g[k];
            a0 += w * hs[0][r + k][c]; a1 += w * hs[1][r + k][c]; a2 += w * hs[2][r + k][c];
        }
        const int64_t p = plane * HW + (int64_t)gy * W + gx;
        const float xv = x[p], yv = y[p];
        const float d = xv - yv;
        const float sgn = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
        dx[p] = (w_l1 * sgn - w_ssim * (a0 + 2.f * xv * a1 + yv * a2)) * inv_m;
    }
    if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0) {
        __shared__ double rs[256], rl[256];
        double s = 0.0, l = 0.0;
        for (int64_t i = threadIdx.x; i < n_partial; i += 256) { s += partial[i].x; l += partial[i].y; }
        rs[threadIdx.x] = s;
        rl[threadIdx.x] = l;
        __syncthreads();
        if (threadIdx.x == 0) {
            double S = 0.0, L1 = 0.0;
            for (int i = 0; i < 256; ++i) { S += rs[i]; L1 += rl[i]; }
            *d_loss = (float)((double)w_l1 * L1 / m_total + (double)w_ssim * (1.0 - S / m_total));
        }
    }
}

Win make_window() {
    double g[11], s = 0.0;
    for (int i = 0; i < 11; ++i) { g[i] = exp(-(double)((i - 5) * (i - 5)) / (2.0 * 1.5 * 1.5)); s += g[i]; }
    Win w;
    for (int i = 0; i < 11; ++i) w.g[i] = (float)(g[i] / s);
    return w;
}

}  // namespace

size_t loss_scratch_bytes(int V, int H, int W) {
    Carver c(nullptr);
    const int64_t px = (int64_t)V * 3 * H * W;
    c.take<float>(px); c.take<float>(px); c.take<float>(px);
    const int64_t nb = (int64_t)((W + TW - 1) / TW) * ((H + TW - 1) / TW) * V * 3;
    c.take<float2>(nb);
    return c.off;
}

void launch_loss(const float* image, const float* target, int V, int H, int W, float w_l1, float w_ssim,
                 float* d_loss, float* dimage, char* scratch, cudaStream_t st) {
    Carver c(scratch);
    const int64_t px = (int64_t)V * 3 * H * W;
    float* dm0 = c.take<float>(px);
    float* dm1 = c.take<float>(px);
    float* dm2 = c.take<float>(px);
    const dim3 grid((W + TW - 1) / TW, (H + TW - 1) / TW, V * 3);
    const int64_t nb = (int64_t)grid.x * grid.y * grid.z;
    float2* partial = c.take<float2>(nb);
    const Win win = make_window();
    k_ssim_fwd<<<grid, 256, 0, st>>>(image, target, H, W, win, dm0, dm1, dm2, partial);
    k_ssim_bwd<<<grid, 256, 0, st>>>(image, target, H, W, win, dm0, dm1, dm2, (float)(1.0 / (double)px),
                                     w_l1, w_ssim, dimage, partial, nb, (double)px, d_loss);
}

}  // namespace gs
