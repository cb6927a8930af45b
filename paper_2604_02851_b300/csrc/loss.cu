// L1 + D-SSIM loss and its image gradient.
//
// Sec. 3.1: the optimiser "compares the result to the captured ground-truth
// images" with the configured loss.  L = w_l1 mean|x - y| + w_ssim (1 - mean
// SSIM), SSIM over an 11x11 Gaussian window (sigma 1.5, normalised), C1 =
// 0.01^2, C2 = 0.03^2, window sums with zero padding, means over every pixel,
// channel and view.
//
// Two tiled kernels, 32x32 outputs per block with a 5-pixel halo staged in
// shared memory and separable 11-tap sums (register-blocked, 4 outputs per
// thread and pass, two moments per packed FP32 instruction):
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
constexpr int SW = TW + 2 * HALO;      // 42 staged rows / columns
constexpr int SP = SW + 1;             // staged row pitch (43): conflict-free blocked reads
constexpr int HP = TW + 1;             // horizontal-pass row pitch (33)
constexpr int RB = 4;                  // outputs per thread along a pass
constexpr float C1 = 0.0001f, C2 = 0.0009f;

struct Win { float g[11]; };

__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Both kernels: 32 x 32 outputs per block of 256 threads.  The horizontal
// 11-tap pass runs on the 42 staged rows, a thread producing RB adjacent
// columns of one row from 14 staged values; the vertical pass gives each
// thread RB adjacent rows of one column from 14 horizontal sums.
__global__ void __launch_bounds__(256)
k_ssim_fwd(const float* __restrict__ x, const float* __restrict__ y, int H, int W, Win win,
           float* __restrict__ dm0, float* __restrict__ dm1, float* __restrict__ dm2,
           float2* __restrict__ partial) {
    __shared__ float sx[SW][SP], sy[SW][SP];
    __shared__ float hs[5][SW][HP];
    const int plane = blockIdx.z;
    const int64_t HW = (int64_t)H * W;
    const float* xp = x + plane * HW;
    const float* yp = y + plane * HW;
    const int ox = blockIdx.x * TW, oy = blockIdx.y * TW;
    {
        // all of this thread's loads in flight before the first store
        constexpr int NL = (SW * SW + 255) / 256;
        float lx[NL], ly[NL];
#pragma unroll
        for (int k = 0; k < NL; ++k) {
            const int i = threadIdx.x + k * 256;
            const int r = i / SW, c = i % SW;
            const int gy = oy + r - HALO, gx = ox + c - HALO;
            const bool in = i < SW * SW && gy >= 0 && gy < H && gx >= 0 && gx < W;
            lx[k] = in ? __ldg(&xp[(int64_t)gy * W + gx]) : 0.f;
            ly[k] = in ? __ldg(&yp[(int64_t)gy * W + gx]) : 0.f;
        }
#pragma unroll
        for (int k = 0; k < NL; ++k) {
            const int i = threadIdx.x + k * 256;
            if (i < SW * SW) {
                sx[i / SW][i % SW] = lx[k];
                sy[i / SW][i % SW] = ly[k];
            }
        }
    }
    __syncthreads();
    // horizontal: task = (row r of 42, column group of RB)
    for (int t = threadIdx.x; t < SW * (TW / RB); t += 256) {
        const int r = t / (TW / RB), c0 = (t % (TW / RB)) * RB;
        // (x, y), (x^2, y^2) and xy of the 14 inputs; pairs use packed FP32
        float2 v[RB + 10], v2[RB + 10];
        float vxy[RB + 10];
#pragma unroll
        for (int j = 0; j < RB + 10; ++j) {
            v[j] = make_float2(sx[r][c0 + j], sy[r][c0 + j]);
            v2[j] = __fmul2_rn(v[j], v[j]);
            vxy[j] = v[j].x * v[j].y;
        }
#pragma unroll
        for (int i = 0; i < RB; ++i) {
            float2 a01 = make_float2(0.f, 0.f), a23 = make_float2(0.f, 0.f);
            float a4 = 0.f;
#pragma unroll
            for (int k = 0; k < 11; ++k) {
                const float2 w2 = make_float2(win.g[k], win.g[k]);
                a01 = __ffma2_rn(w2, v[i + k], a01);
                a23 = __ffma2_rn(w2, v2[i + k], a23);
                a4 = fmaf(win.g[k], vxy[i + k], a4);
            }
            hs[0][r][c0 + i] = a01.x; hs[1][r][c0 + i] = a01.y; hs[2][r][c0 + i] = a23.x;
            hs[3][r][c0 + i] = a23.y; hs[4][r][c0 + i] = a4;
        }
    }
    __syncthreads();
    // vertical: thread = (column c, row group of RB)
    float ssum = 0.f, l1 = 0.f;
    {
        const int c = threadIdx.x % TW, r0 = (threadIdx.x / TW) * RB;
        float2 m01[RB], m23[RB];
        float m4[RB];
#pragma unroll
        for (int i = 0; i < RB; ++i) { m01[i] = m23[i] = make_float2(0.f, 0.f); m4[i] = 0.f; }
#pragma unroll
        for (int j = 0; j < RB + 10; ++j) {
            const float2 h01 = make_float2(hs[0][r0 + j][c], hs[1][r0 + j][c]);
            const float2 h23 = make_float2(hs[2][r0 + j][c], hs[3][r0 + j][c]);
            const float h4 = hs[4][r0 + j][c];
#pragma unroll
            for (int i = 0; i < RB; ++i) {
                const int k = j - i;
                if (k < 0 || k > 10) continue;
                const float2 w2 = make_float2(win.g[k], win.g[k]);
                m01[i] = __ffma2_rn(w2, h01, m01[i]);
                m23[i] = __ffma2_rn(w2, h23, m23[i]);
                m4[i] = fmaf(win.g[k], h4, m4[i]);
            }
        }
        const int gx = ox + c;
#pragma unroll
        for (int i = 0; i < RB; ++i) {
            const int gy = oy + r0 + i;
            if (gy >= H || gx >= W) continue;
            const float mx = m01[i].x, my = m01[i].y;
            const float sxx = m23[i].x - mx * mx, syy = m23[i].y - my * my, sxy = m4[i] - mx * my;
            const float n1 = 2.f * mx * my + C1, n2 = 2.f * sxy + C2;
            const float d1 = mx * mx + my * my + C1, d2 = sxx + syy + C2;
            const float rn1 = rcp_approx(n1), rn2 = rcp_approx(n2), rd1 = rcp_approx(d1), rd2 = rcp_approx(d2);
            const float S = n1 * n2 * rd1 * rd2;
            const int64_t p = plane * HW + (int64_t)gy * W + gx;
            dm0[p] = 2.f * S * (my * rn1 - my * rn2 - mx * rd1 + mx * rd2);
            dm1[p] = -S * rd2;
            dm2[p] = 2.f * S * rn2;
            ssum += S;
            l1 += fabsf(sx[r0 + i + HALO][c + HALO] - sy[r0 + i + HALO][c + HALO]);
        }
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
    __shared__ float sm[3][SW][SP];
    __shared__ float hs[3][SW][HP];
    const int plane = blockIdx.z;
    const int64_t HW = (int64_t)H * W;
    const int ox = blockIdx.x * TW, oy = blockIdx.y * TW;
    // the image and target at this thread's outputs, fetched early
    float xo[RB], yo[RB];
    {
        const int c = threadIdx.x % TW, r0 = (threadIdx.x / TW) * RB, gx = ox + c;
#pragma unroll
        for (int i = 0; i < RB; ++i) {
            const int gy = oy + r0 + i;
            const bool in = gy < H && gx < W;
            const int64_t p = plane * HW + (int64_t)gy * W + gx;
            xo[i] = in ? __ldg(&x[p]) : 0.f;
            yo[i] = in ? __ldg(&y[p]) : 0.f;
        }
    }
    {
        // all of this thread's loads in flight before the first store
        constexpr int NL = (SW * SW + 255) / 256;
        float l0[NL], l1[NL], l2[NL];
#pragma unroll
        for (int k = 0; k < NL; ++k) {
            const int i = threadIdx.x + k * 256;
            const int r = i / SW, c = i % SW;
            const int gy = oy + r - HALO, gx = ox + c - HALO;
            const bool in = i < SW * SW && gy >= 0 && gy < H && gx >= 0 && gx < W;
            const int64_t p = plane * HW + (int64_t)gy * W + gx;
            l0[k] = in ? __ldg(&dm0[p]) : 0.f;
            l1[k] = in ? __ldg(&dm1[p]) : 0.f;
            l2[k] = in ? __ldg(&dm2[p]) : 0.f;
        }
#pragma unroll
        for (int k = 0; k < NL; ++k) {
            const int i = threadIdx.x + k * 256;
            if (i < SW * SW) {
                sm[0][i / SW][i % SW] = l0[k];
                sm[1][i / SW][i % SW] = l1[k];
                sm[2][i / SW][i % SW] = l2[k];
            }
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < SW * (TW / RB); t += 256) {
        const int r = t / (TW / RB), c0 = (t % (TW / RB)) * RB;
        float2 v01[RB + 10];
        float v2[RB + 10];
#pragma unroll
        for (int j = 0; j < RB + 10; ++j) {
            v01[j] = make_float2(sm[0][r][c0 + j], sm[1][r][c0 + j]);
            v2[j] = sm[2][r][c0 + j];
        }
#pragma unroll
        for (int i = 0; i < RB; ++i) {
            float2 a01 = make_float2(0.f, 0.f);
            float a2 = 0.f;
#pragma unroll
            for (int k = 0; k < 11; ++k) {
                a01 = __ffma2_rn(make_float2(win.g[k], win.g[k]), v01[i + k], a01);
                a2 = fmaf(win.g[k], v2[i + k], a2);
            }
            hs[0][r][c0 + i] = a01.x; hs[1][r][c0 + i] = a01.y; hs[2][r][c0 + i] = a2;
        }
    }
    __syncthreads();
    {
        const int c = threadIdx.x % TW, r0 = (threadIdx.x / TW) * RB;
        float2 a01[RB];
        float a2[RB];
#pragma unroll
        for (int i = 0; i < RB; ++i) { a01[i] = make_float2(0.f, 0.f); a2[i] = 0.f; }
#pragma unroll
        for (int j = 0; j < RB + 10; ++j) {
            const float2 h01 = make_float2(hs[0][r0 + j][c], hs[1][r0 + j][c]);
            const float h2 = hs[2][r0 + j][c];
#pragma unroll
            for (int i = 0; i < RB; ++i) {
                const int k = j - i;
                if (k < 0 || k > 10) continue;
                a01[i] = __ffma2_rn(make_float2(win.g[k], win.g[k]), h01, a01[i]);
                a2[i] = fmaf(win.g[k], h2, a2[i]);
            }
        }
        const int gx = ox + c;
#pragma unroll
        for (int i = 0; i < RB; ++i) {
            const int gy = oy + r0 + i;
            if (gy >= H || gx >= W) continue;
            const int64_t p = plane * HW + (int64_t)gy * W + gx;
            const float xv = xo[i], yv = yo[i];
            const float d = xv - yv;
            const float sgn = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
            dx[p] = (w_l1 * sgn - w_ssim * (a01[i].x + 2.f * xv * a01[i].y + yv * a2[i])) * inv_m;
        }
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
