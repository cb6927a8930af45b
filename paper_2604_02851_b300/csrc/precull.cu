// Preculling visibility of grid cells (Sec. 3.3: Gaussians are assigned to
// grid cells, each camera determines its visible cells by depth testing, and
// only Gaussians of visible cells enter rendering and optimisation).
//
// Per view, the depth buffer's max pyramid is built level by level (level
// k + 1 of size ((w + 1) / 2, (h + 1) / 2) holds the maxima of 2x2 blocks).
// One thread per cell then projects the cell's 8 corners into every view
// (float32 with fused multiply-adds, IEEE division), takes the pixel range of
// the corners (or the whole image at depth `near` when the cell straddles the
// near plane), picks the first pyramid level at which that range spans at
// most two texels per axis and keeps the cell when its nearest corner depth is
// at most the maximum of those texels.  The test is conservative: a cell
// whose pixels show something at or behind it is never dropped.
#include <math.h>

#include "gs_internal.cuh"

namespace gs {
namespace {

__host__ __device__ inline size_t mip_floats(int W, int H) {
    size_t s = 0;
    for (;;) {
        s += (size_t)W * H;
        if (W == 1 && H == 1) break;
        W = (W + 1) / 2;
        H = (H + 1) / 2;
    }
    return s;
}

__global__ void k_mip_level(const float* __restrict__ in, int w, int h, float* __restrict__ out, int w2, int h2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)w2 * h2) return;
    const int x = (int)(i % w2), y = (int)(i / w2);
    float m = -INFINITY;
#pragma unroll
    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
        for (int dx = 0; dx < 2; ++dx) {
            const int yy = 2 * y + dy, xx = 2 * x + dx;
            if (yy < h && xx < w) m = fmaxf(m, in[(size_t)yy * w + xx]);
        }
    out[i] = m;
}

__global__ void __launch_bounds__(256)
k_cell_visibility(const gs_camera* __restrict__ cams, int V, const float* __restrict__ mips, float ox, float oy,
                  float oz, float size, int nx, int ny, int nz, uint8_t* __restrict__ vis) {
    const int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t ncell = (int64_t)nx * ny * nz;
    if (cell >= ncell) return;
    const int cx = (int)(cell % nx), cy = (int)((cell / nx) % ny), cz = (int)(cell / ((int64_t)nx * ny));
    uint8_t seen = 0;
    size_t base = 0;
    for (int v = 0; v < V && !seen; ++v) {
        const gs_camera c = cams[v];
        const int W = c.width, H = c.height;
        const float* mv = mips + base;
        base += mip_floats(W, H);
        float umin = INFINITY, umax = -INFINITY, vmin = INFINITY, vmax = -INFINITY, zmin = INFINITY;
        int behind = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const float px = __fmaf_rn(size, (float)(cx + (k & 1)), ox);
            const float py = __fmaf_rn(size, (float)(cy + ((k >> 1) & 1)), oy);
            const float pz = __fmaf_rn(size, (float)(cz + ((k >> 2) & 1)), oz);
            const float X = __fmaf_rn(c.R[0], px, __fmaf_rn(c.R[1], py, __fmaf_rn(c.R[2], pz, c.t[0])));
            const float Y = __fmaf_rn(c.R[3], px, __fmaf_rn(c.R[4], py, __fmaf_rn(c.R[5], pz, c.t[1])));
            const float Z = __fmaf_rn(c.R[6], px, __fmaf_rn(c.R[7], py, __fmaf_rn(c.R[8], pz, c.t[2])));
            if (Z <= c.near_plane) { ++behind; continue; }
            const float u = __fmaf_rn(c.fx, __fdiv_rn(X, Z), c.cx), w = __fmaf_rn(c.fy, __fdiv_rn(Y, Z), c.cy);
            umin = fminf(umin, u); umax = fmaxf(umax, u);
            vmin = fminf(vmin, w); vmax = fmaxf(vmax, w);
            zmin = fminf(zmin, Z);
        }
        if (behind == 8) continue;
        long long x0, x1, y0, y1;
        if (behind) {
            x0 = 0; x1 = W - 1; y0 = 0; y1 = H - 1; zmin = c.near_plane;
        } else {
            x0 = (long long)floorf(umin); x1 = (long long)floorf(umax);
            y0 = (long long)floorf(vmin); y1 = (long long)floorf(vmax);
            if (x1 < 0 || y1 < 0 || x0 > W - 1 || y0 > H - 1) continue;
            x0 = x0 < 0 ? 0 : x0; y0 = y0 < 0 ? 0 : y0;
            x1 = x1 > W - 1 ? W - 1 : x1; y1 = y1 > H - 1 ? H - 1 : y1;
        }
        // first level whose texels cover the range with at most 2 per axis
        int L = 0, w = W, h = H;
        size_t off = 0;
        while ((w > 1 || h > 1) && (((x1 >> L) - (x0 >> L)) > 1 || ((y1 >> L) - (y0 >> L)) > 1)) {
            off += (size_t)w * h;
            w = (w + 1) / 2;
            h = (h + 1) / 2;
            ++L;
        }
        float m = -INFINITY;
        for (long long j = y0 >> L; j <= (y1 >> L); ++j)
            for (long long i = x0 >> L; i <= (x1 >> L); ++i) m = fmaxf(m, mv[off + (size_t)j * w + i]);
        if (zmin <= m) seen = 1;
    }
    vis[cell] = seen;
}

}  // namespace

size_t precull_scratch_bytes(const gs_camera* host_cams, int V) {
    size_t s = 0;
    for (int v = 0; v < V; ++v) s += mip_floats(host_cams[v].width, host_cams[v].height);
    return align_up(s * sizeof(float), 256);
}

void launch_cell_visibility(const gs_camera* d_cams, const gs_camera* host_cams, int V, const float* depth,
                            const gs_precull& grid, uint8_t* vis, char* scratch, cudaStream_t st) {
    float* mips = reinterpret_cast<float*>(scratch);
    size_t base = 0, doff = 0;
    for (int v = 0; v < V; ++v) {
        int w = host_cams[v].width, h = host_cams[v].height;
        float* lvl = mips + base;
        cudaMemcpyAsync(lvl, depth + doff, sizeof(float) * (size_t)w * h, cudaMemcpyDeviceToDevice, st);
        doff += (size_t)w * h;
        while (w > 1 || h > 1) {
            const int w2 = (w + 1) / 2, h2 = (h + 1) / 2;
            float* next = lvl + (size_t)w * h;
            const int64_t cnt = (int64_t)w2 * h2;
            k_mip_level<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(lvl, w, h, next, w2, h2);
            lvl = next;
            w = w2;
            h = h2;
        }
        base += mip_floats(host_cams[v].width, host_cams[v].height);
    }
    const int64_t ncell = (int64_t)grid.dims[0] * grid.dims[1] * grid.dims[2];
    if (ncell > 0)
        k_cell_visibility<<<(unsigned)((ncell + 255) / 256), 256, 0, st>>>(
            d_cams, V, mips, grid.origin[0], grid.origin[1], grid.origin[2], grid.cell_size, grid.dims[0],
            grid.dims[1], grid.dims[2], vis);
}

}  // namespace gs
