// Light visibility (Sec. 3.4.1): a light-space depth map seen by an
// orthographic camera attached to the directional light, and the test of each
// Gaussian centre against it.
//
// The paper takes the map from the engine's shadow pass over its meshes; here
// it is rendered from the Gaussians: texel (i, j) keeps the smallest light
// depth of the Gaussians whose splat alpha o exp(-q/2) at the texel centre
// reaches alpha_min.  Each lane sets up one Gaussian's footprint, then the
// warp splats its 32 Gaussians in turn, each lane walking columns of the
// bounding box with the quadratic stepped row by row, and merging depths with
// a float atomic min, so the map does not depend on the order of the
// Gaussians.
#include "gauss.cuh"

namespace gs {
namespace {

// Float min through integer atomics: non-negative floats order like their
// int bits, negative floats inversely like their uint bits.  The map starts
// at +inf; -0 is folded into +0 so that equal depths give equal bits.
__device__ __forceinline__ void atomic_min_float(float* addr, float v) {
    v += 0.f;
    if (v >= 0.f)
        atomicMin(reinterpret_cast<int*>(addr), __float_as_int(v));
    else
        atomicMax(reinterpret_cast<unsigned int*>(addr), __float_as_uint(v));
}

__global__ void k_light_clear(float* depth, int64_t count) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) depth[i] = __int_as_float(0x7f800000);
}

// World mean of Gaussian g in light space: (u, v) in texels, z light depth.
__device__ __forceinline__ float3 to_light(const gs_light_camera& lc, float3 mu) {
    const float dx = mu.x - lc.origin[0], dy = mu.y - lc.origin[1], dz = mu.z - lc.origin[2];
    const float xl = lc.R[0] * dx + lc.R[1] * dy + lc.R[2] * dz;
    const float yl = lc.R[3] * dx + lc.R[4] * dy + lc.R[5] * dz;
    const float zl = lc.R[6] * dx + lc.R[7] * dy + lc.R[8] * dz;
    return make_float3(xl / lc.texel + 0.5f * (float)lc.width, yl / lc.texel + 0.5f * (float)lc.height, zl);
}

// Footprint of one Gaussian on the map: centre (u, v), light depth z, conic
// (A, B, C) in texel units, bound tau = 2 ln(o / alpha_min), and the texel
// box [i0, i0 + nw) x [j0, j0 + nh).  Returns false when nothing is covered.
struct Splat {
    float u, v, z, A, B, C, tau;
    int i0, j0, nw, nh;
};

__device__ __forceinline__ bool light_splat(const float4* __restrict__ P, int64_t n, const Dyn& dyn,
                                            const gs_light_camera& lc, int64_t g, Splat& s) {
    Gauss G;
    load_gauss(P, n, g, G);
    apply_dyn(dyn, g, G);
    const float3 p = to_light(lc, G.mu);
    // nothing is covered below alpha_min
    s.tau = 2.f * logf(G.opac / lc.alpha_min);
    if (!(s.tau >= 0.f) || !isfinite(p.x) || !isfinite(p.y) || !isfinite(p.z)) return false;
    // Sigma2 = R_2 Sigma R_2^T / texel^2 + 0.3 I
    const float* S = G.S;
    const float* R = lc.R;
    const float S0[3] = {S[0] * R[0] + S[1] * R[1] + S[2] * R[2], S[1] * R[0] + S[3] * R[1] + S[4] * R[2],
                         S[2] * R[0] + S[4] * R[1] + S[5] * R[2]};
    const float S1[3] = {S[0] * R[3] + S[1] * R[4] + S[2] * R[5], S[1] * R[3] + S[3] * R[4] + S[4] * R[5],
                         S[2] * R[3] + S[4] * R[4] + S[5] * R[5]};
    const float ih2 = 1.f / (lc.texel * lc.texel);
    const float a = (R[0] * S0[0] + R[1] * S0[1] + R[2] * S0[2]) * ih2 + kDilation;
    const float b = (R[3] * S0[0] + R[4] * S0[1] + R[5] * S0[2]) * ih2;
    const float c = (R[3] * S1[0] + R[4] * S1[1] + R[5] * S1[2]) * ih2 + kDilation;
    const float det = a * c - b * b;
    if (!(det > 0.f)) return false;
    const float id = 1.f / det;
    s.A = c * id; s.B = -b * id; s.C = a * id;
    // q <= tau implies |d|^2 <= tau * lmax; widened a little against rounding
    const float mid = 0.5f * (a + c);
    const float lmax = mid + sqrtf(fmaxf(0.f, mid * mid - det));
    const float r = sqrtf(s.tau * lmax) * 1.0001f + 0.01f;
    const float W = (float)lc.width, H = (float)lc.height;
    s.i0 = (int)fminf(fmaxf(ceilf(p.x - r - 0.5f), 0.f), W);
    const int i1 = (int)fminf(fmaxf(floorf(p.x + r - 0.5f), -1.f), W - 1.f);
    s.j0 = (int)fminf(fmaxf(ceilf(p.y - r - 0.5f), 0.f), H);
    const int j1 = (int)fminf(fmaxf(floorf(p.y + r - 0.5f), -1.f), H - 1.f);
    s.nw = i1 - s.i0 + 1;
    s.nh = j1 - s.j0 + 1;
    s.u = p.x; s.v = p.y; s.z = p.z;
    return s.nw > 0 && s.nh > 0;
}

// Each lane sets up one Gaussian's footprint; the warp then walks the
// footprints one after another, its lanes taking the footprint's columns.
__global__ void __launch_bounds__(256)
k_light_depth(const float4* __restrict__ P, int64_t n, Dyn dyn, gs_light_camera lc, float* __restrict__ depth) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    Splat mine{};
    const bool ok = g < n && light_splat(P, n, dyn, lc, g, mine);
    unsigned todo = __ballot_sync(0xffffffffu, ok);
    while (todo) {
        const int src = __ffs(todo) - 1;
        todo &= todo - 1;
        const float u = __shfl_sync(0xffffffffu, mine.u, src), v = __shfl_sync(0xffffffffu, mine.v, src);
        const float z = __shfl_sync(0xffffffffu, mine.z, src), tau = __shfl_sync(0xffffffffu, mine.tau, src);
        const float A = __shfl_sync(0xffffffffu, mine.A, src), B = __shfl_sync(0xffffffffu, mine.B, src);
        const float C = __shfl_sync(0xffffffffu, mine.C, src);
        const int i0 = __shfl_sync(0xffffffffu, mine.i0, src), j0 = __shfl_sync(0xffffffffu, mine.j0, src);
        const int nw = __shfl_sync(0xffffffffu, mine.nw, src), nh = __shfl_sync(0xffffffffu, mine.nh, src);
        // lane l walks the columns l, l + 32, ... of the box top to bottom,
        // stepping the quadratic by rows: q(dy + 1) = q + 2 B dx + C (2 dy + 1)
        // (rounding differences at q ~ tau decide a boundary texel either way)
        const float twoB = 2.f * B;
        for (int ci = lane; ci < nw; ci += 32) {
            const float dx = (float)(i0 + ci) + 0.5f - u;
            float dy = (float)j0 + 0.5f - v;
            float q = (A * dx + twoB * dy) * dx + C * dy * dy;
            const float qx = twoB * dx + C;  // row step is qx + 2 C dy
            float* texel = depth + (int64_t)j0 * lc.width + (i0 + ci);
            for (int r = 0; r < nh; ++r) {
                if (q <= tau) atomic_min_float(texel, z);
                q += qx + 2.f * C * dy;
                dy += 1.f;
                texel += lc.width;
            }
        }
    }
}

__global__ void __launch_bounds__(256)
k_light_vis(const float4* __restrict__ P, int64_t n, Dyn dyn, gs_light_camera lc, const float* __restrict__ depth,
            uint8_t* __restrict__ vis) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    const float4 p0 = P[g];
    float3 mu = make_float3(p0.x, p0.y, p0.z);
    if (dyn.group) {
        const uint32_t grp = min((uint32_t)dyn.group[g], (uint32_t)(dyn.n_groups - 1));
        const float4 q = dyn.poses[2 * grp], t = dyn.poses[2 * grp + 1];
        float Rg[9];
        quat_rot(q.x, q.y, q.z, q.w, Rg);
        mu = make_float3(Rg[0] * mu.x + Rg[1] * mu.y + Rg[2] * mu.z + t.x,
                         Rg[3] * mu.x + Rg[4] * mu.y + Rg[5] * mu.z + t.y,
                         Rg[6] * mu.x + Rg[7] * mu.y + Rg[8] * mu.z + t.z);
    }
    const float3 p = to_light(lc, mu);
    const float fi = floorf(p.x), fj = floorf(p.y);
    uint8_t out = 255;
    if (fi >= 0.f && fi < (float)lc.width && fj >= 0.f && fj < (float)lc.height) {
        const float D = __ldg(&depth[(int64_t)fj * lc.width + (int64_t)fi]);
        out = p.z <= D + lc.bias ? 255 : 0;
    }
    vis[g] = out;
}

}  // namespace

void launch_light_depth(const float* params, int64_t n, const Dyn& dyn, const gs_light_camera& lc, float* depth,
                        int clear, cudaStream_t st) {
    const int64_t count = (int64_t)lc.width * lc.height;
    if (clear) k_light_clear<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(depth, count);
    if (n <= 0) return;
    const int threads = 256;
    const unsigned blocks = (unsigned)((n + threads - 1) / threads);
    k_light_depth<<<blocks, threads, 0, st>>>(reinterpret_cast<const float4*>(params), n, dyn, lc, depth);
}

void launch_light_visibility(const float* params, int64_t n, const Dyn& dyn, const gs_light_camera& lc,
                             const float* depth, uint8_t* vis, cudaStream_t st) {
    if (n <= 0) return;
    const int threads = 256;
    const unsigned blocks = (unsigned)((n + threads - 1) / threads);
    k_light_vis<<<blocks, threads, 0, st>>>(reinterpret_cast<const float4*>(params), n, dyn, lc, depth, vis);
}

}  // namespace gs
