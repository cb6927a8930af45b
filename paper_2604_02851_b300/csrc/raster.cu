// Per-tile front-to-back alpha compositing and its reverse-order adjoint.
//
// Sec. 3.2.3: the model is refined by differentiable rendering as in the
// cited 3DGS method.  One block owns one B x B pixel tile; its sorted list of
// Gaussians is streamed through shared memory in batches, and every pixel of
// the tile walks each batch.  A thread owns a strip of B/4 pixels of one row,
// so a fragment's shared-memory reads and its per-warp gradient reduction
// serve several pixels.
//
// Forward: per pixel, alpha = min(0.99, o e^P) with P the conic quadratic
// form, skipped when P > 0 or alpha < 1/255 (tested as P log2(e) <
// -log2(255 o) before the exponential, which is evaluated in base 2);
// compositing stops before the fragment that would take T below 1e-4.  A block leaves as soon as every pixel is done (block vote).
//
// Backward: no per-fragment state is stored.  Each pixel starts from its
// final transmittance and last-contributor position and walks its list
// backwards, recovering T_j = T_{j+1} / (1 - alpha_j) and the colour behind
// the fragment by the recursion R_{j-1} = alpha_j c_j + (1 - alpha_j) R_j
// (R = background behind the last fragment).  Per fragment, a thread sums its
// pixels' 9 gradient values, the warp sums them with shuffles, the warp sums
// of a batch are added in shared memory, and each batch ends with one set of
// vector atomics per Gaussian into the per-view 2D gradient record.
#include "gs_internal.cuh"

namespace gs {
namespace {

__device__ __forceinline__ int find_view(const ViewInfo* __restrict__ vt, int V, int64_t gt) {
    int lo = 0, hi = V;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (vt[mid].tile_off <= gt) lo = mid; else hi = mid;
    }
    return lo;
}

// Thread layout: a B x B tile is covered by B rows of TPR threads; each
// thread owns a strip of PX = B / TPR adjacent pixels of one row, so the
// shared-memory reads of a fragment and the warp reductions of its gradient
// are shared by PX pixels.  B * TPR is a multiple of 32 (whole warps).
constexpr float kLog2e = 1.4426950408889634f;

// The exponent is evaluated in base 2: with q = -log2(e)/2 (A, 2B, C), the
// quadratic form P log2(e) = (qA dx + qB dy) dx + qC dy^2 and e^P = 2^(P log2 e);
// the cut-off alpha < 1/255, o e^P < 1/255, is P log2(e) < -log2(255 o).
__device__ __forceinline__ float ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float4 log2_conic(float4 co) {
    return make_float4(-0.5f * kLog2e * co.x, -kLog2e * co.y, -0.5f * kLog2e * co.z, 0.f);
}
__device__ __forceinline__ float cutoff_log2(float o) { return -__log2f(255.f * o); }

template <int B, int TPR>
__global__ void __launch_bounds__(B * TPR)
k_render_fwd(const float4* __restrict__ proj, const ViewInfo* __restrict__ vt, int V, int64_t n,
             const uint32_t* __restrict__ vals, const uint2* __restrict__ ranges, float3 bg,
             float* __restrict__ image, float* __restrict__ T_final, uint32_t* __restrict__ n_contrib) {
    constexpr int NT = B * TPR;        // threads per block
    constexpr int PX = B / TPR;        // pixels per thread
    static_assert(NT % 32 == 0, "whole warps");
    constexpr int BATCH = 2 * NT;      // fragments staged per round
    __shared__ float4 s_a[BATCH];      // u, v, opacity, log2 cut-off
    __shared__ float4 s_q[BATCH];      // base-2 conic coefficients
    __shared__ float4 s_c[BATCH];      // r, g, b
    const int64_t gt = blockIdx.x;
    if (gt >= vt[V].tile_off) return;
    const int v = find_view(vt, V, gt);
    const ViewInfo vi = vt[v];
    const int lt = (int)(gt - vi.tile_off);
    const int row = (int)threadIdx.x / TPR;
    const int px0 = (lt % vi.tx) * B + ((int)threadIdx.x % TPR) * PX;
    const int py = (lt / vi.tx) * B + row;
    const float fy = (float)py + 0.5f;
    const float fx0 = (float)px0 + 0.5f;
    const uint2 rg = ranges[gt];
    const int64_t rbase = (int64_t)v * n;

    float T[PX], Cr[PX], Cg[PX], Cb[PX];
    uint32_t last[PX];
    uint32_t live = 0;  // bit k: pixel k still compositing
#pragma unroll
    for (int k = 0; k < PX; ++k) {
        T[k] = 1.f; Cr[k] = Cg[k] = Cb[k] = 0.f; last[k] = 0;
        if (px0 + k < vi.width && py < vi.height) live |= 1u << k;
    }
    for (uint32_t start = rg.x; start < rg.y; start += BATCH) {
        if (__syncthreads_count(live != 0) == 0) break;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int slot = threadIdx.x + h * NT;
            const uint32_t idx = start + slot;
            if (idx < rg.y) {
                const int64_t r = (rbase + vals[idx]) * 4;
                const float4 a = proj[r], b = proj[r + 1], c = proj[r + 2];
                s_a[slot] = make_float4(a.x, a.y, a.w, cutoff_log2(a.w));
                s_q[slot] = log2_conic(b);
                s_c[slot] = c;
            }
        }
        __syncthreads();
        const int cnt = (int)min((uint32_t)BATCH, rg.y - start);
        for (int j = 0; j < cnt && live; ++j) {
            const float4 a = s_a[j];
            const float4 q = s_q[j];
            const float dy = a.y - fy;
            const float qb = q.y * dy;
            const float qc = q.z * dy * dy;
            const float dx0 = a.x - fx0;
#pragma unroll
            for (int k = 0; k < PX; ++k) {
                if (!(live & (1u << k))) continue;
                const float dx = dx0 - (float)k;
                const float P2 = (q.x * dx + qb) * dx + qc;
                if (P2 > 0.f || P2 < a.w) continue;
                const float al = fminf(kAlphaMax, a.z * ex2(P2));
                const float Tn = T[k] * (1.f - al);
                if (Tn < kTMin) { live &= ~(1u << k); continue; }
                const float4 c = s_c[j];
                const float w = al * T[k];
                Cr[k] += c.x * w; Cg[k] += c.y * w; Cb[k] += c.z * w;
                T[k] = Tn;
                last[k] = start + j - rg.x + 1;
            }
        }
    }
    const int64_t HW = (int64_t)vi.width * vi.height;
    float* img = image + 3 * vi.pix_off;
#pragma unroll
    for (int k = 0; k < PX; ++k) {
        const int px = px0 + k;
        if (px >= vi.width || py >= vi.height) continue;
        const int64_t pix = (int64_t)py * vi.width + px;
        img[pix] = Cr[k] + T[k] * bg.x;
        img[HW + pix] = Cg[k] + T[k] * bg.y;
        img[2 * HW + pix] = Cb[k] + T[k] * bg.z;
        if (T_final) T_final[vi.pix_off + pix] = T[k];
        if (n_contrib) n_contrib[vi.pix_off + pix] = last[k];
    }
}

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
    return x;
}

// Warp sums of 8 values at once (reduce-scatter): at the exchanges over lane
// bits 4, 3 and 2 a lane keeps half of its partial vector and receives the
// partner's sums of that half; two full exchanges over bits 1 and 0 finish.
// On return every lane l holds the warp sum of value l >> 2.  14 shuffles
// instead of 40.
__device__ __forceinline__ float warp_sum8(const float (&v)[8], int lane) {
    float a[4], b[2];
    const bool u4 = lane & 16, u3 = lane & 8, u2 = lane & 4;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float send = u4 ? v[i] : v[i + 4];
        const float keep = u4 ? v[i + 4] : v[i];
        a[i] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, 16);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float send = u3 ? a[i] : a[i + 2];
        const float keep = u3 ? a[i + 2] : a[i];
        b[i] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, 8);
    }
    const float send = u2 ? b[0] : b[1];
    float c = (u2 ? b[1] : b[0]) + __shfl_xor_sync(0xFFFFFFFFu, send, 4);
    c += __shfl_xor_sync(0xFFFFFFFFu, c, 2);
    c += __shfl_xor_sync(0xFFFFFFFFu, c, 1);
    return c;
}

// Approximate reciprocal (relative error below 2^-22).
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Geometry gradients from five sums over a fragment's pixels:
//   S1 = sum dP dx, S2 = sum dP dy, S3 = sum dP dx^2, S4 = sum dP dx dy,
//   S5 = sum dP dy^2  (dP = dL/dP, dx = u - px, dy = v - py), so that
//   dL/du = -A S1 - B S2, dL/dv = -C S2 - B S1,
//   dL/dA = -S3 / 2, dL/dB = -S4, dL/dC = -S5 / 2.
// A thread's pixels share one row (one dy): it keeps sum dP, sum dP dx and
// sum dP dx^2 per pixel and forms S2, S4, S5 with its dy once per fragment.
template <int B, int TPR>
__global__ void __launch_bounds__(B * TPR)
k_raster_bwd(const float4* __restrict__ proj, const ViewInfo* __restrict__ vt, int V, int64_t n,
             const uint32_t* __restrict__ vals, const uint2* __restrict__ ranges, float3 bg,
             const float* __restrict__ T_final, const uint32_t* __restrict__ n_contrib,
             const float* __restrict__ dimage, float* __restrict__ grad2d, int64_t n_active) {
    constexpr int NT = B * TPR;
    constexpr int PX = B / TPR;
    static_assert(NT % 32 == 0, "whole warps");
    constexpr int BATCH = NT;
    __shared__ float4 s_a[BATCH];   // u, v, opacity, log2 cut-off
    __shared__ float4 s_q[BATCH];   // base-2 conic coefficients
    __shared__ float4 s_b[BATCH];   // conic A, B, C
    __shared__ float4 s_c[BATCH];   // r, g, b
    __shared__ uint32_t s_g[BATCH];
    __shared__ float s_acc[9][BATCH];
    __shared__ uint32_t s_max;
    const int64_t gt = blockIdx.x;
    if (gt >= vt[V].tile_off) return;
    const int v = find_view(vt, V, gt);
    const ViewInfo vi = vt[v];
    const int lt = (int)(gt - vi.tile_off);
    const int row = (int)threadIdx.x / TPR;
    const int px0 = (lt % vi.tx) * B + ((int)threadIdx.x % TPR) * PX;
    const int py = (lt / vi.tx) * B + row;
    const float fy = (float)py + 0.5f;
    const float fx0 = (float)px0 + 0.5f;
    const uint2 rg = ranges[gt];
    const int64_t rbase = (int64_t)v * n;
    const int lane = threadIdx.x & 31;

    float T[PX], dCr[PX], dCg[PX], dCb[PX], Rr[PX], Rg[PX], Rb[PX];
    uint32_t last[PX];
    uint32_t mylast = 0;
    const int64_t HW = (int64_t)vi.width * vi.height;
    const float* dimg = dimage + 3 * vi.pix_off;
#pragma unroll
    for (int k = 0; k < PX; ++k) {
        const int px = px0 + k;
        T[k] = 1.f; dCr[k] = dCg[k] = dCb[k] = 0.f; last[k] = 0;
        Rr[k] = bg.x; Rg[k] = bg.y; Rb[k] = bg.z;
        if (px < vi.width && py < vi.height) {
            const int64_t pix = (int64_t)py * vi.width + px;
            T[k] = T_final[vi.pix_off + pix];
            last[k] = n_contrib[vi.pix_off + pix];
            dCr[k] = dimg[pix]; dCg[k] = dimg[HW + pix]; dCb[k] = dimg[2 * HW + pix];
            mylast = max(mylast, last[k]);
        }
    }
    if (threadIdx.x == 0) s_max = 0;
    __syncthreads();
    if (mylast) atomicMax(&s_max, mylast);
    __syncthreads();
    const uint32_t maxl = s_max;

    for (int64_t bend = maxl; bend > 0; bend -= BATCH) {
        const uint32_t bstart = bend > BATCH ? (uint32_t)(bend - BATCH) : 0u;
        const int cnt = (int)(bend - bstart);
        __syncthreads();  // the previous batch's flush is complete
        if ((int)threadIdx.x < cnt) {
            const uint32_t g = vals[rg.x + bstart + threadIdx.x];
            const int64_t r = (rbase + g) * 4;
            const float4 a = proj[r], b = proj[r + 1], c = proj[r + 2];
            s_a[threadIdx.x] = make_float4(a.x, a.y, a.w, cutoff_log2(a.w));
            s_q[threadIdx.x] = log2_conic(b);
            s_b[threadIdx.x] = b;
            s_c[threadIdx.x] = c;
            s_g[threadIdx.x] = g;
#pragma unroll
            for (int q = 0; q < 9; ++q) s_acc[q][threadIdx.x] = 0.f;
        }
        __syncthreads();
        for (int j = cnt - 1; j >= 0; --j) {
            const uint32_t pos = bstart + (uint32_t)j;
            if (!__any_sync(0xFFFFFFFFu, pos < mylast)) continue;
            const float4 a = s_a[j];
            const float4 q = s_q[j];
            const float4 c = s_c[j];
            const float dy = a.y - fy;
            const float qb = q.y * dy;
            const float qc = q.z * dy * dy;
            const float dx0 = a.x - fx0;
            float s0 = 0.f, s1 = 0.f, s2 = 0.f, g5 = 0.f, g6 = 0.f, g7 = 0.f, g8 = 0.f;
            bool contrib = false;
#pragma unroll
            for (int k = 0; k < PX; ++k) {
                if (pos >= last[k]) continue;
                const float dx = dx0 - (float)k;
                const float P2 = (q.x * dx + qb) * dx + qc;
                if (P2 > 0.f || P2 < a.w) continue;
                contrib = true;
                const float G = ex2(P2);
                const float raw = a.z * G;
                const float al = fminf(kAlphaMax, raw);
                const float Tj = T[k] * rcp_approx(1.f - al);
                T[k] = Tj;
                const float w = al * Tj;
                g6 += w * dCr[k]; g7 += w * dCg[k]; g8 += w * dCb[k];
                const float er = c.x - Rr[k], eg = c.y - Rg[k], eb = c.z - Rb[k];
                const float dal = Tj * (dCr[k] * er + dCg[k] * eg + dCb[k] * eb);
                Rr[k] += al * er;
                Rg[k] += al * eg;
                Rb[k] += al * eb;
                const bool free = raw <= kAlphaMax;
                const float dP = free ? dal * raw : 0.f;
                g5 += free ? dal * G : 0.f;
                const float t = dP * dx;
                s0 += dP;
                s1 += t;
                s2 += t * dx;
            }
            // frozen Gaussians (index >= n_active) take part in the
            // recursion but need no gradient
            if (s_g[j] < n_active && __any_sync(0xFFFFFFFFu, contrib)) {
                // lane 4q ends with sum q of (S1, S2, S3, S4, S5, g5, g6, g7)
                const float vals8[8] = {s1, s0 * dy, s2, s1 * dy, s0 * dy * dy, g5, g6, g7};
                const float mine = warp_sum8(vals8, lane);
                const float S1 = __shfl_sync(0xFFFFFFFFu, mine, 0), S2 = __shfl_sync(0xFFFFFFFFu, mine, 4);
                g8 = warp_sum(g8);
                const int q = lane >> 2;
                if ((lane & 3) == 0 || lane == 1) {
                    // the conic and mean gradients from the five sums:
                    // dL/du = -A S1 - B S2, dL/dv = -C S2 - B S1,
                    // dL/dA = -S3 / 2, dL/dB = -S4, dL/dC = -S5 / 2
                    const float4 co = s_b[j];
                    float val;
                    int slot;
                    if (lane == 1) { val = g8; slot = 8; }
                    else {
                        slot = q;
                        val = q == 0 ? -co.x * S1 - co.y * S2
                            : q == 1 ? -co.z * S2 - co.y * S1
                            : q == 2 ? -0.5f * mine
                            : q == 3 ? -mine
                            : q == 4 ? -0.5f * mine : mine;
                    }
                    if (NT == 32) s_acc[slot][j] += val;
                    else atomicAdd(&s_acc[slot][j], val);
                }
            }
        }
        __syncthreads();
        if ((int)threadIdx.x < cnt) {
            const int t = threadIdx.x;
            const float4 A = make_float4(s_acc[0][t], s_acc[1][t], s_acc[2][t], s_acc[3][t]);
            const float4 Bv = make_float4(s_acc[4][t], s_acc[5][t], s_acc[6][t], s_acc[7][t]);
            const float Cv = s_acc[8][t];
            float* dst = grad2d + (rbase + s_g[t]) * kGradStride;
            if (A.x != 0.f || A.y != 0.f || A.z != 0.f || A.w != 0.f)
                atomicAdd(reinterpret_cast<float4*>(dst), A);
            if (Bv.x != 0.f || Bv.y != 0.f || Bv.z != 0.f || Bv.w != 0.f)
                atomicAdd(reinterpret_cast<float4*>(dst + 4), Bv);
            if (Cv != 0.f) atomicAdd(dst + 8, Cv);
        }
    }
}

}  // namespace

void launch_render_fwd(const float* proj, const ViewInfo* vt, int V, int64_t n, int tile, int tpr,
                       const uint32_t* vals, const uint32_t* ranges, float3 bg, float* image,
                       float* T_final, uint32_t* n_contrib, int64_t total_tiles, cudaStream_t st) {
    if (total_tiles <= 0) return;
    const float4* p = reinterpret_cast<const float4*>(proj);
    const uint2* r = reinterpret_cast<const uint2*>(ranges);
    const unsigned nb = (unsigned)total_tiles;
    if (tile == 8)
        k_render_fwd<8, 4><<<nb, 32, 0, st>>>(p, vt, V, n, vals, r, bg, image, T_final, n_contrib);
    else if (tpr == 2)
        k_render_fwd<16, 2><<<nb, 32, 0, st>>>(p, vt, V, n, vals, r, bg, image, T_final, n_contrib);
    else
        k_render_fwd<16, 4><<<nb, 64, 0, st>>>(p, vt, V, n, vals, r, bg, image, T_final, n_contrib);
}

void launch_raster_bwd(const float* proj, const ViewInfo* vt, int V, int64_t n, int tile, int tpr,
                       const uint32_t* vals, const uint32_t* ranges, float3 bg, const float* T_final,
                       const uint32_t* n_contrib, const float* dimage, float* grad2d,
                       int64_t total_tiles, cudaStream_t st, int64_t n_active) {
    if (n_active < 0) n_active = n;
    cudaMemsetAsync(grad2d, 0, sizeof(float) * kGradStride * (size_t)V * (size_t)n, st);
    if (total_tiles <= 0) return;
    const float4* p = reinterpret_cast<const float4*>(proj);
    const uint2* r = reinterpret_cast<const uint2*>(ranges);
    const unsigned nb = (unsigned)total_tiles;
    if (tile == 8)
        k_raster_bwd<8, 4><<<nb, 32, 0, st>>>(p, vt, V, n, vals, r, bg, T_final, n_contrib, dimage, grad2d, n_active);
    else if (tpr == 2)
        k_raster_bwd<16, 2><<<nb, 32, 0, st>>>(p, vt, V, n, vals, r, bg, T_final, n_contrib, dimage, grad2d, n_active);
    else
        k_raster_bwd<16, 4><<<nb, 64, 0, st>>>(p, vt, V, n, vals, r, bg, T_final, n_contrib, dimage, grad2d, n_active);
}

}  // namespace gs
