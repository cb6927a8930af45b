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
// form (P <= 0: the conic is positive definite), skipped when alpha < 1/255
// (tested as P log2(e) < -log2(255 o) before the exponential, which is
// evaluated in base 2); compositing stops before the fragment that would take
// T below 1e-4.  A block leaves as soon as every pixel is done (block vote).
// A thread's pixels are processed in pairs with packed float2 arithmetic
// (one instruction for both pixels of a pair), without a branch per pixel.
//
// Backward: no per-fragment state is stored.  Each pixel starts from its
// final transmittance and last-contributor position and walks its list
// backwards, recovering T_j = T_{j+1} / (1 - alpha_j) and the colour behind
// the fragment by the recursion R_{j-1} = alpha_j c_j + (1 - alpha_j) R_j
// (R = background behind the last fragment), kept as its product with the
// pixel's fixed dL/dC.  Per fragment, a thread sums its
// pixels' 9 gradient values, the warp sums them with shuffles, the warp sums
// of a batch are added in shared memory, and each batch ends with one set of
// vector atomics per Gaussian into the per-view 2D gradient record.
#include <type_traits>

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

// The tile a block composites.  With a super-tile order (chunk-bitmap lists)
// block b takes slot b % 64 of the (b / 64)-th super-tile of the order, and
// returns false for slots outside the view; else block b takes tile b.
__device__ __forceinline__ bool block_tile(const ViewInfo* __restrict__ vt, int V, const CoarseLists& cl,
                                           int64_t& gt, int& v) {
    if (cl.sorder) {
        const int64_t sidx = cl.sorder[blockIdx.x >> (2 * kSuperShift)];
        if (sidx >= vt[V].stile_off) return false;
        int lo = 0, hi = V;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (vt[mid].stile_off <= sidx) lo = mid; else hi = mid;
        }
        v = lo;
        const ViewInfo& vi = vt[v];
        const int ls = (int)(sidx - vi.stile_off);
        const int k = (int)(blockIdx.x & (kSuper * kSuper - 1));
        const int tx = (ls % vi.stx) * kSuper + (k & (kSuper - 1));
        const int ty = (ls / vi.stx) * kSuper + (k >> kSuperShift);
        if (tx >= vi.tx || ty >= vi.ty) return false;
        gt = vi.tile_off + (int64_t)ty * vi.tx + tx;
        return true;
    }
    gt = blockIdx.x;
    if (gt >= vt[V].tile_off) return false;
    v = find_view(vt, V, gt);
    return true;
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

// Tile culling of staged fragments.  A tile's list holds every Gaussian whose
// 3-sigma square meets the tile; many of them reach no pixel of it with
// alpha >= 1/255 (an elongated or faint splat misses the corner tiles of its
// square).  The largest base-2 exponent over the tile's pixel-centre box
// decides: P2 = qA dx^2 + qB dx dy + qC dy^2 (qA, qC < 0) is concave, so its
// maximum over the box is 0 when the centre lies inside and otherwise the
// largest of the maxima along the four edges.  A fragment is dropped when
// that maximum lies below the cut-off by more than kCullMargin, far beyond
// the rounding of either evaluation, so every pixel's own test would have
// rejected it: images, transmittances, contributor counts and gradients are
// unchanged.  Kept fragments carry their position in the list.
constexpr float kCullMargin = 0.01f;

// A fragment whose opacity is at most kNoClampOpacity never reaches the 0.99
// alpha clamp: alpha = o e^P with P <= 0 up to float32 rounding (a few
// 1e-7), so alpha <= o (1 + 1e-6) < 0.99.  For such fragments the adjoint
// takes alpha = o e^P without the min and dL/dP = dL/dalpha alpha without the
// clamp test: the same values, fewer instructions.
constexpr float kNoClampOpacity = 0.9899f;

__device__ __forceinline__ float box_max_exponent(float4 q, float dxl, float dxh, float dyl, float dyh) {
    if (dxl <= 0.f && dxh >= 0.f && dyl <= 0.f && dyh >= 0.f) return 0.f;
    const float ia = __fdividef(0.5f, q.x), ic = __fdividef(0.5f, q.z);  // the margin covers the approximation
    float best = __int_as_float(0xff800000);
    const float ex[2] = {dxl, dxh}, ey[2] = {dyl, dyh};
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const float D = ex[e];  // edge dx = D: dP/ddy = 0 at dy = -qB D / (2 qC)
        const float dy = fminf(fmaxf(-q.y * D * ic, dyl), dyh);
        best = fmaxf(best, (q.x * D + q.y * dy) * D + q.z * dy * dy);
        const float E = ey[e];  // edge dy = E
        const float dx = fminf(fmaxf(-q.y * E * ia, dxl), dxh);
        best = fmaxf(best, (q.x * dx + q.y * E) * dx + q.z * E * E);
    }
    return best;
}

// true when the fragment can reach a pixel centre of the tile whose pixel
// centres span [x0, x1] x [y0, y1]
__device__ __forceinline__ bool reaches_tile(float4 a, float4 q, float x0, float x1, float y0, float y1) {
    return box_max_exponent(q, a.x - x1, a.x - x0, a.y - y1, a.y - y0) >= a.w - kCullMargin;
}

// Blocks per SM the compositing kernel is compiled for: a one-warp tile gets
// 85 registers a thread (24 tiles an SM), wider tiles 64 registers so that
// 1024 threads fit (measured faster than 768 at 85 despite a few spills).
template <int B, int TPR>
constexpr int fwd_min_blocks() { return B * TPR == 32 ? 24 : 1024 / (B * TPR); }

// Tile gt's place in the chunk-bitmap lists: its super-tile s, its local
// index k (8 y + x) there, the super-tile's chunks [c0, c1) and first item.
struct TileChunks {
    uint32_t c0, c1, k, item0;
};

__device__ __forceinline__ TileChunks tile_chunks(const CoarseLists& cl, const ViewInfo& vi, int lt) {
    const int tx = lt % vi.tx, ty = lt / vi.tx;
    const int64_t sidx = vi.stile_off + (int64_t)(ty >> kSuperShift) * vi.stx + (tx >> kSuperShift);
    TileChunks t;
    const uint32_t nch = *cl.d_n_chunks;
    t.c0 = min(cl.chunk_first[sidx], nch);
    t.c1 = min(cl.chunk_first[sidx + 1], nch);
    t.k = (uint32_t)(((ty & (kSuper - 1)) << kSuperShift) | (tx & (kSuper - 1)));
    t.item0 = cl.cranges[sidx].x;
    return t;
}

// The marked items of chunk c for this tile, in list order, into s_cand
// (positions: indices into citems); returns their count.  NT threads, each
// owning 256 / NT consecutive bits of the chunk's 256-bit mask `word`
// (this thread's 32-bit word of it); positions at or past `limit` are
// dropped.  Ends with a barrier.
template <int NT>
__device__ __forceinline__ int chunk_candidates(uint32_t word, uint32_t item_base, uint32_t limit,
                                                uint32_t* s_cand, int* s_ctot) {
    constexpr int BPT = kChunkItems / NT;
    static_assert(BPT == 4 || BPT == 8, "4 or 8 bits a thread");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t my = (word >> ((threadIdx.x * BPT) & 31)) & ((1u << BPT) - 1u);
    const uint32_t a = item_base + threadIdx.x * BPT;
    if (a >= limit) my = 0u;
    else if (limit - a < (uint32_t)BPT) my &= (1u << (limit - a)) - 1u;
    const uint32_t pc = __popc(my);
    uint32_t incl = pc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += y;
    }
    int total;
    uint32_t off = incl - pc;
    if (NT > 32) {
        if (lane == 31) s_ctot[warp] = (int)incl;
        __syncthreads();
        total = 0;
#pragma unroll
        for (int w = 0; w < NT / 32; ++w) {
            if (w < warp) off += (uint32_t)s_ctot[w];
            total += s_ctot[w];
        }
    } else {
        total = (int)__shfl_sync(0xFFFFFFFFu, incl, 31);
    }
    while (my) {
        const int b = __ffs(my) - 1;
        my &= my - 1u;
        s_cand[off++] = a + (uint32_t)b;
    }
    __syncthreads();
    return total;
}

template <int B, int TPR, bool COARSE>
__global__ void __launch_bounds__(B * TPR, fwd_min_blocks<B, TPR>())
k_render_fwd(const float4* __restrict__ proj, const ViewInfo* __restrict__ vt, int V, int64_t n,
             const uint32_t* __restrict__ vals, const uint2* __restrict__ ranges, CoarseLists cl, float3 bg,
             float* __restrict__ image, float* __restrict__ T_final, uint32_t* __restrict__ n_contrib, int rec4) {
    constexpr int NT = B * TPR;        // threads per block
    constexpr int PX = B / TPR;        // pixels per thread
    constexpr int NP = PX / 2;         // pixel pairs per thread
    static_assert(NT % 32 == 0 && PX % 2 == 0, "whole warps, pixel pairs");
    // fragments staged per round: two slots a thread for expanded lists,
    // one for chunk bitmaps (a chunk holds ~37 of a tile's candidates)
    constexpr int SLOTS = COARSE ? 1 : 2;
    constexpr int BATCH = SLOTS * NT;
    constexpr int NW = NT / 32;
    __shared__ float4 s_a[BATCH];      // u, v, opacity, log2 cut-off
    __shared__ float4 s_q[BATCH];      // base-2 conic coefficients
    __shared__ float4 s_c[BATCH];      // r, g, b
    __shared__ uint32_t s_pos[BATCH];  // position in the tile's list
    __shared__ int s_wcnt[2 * NW];
    int64_t gt;
    int v;
    if (!block_tile(vt, V, cl, gt, v)) return;
    const ViewInfo vi = vt[v];
    const int lt = (int)(gt - vi.tile_off);
    const int row = (int)threadIdx.x / TPR;
    const int px0 = (lt % vi.tx) * B + ((int)threadIdx.x % TPR) * PX;
    const int py = (lt / vi.tx) * B + row;
    const float tx0 = (float)((lt % vi.tx) * B) + 0.5f, ty0 = (float)((lt / vi.tx) * B) + 0.5f;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float fy = (float)py + 0.5f;
    const float fx0 = (float)px0 + 0.5f;
    const int64_t rbase = (int64_t)v * n;
    __shared__ uint32_t s_cand[COARSE ? kChunkItems : 1];
    __shared__ int s_ctot[NW];

    // pixel pairs (2p, 2p + 1) in packed float2 registers.  nk holds the
    // negated offset of each pixel from the strip's first one (dx = dx0 + nk,
    // exactly dx0 - k) while it composites and +inf once it has stopped (or
    // lies outside the image): then dx = +inf and the exponent (concave, its
    // dx^2 coefficient negative) is -inf, which fails the alpha cut-off test.
    const float kPosInf = __int_as_float(0x7f800000);
    float2 T[NP], Cr[NP], Cg[NP], Cb[NP], nk[NP];
    uint32_t last[PX];
    int nlive = 0;  // pixels of this thread still compositing
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        T[p] = make_float2(1.f, 1.f);
        Cr[p] = Cg[p] = Cb[p] = make_float2(0.f, 0.f);
        const bool in0 = px0 + 2 * p < vi.width && py < vi.height;
        const bool in1 = px0 + 2 * p + 1 < vi.width && py < vi.height;
        nk[p] = make_float2(in0 ? -(float)(2 * p) : kPosInf, in1 ? -(float)(2 * p + 1) : kPosInf);
        nlive += (int)in0 + (int)in1;
    }
#pragma unroll
    for (int k = 0; k < PX; ++k) last[k] = 0;
    // One round: list items [0, nslot) of a window, item(i, pos, g) giving
    // item i's list position and Gaussian.  The fragments that reach the
    // tile are staged in list order, then composited.
    auto round = [&](int nslot, auto item) {
        // stage the fragments of this round that reach the tile, in list order
        float4 ra[SLOTS], rq[SLOTS], rc[SLOTS];
        bool keep[SLOTS];
        uint32_t ipos[SLOTS];
#pragma unroll
        for (int h = 0; h < SLOTS; ++h) {
            const int slot = (int)threadIdx.x + h * NT;
            keep[h] = false;
            if (slot < nslot) {
                uint32_t g;
                item(slot, ipos[h], g);
                const int64_t r = (rbase + g) * rec4;
                const float4 a = proj[r], b = proj[r + 1];
                rc[h] = proj[r + 2];
                ra[h] = make_float4(a.x, a.y, a.w, cutoff_log2(a.w));
                rq[h] = log2_conic(b);
                keep[h] = reaches_tile(ra[h], rq[h], tx0, tx0 + (float)(B - 1), ty0, ty0 + (float)(B - 1));
            }
        }
        uint32_t m[SLOTS];
#pragma unroll
        for (int h = 0; h < SLOTS; ++h) {
            m[h] = __ballot_sync(0xFFFFFFFFu, keep[h]);
            if (lane == 0) s_wcnt[h * NW + warp] = __popc(m[h]);
        }
        __syncthreads();
        int cnt = 0, off[SLOTS];
#pragma unroll
        for (int h = 0; h < SLOTS; ++h) off[h] = 0;
#pragma unroll
        for (int w = 0; w < SLOTS * NW; ++w) {
#pragma unroll
            for (int h = 0; h < SLOTS; ++h)
                if (w < h * NW + warp) off[h] += s_wcnt[w];
            cnt += s_wcnt[w];
        }
        const uint32_t ltm = (1u << lane) - 1u;
#pragma unroll
        for (int h = 0; h < SLOTS; ++h) {
            if (!keep[h]) continue;
            const int d = off[h] + __popc(m[h] & ltm);
            s_a[d] = ra[h]; s_q[d] = rq[h]; s_c[d] = rc[h]; s_pos[d] = ipos[h];
        }
        __syncthreads();
        for (int j = 0; j < cnt && nlive; ++j) {
            const float4 a = s_a[j];
            const float4 q = s_q[j];
            const float dy = a.y - fy;
            const float qb = q.y * dy;
            const float qc = q.z * dy * dy;
            const float dx0 = a.x - fx0;
            const float2 qx2 = make_float2(q.x, q.x), qb2 = make_float2(qb, qb), qc2 = make_float2(qc, qc);
            const float2 o2 = make_float2(a.z, a.z), dx02 = make_float2(dx0, dx0);
            const uint32_t pos1 = s_pos[j] + 1;
            // pairs in groups of two: one branch per group, so that the two
            // pairs' chains interleave (a pair without a valid pixel is an
            // exact no-op: alpha 0 leaves T, the colour and last unchanged)
            constexpr int GP = NP < 2 ? NP : 2;
#pragma unroll
            for (int p0 = 0; p0 < NP; p0 += GP) {
                float2 P2g[GP];
                bool v0g[GP], v1g[GP];
                bool any = false;
#pragma unroll
                for (int u = 0; u < GP; ++u) {
                    const int p = p0 + u;
                    const float2 dx = __fadd2_rn(dx02, nk[p]);
                    // the conic is positive definite, so P2 <= 0 up to rounding;
                    // the fragment counts where alpha >= 1/255
                    P2g[u] = __ffma2_rn(__ffma2_rn(qx2, dx, qb2), dx, qc2);
                    v0g[u] = P2g[u].x >= a.w;
                    v1g[u] = P2g[u].y >= a.w;
                    any = any || v0g[u] || v1g[u];
                }
                if (!any) continue;
#pragma unroll
                for (int u = 0; u < GP; ++u) {
                const int p = p0 + u;
                const int k0 = 2 * p, k1 = 2 * p + 1;
                const float2 P2 = P2g[u];
                bool v0 = v0g[u], v1 = v1g[u];
                const float2 raw = __fmul2_rn(o2, make_float2(v0 ? ex2(P2.x) : 0.f, v1 ? ex2(P2.y) : 0.f));
                float2 al = make_float2(fminf(kAlphaMax, raw.x), fminf(kAlphaMax, raw.y));
                float2 Tn = __fmul2_rn(T[p], __ffma2_rn(al, make_float2(-1.f, -1.f), make_float2(1.f, 1.f)));
                // T >= 1e-4 holds for every pixel still compositing, and a pixel
                // this fragment misses keeps its T: only a covered pixel can
                // fall below.  It stops before this fragment.
                if (Tn.x < kTMin || Tn.y < kTMin) {
                    if (Tn.x < kTMin) { al.x = 0.f; Tn.x = T[p].x; nk[p].x = kPosInf; v0 = false; --nlive; }
                    if (Tn.y < kTMin) { al.y = 0.f; Tn.y = T[p].y; nk[p].y = kPosInf; v1 = false; --nlive; }
                }
                const float4 c = s_c[j];
                const float2 w = __fmul2_rn(al, T[p]);
                Cr[p] = __ffma2_rn(w, make_float2(c.x, c.x), Cr[p]);
                Cg[p] = __ffma2_rn(w, make_float2(c.y, c.y), Cg[p]);
                Cb[p] = __ffma2_rn(w, make_float2(c.z, c.z), Cb[p]);
                T[p] = Tn;
                if (v0) last[k0] = pos1;
                if (v1) last[k1] = pos1;
                }
            }
        }
    };
    if (!COARSE) {
        const uint2 rg = ranges[gt];
        for (uint32_t start = rg.x; start < rg.y; start += BATCH) {
            if (__syncthreads_count(nlive != 0) == 0) break;
            round((int)min((uint32_t)BATCH, rg.y - start), [&](int i, uint32_t& pos, uint32_t& g) {
                pos = start + (uint32_t)i - rg.x;
                g = vals[start + (uint32_t)i];
            });
        }
    } else {
        // chunk by chunk: this thread's bitmap word of the next chunk is
        // requested while the current one is composited
        const TileChunks tc = tile_chunks(cl, vi, lt);
        const uint32_t wsel = (threadIdx.x * (kChunkItems / NT)) >> 5;
        const uint32_t* bm = cl.bitmap + (size_t)tc.k * 8 + wsel;
        uint32_t wnext = tc.c0 < tc.c1 ? bm[(size_t)tc.c0 * 512] : 0u;
        for (uint32_t c = tc.c0; c < tc.c1; ++c) {
            if (__syncthreads_count(nlive != 0) == 0) break;
            const uint32_t word = wnext;
            if (c + 1 < tc.c1) wnext = bm[(size_t)(c + 1) * 512];
            const int cnt = chunk_candidates<NT>(word, tc.item0 + (c - tc.c0) * kChunkItems, 0xFFFFFFFFu, s_cand,
                                                 s_ctot);
            bool stop = false;
            for (int w0 = 0; w0 < cnt; w0 += BATCH) {
                if (w0 > 0 && __syncthreads_count(nlive != 0) == 0) { stop = true; break; }
                round(min(BATCH, cnt - w0), [&](int i, uint32_t& pos, uint32_t& g) {
                    pos = s_cand[w0 + i];
                    g = cl.cvals[pos];
                });
            }
            if (stop) break;
        }
    }
    const int64_t HW = (int64_t)vi.width * vi.height;
    float* img = image + 3 * vi.pix_off;
#pragma unroll
    for (int k = 0; k < PX; ++k) {
        const int px = px0 + k;
        if (px >= vi.width || py >= vi.height) continue;
        const int64_t pix = (int64_t)py * vi.width + px;
        const float2 t2 = T[k >> 1], r2 = Cr[k >> 1], g2 = Cg[k >> 1], b2 = Cb[k >> 1];
        const float Tk = (k & 1) ? t2.y : t2.x;
        img[pix] = ((k & 1) ? r2.y : r2.x) + Tk * bg.x;
        img[HW + pix] = ((k & 1) ? g2.y : g2.x) + Tk * bg.y;
        img[2 * HW + pix] = ((k & 1) ? b2.y : b2.x) + Tk * bg.z;
        if (T_final) T_final[vi.pix_off + pix] = Tk;
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
// Blocks per SM the adjoint is compiled for: with 8-pixel strips (one warp
// per tile) the register budget is set so that 26 tiles fit on an SM (78
// registers; 24, 28 and 30 measured: 30 falls off a spill cliff), with
// 4-pixel strips 1024 threads.
template <int B, int TPR>
constexpr int bwd_min_blocks() { return B * TPR == 32 ? 26 : 1024 / (B * TPR); }

template <int B, int TPR, bool COARSE>
__global__ void __launch_bounds__(B * TPR, bwd_min_blocks<B, TPR>())
k_raster_bwd(const float4* __restrict__ proj, const ViewInfo* __restrict__ vt, int V, int64_t n,
             const uint32_t* __restrict__ vals, const uint2* __restrict__ ranges, CoarseLists cl, float3 bg,
             const float* __restrict__ T_final, const uint32_t* __restrict__ n_contrib,
             const float* __restrict__ dimage, float* __restrict__ grad2d, int64_t n_active, int rec4) {
    constexpr int NT = B * TPR;
    constexpr int PX = B / TPR;
    constexpr int NP = PX / 2;
    static_assert(NT % 32 == 0 && PX % 2 == 0, "whole warps, pixel pairs");
    constexpr int BATCH = NT;
    __shared__ float4 s_a[BATCH];   // u, v, opacity, log2 cut-off
    __shared__ float4 s_q[BATCH];   // base-2 conic coefficients
    __shared__ float4 s_b[BATCH];   // conic A, B, C
    __shared__ float4 s_c[BATCH];   // r, g, b
    __shared__ uint32_t s_g[BATCH];
    __shared__ uint32_t s_pos[BATCH];  // position in the tile's list
    __shared__ float s_acc[9][BATCH + 1];  // raw sums per fragment, padded: the 9 sit in different banks
    __shared__ uint32_t s_max;
    __shared__ int s_wcnt[NT / 32];
    __shared__ uint32_t s_cand[COARSE ? kChunkItems : 1];
    __shared__ int s_ctot[NT / 32];
    int64_t gt;
    int v;
    if (!block_tile(vt, V, cl, gt, v)) return;
    const ViewInfo vi = vt[v];
    const int lt = (int)(gt - vi.tile_off);
    const int row = (int)threadIdx.x / TPR;
    const int px0 = (lt % vi.tx) * B + ((int)threadIdx.x % TPR) * PX;
    const int py = (lt / vi.tx) * B + row;
    const float fy = (float)py + 0.5f;
    const float fx0 = (float)px0 + 0.5f;
    const float tx0 = (float)((lt % vi.tx) * B) + 0.5f, ty0 = (float)((lt / vi.tx) * B) + 0.5f;
    const int64_t rbase = (int64_t)v * n;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    // pixel pairs (2p, 2p + 1) in packed float2 registers.  The colour behind
    // a fragment, R, enters the gradient only as dL/dC . R (dL/dC is fixed per
    // pixel), so the walk keeps that scalar X instead of R:
    //   dL/dalpha_j = T_j (dL/dC . c_j - X_j),  X_{j-1} = X_j + alpha_j (dL/dC . c_j - X_j).
    float2 T[NP], X[NP];
    // dL/dC per pixel pair: read-only in the walk, kept in this thread's
    // column of shared memory instead of 3 NP register pairs
    __shared__ float2 s_dC[3][NP][NT];
    uint32_t last[PX];
    uint32_t mylast = 0;
    const int64_t HW = (int64_t)vi.width * vi.height;
    const float* dimg = dimage + 3 * vi.pix_off;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        float t[2] = {1.f, 1.f}, r[2] = {0.f, 0.f}, g[2] = {0.f, 0.f}, b[2] = {0.f, 0.f};
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int k = 2 * p + e;
            const int px = px0 + k;
            last[k] = 0;
            if (px < vi.width && py < vi.height) {
                const int64_t pix = (int64_t)py * vi.width + px;
                t[e] = T_final[vi.pix_off + pix];
                last[k] = n_contrib[vi.pix_off + pix];
                r[e] = dimg[pix]; g[e] = dimg[HW + pix]; b[e] = dimg[2 * HW + pix];
                mylast = max(mylast, last[k]);
            }
        }
        T[p] = make_float2(t[0], t[1]);
        s_dC[0][p][threadIdx.x] = make_float2(r[0], r[1]);
        s_dC[1][p][threadIdx.x] = make_float2(g[0], g[1]);
        s_dC[2][p][threadIdx.x] = make_float2(b[0], b[1]);
        X[p] = make_float2(r[0] * bg.x + g[0] * bg.y + b[0] * bg.z, r[1] * bg.x + g[1] * bg.y + b[1] * bg.z);
    }
    if (threadIdx.x == 0) s_max = 0;
    __syncthreads();
    if (mylast) atomicMax(&s_max, mylast);
    __syncthreads();
    const uint32_t maxl = s_max;

    // One round: list items [0, nslot) of a window (item(i, pos, g): list
    // position and Gaussian), staged in list order and walked back to front.
    auto round = [&](int nslot, auto item) {
        __syncthreads();  // the previous batch's flush is complete
        // stage the fragments of this round that reach the tile, in list order
        bool keep = false;
        uint32_t g = 0, ipos = 0;
        float4 a, b, c, aq, qq;
        if ((int)threadIdx.x < nslot) {
            item((int)threadIdx.x, ipos, g);
            const int64_t r = (rbase + g) * rec4;
            a = proj[r]; b = proj[r + 1]; c = proj[r + 2];
            aq = make_float4(a.x, a.y, a.w, cutoff_log2(a.w));
            qq = log2_conic(b);
            keep = reaches_tile(aq, qq, tx0, tx0 + (float)(B - 1), ty0, ty0 + (float)(B - 1));
        }
        const uint32_t km = __ballot_sync(0xFFFFFFFFu, keep);
        int off = 0, cnt = __popc(km);
        if (NT > 32) {
            if (lane == 0) s_wcnt[warp] = __popc(km);
            __syncthreads();
            cnt = 0;
#pragma unroll
            for (int w = 0; w < NT / 32; ++w) {
                if (w < warp) off += s_wcnt[w];
                cnt += s_wcnt[w];
            }
        }
        if (keep) {
            const int d = off + __popc(km & ((1u << lane) - 1u));
            s_a[d] = aq;
            s_q[d] = qq;
            s_b[d] = b;
            s_c[d] = c;
            s_g[d] = g;
            s_pos[d] = ipos;
#pragma unroll
            for (int q = 0; q < 9; ++q) s_acc[q][d] = 0.f;
        }
        __syncthreads();
        // one fragment over this thread's pixel pairs, accumulating the
        // pixels' dL/dP sums and colour gradients; CL: the fragment's opacity
        // can reach the alpha clamp
        auto walk = [&](auto clamp_tag, const uint32_t pos, const float4 a, const float4 q, const float4 c, float dy,
                        float2& s0, float2& s1, float2& s2, float2& g6, float2& g7, float2& g8) -> bool {
            constexpr bool CL = decltype(clamp_tag)::value;
            const float qb = q.y * dy;
            const float qc = q.z * dy * dy;
            const float dx0 = a.x - fx0;
            const float2 qx2 = make_float2(q.x, q.x), qb2 = make_float2(qb, qb), qc2 = make_float2(qc, qc);
            const float2 o2 = make_float2(a.z, a.z), m1 = make_float2(-1.f, -1.f), one = make_float2(1.f, 1.f);
            const float2 cr = make_float2(c.x, c.x), cg = make_float2(c.y, c.y), cb = make_float2(c.z, c.z);
            bool contrib = false;
            // pairs in groups of two: one branch per group, so that the two
            // pairs' chains interleave (a pair without a valid pixel is an
            // exact no-op: alpha 0 leaves T, X and every sum unchanged)
            constexpr int GP = 2;
#pragma unroll
            for (int p0 = 0; p0 < NP; p0 += GP) {
                float2 dxg[GP], P2g[GP];
                bool v0g[GP], v1g[GP];
                bool any = false;
#pragma unroll
                for (int u = 0; u < GP; ++u) {
                    const int p = p0 + u;
                    const int k0 = 2 * p, k1 = 2 * p + 1;
                    dxg[u] = make_float2(dx0 - (float)k0, dx0 - (float)k1);
                    P2g[u] = __ffma2_rn(__ffma2_rn(qx2, dxg[u], qb2), dxg[u], qc2);
                    v0g[u] = pos < last[k0] && P2g[u].x >= a.w;
                    v1g[u] = pos < last[k1] && P2g[u].y >= a.w;
                    any = any || v0g[u] || v1g[u];
                }
                if (!any) continue;
                contrib = true;
#pragma unroll
                for (int u = 0; u < GP; ++u) {
                    const int p = p0 + u;
                    const bool v0 = v0g[u], v1 = v1g[u];
                    const float2 dx = dxg[u], P2 = P2g[u];
                    const float2 raw = __fmul2_rn(o2, make_float2(v0 ? ex2(P2.x) : 0.f, v1 ? ex2(P2.y) : 0.f));
                    const float2 al = CL ? make_float2(fminf(kAlphaMax, raw.x), fminf(kAlphaMax, raw.y)) : raw;
                    const float2 om = __ffma2_rn(al, m1, one);  // 1 - alpha
                    const float2 Tj = make_float2(v0 ? T[p].x * rcp_approx(om.x) : T[p].x,
                                                  v1 ? T[p].y * rcp_approx(om.y) : T[p].y);
                    T[p] = Tj;
                    const float2 w = __fmul2_rn(al, Tj);
                    const float2 dCr = s_dC[0][p][threadIdx.x], dCg = s_dC[1][p][threadIdx.x],
                                 dCb = s_dC[2][p][threadIdx.x];
                    g6 = __ffma2_rn(w, dCr, g6);
                    g7 = __ffma2_rn(w, dCg, g7);
                    g8 = __ffma2_rn(w, dCb, g8);
                    // e = dL/dC . (c - R)
                    const float2 e = __ffma2_rn(dCb, cb, __ffma2_rn(dCg, cg, __ffma2_rn(dCr, cr, make_float2(-X[p].x, -X[p].y))));
                    const float2 dal = __fmul2_rn(Tj, e);
                    X[p] = __ffma2_rn(al, e, X[p]);
                    // dL/dP = dL/dalpha * alpha where alpha is not clamped
                    const float2 dP = CL ? __fmul2_rn(dal, make_float2(raw.x <= kAlphaMax ? raw.x : 0.f,
                                                                      raw.y <= kAlphaMax ? raw.y : 0.f))
                                         : __fmul2_rn(dal, raw);
                    const float2 t = __fmul2_rn(dP, dx);
                    s0 = __fadd2_rn(s0, dP);
                    s1 = __fadd2_rn(s1, t);
                    s2 = __ffma2_rn(t, dx, s2);
                }
            }
            return contrib;
        };
        for (int j = cnt - 1; j >= 0; --j) {
            const uint32_t pos = s_pos[j];
            if (!__any_sync(0xFFFFFFFFu, pos < mylast)) continue;
            const float4 a = s_a[j];
            const float4 q = s_q[j];
            const float4 c = s_c[j];
            const float dy = a.y - fy;
            const float2 zero = make_float2(0.f, 0.f);
            float2 s0 = zero, s1 = zero, s2 = zero, g6 = zero, g7 = zero, g8 = zero;
            // uniform over the warp: every lane reads the same fragment
            const bool contrib = a.z > kNoClampOpacity
                                     ? walk(std::true_type{}, pos, a, q, c, dy, s0, s1, s2, g6, g7, g8)
                                     : walk(std::false_type{}, pos, a, q, c, dy, s0, s1, s2, g6, g7, g8);
            // frozen Gaussians (index >= n_active) take part in the
            // recursion but need no gradient
            if (s_g[j] < n_active && __any_sync(0xFFFFFFFFu, contrib)) {
                // nine sums per fragment: S1 = sum dP dx, S2 = sum dP dy,
                // S3 = sum dP dx^2, S4 = sum dP dx dy, S5 = sum dP dy^2,
                // S0 = sum dP and the three colour sums; lane 4q ends with
                // the warp's sum q of the first eight
                const float f0 = s0.x + s0.y, f1 = s1.x + s1.y;
                const float vals8[8] = {f1, f0 * dy, s2.x + s2.y, f1 * dy, f0 * dy * dy, f0, g6.x + g6.y,
                                        g7.x + g7.y};
                const float mine = warp_sum8(vals8, lane);
                const float gb = warp_sum(g8.x + g8.y);
                if ((lane & 3) == 0) {
                    if (NT == 32) s_acc[lane >> 2][j] += mine;
                    else atomicAdd(&s_acc[lane >> 2][j], mine);
                }
                if (lane == 1) {
                    if (NT == 32) s_acc[8][j] += gb;
                    else atomicAdd(&s_acc[8][j], gb);
                }
            }
        }
        __syncthreads();
        if ((int)threadIdx.x < cnt) {
            // the conic, mean and opacity gradients from the sums:
            // dL/du = -A S1 - B S2, dL/dv = -C S2 - B S1, dL/dA = -S3 / 2,
            // dL/dB = -S4, dL/dC = -S5 / 2, dL/do = S0 / o (G = alpha / o
            // where alpha is not clamped)
            const int t = threadIdx.x;
            const float S1 = s_acc[0][t], S2 = s_acc[1][t], S3 = s_acc[2][t], S4 = s_acc[3][t];
            const float S5 = s_acc[4][t], S0 = s_acc[5][t];
            const float4 co = s_b[t];
            const float4 A = make_float4(-co.x * S1 - co.y * S2, -co.z * S2 - co.y * S1, -0.5f * S3, -S4);
            const float4 Bv = make_float4(-0.5f * S5, S0 / s_a[t].z, s_acc[6][t], s_acc[7][t]);
            const float Cv = s_acc[8][t];
            float* dst = grad2d + (rbase + s_g[t]) * kGradStride;
            if (A.x != 0.f || A.y != 0.f || A.z != 0.f || A.w != 0.f)
                atomicAdd(reinterpret_cast<float4*>(dst), A);
            if (Bv.x != 0.f || Bv.y != 0.f || Bv.z != 0.f || Bv.w != 0.f)
                atomicAdd(reinterpret_cast<float4*>(dst + 4), Bv);
            if (Cv != 0.f) atomicAdd(dst + 8, Cv);
        }
    };
    if (!COARSE) {
        const uint2 rg = ranges[gt];
        for (int64_t bend = maxl; bend > 0; bend -= BATCH) {
            const uint32_t bstart = bend > BATCH ? (uint32_t)(bend - BATCH) : 0u;
            round((int)(bend - bstart), [&](int i, uint32_t& pos, uint32_t& g) {
                pos = bstart + (uint32_t)i;
                g = vals[rg.x + bstart + (uint32_t)i];
            });
        }
    } else if (maxl > 0) {
        // chunks back to front from the one holding position maxl - 1 (the
        // last contributor of any pixel); the previous chunk's bitmap word is
        // requested while the current one is processed
        const TileChunks tc = tile_chunks(cl, vi, lt);
        const uint32_t wsel = (threadIdx.x * (kChunkItems / NT)) >> 5;
        const uint32_t* bm = cl.bitmap + (size_t)tc.k * 8 + wsel;
        if (tc.c1 > tc.c0 && maxl - 1 >= tc.item0) {
            uint32_t chi = tc.c0 + (maxl - 1 - tc.item0) / kChunkItems;
            if (chi > tc.c1 - 1) chi = tc.c1 - 1;
            uint32_t wprev = bm[(size_t)chi * 512];
            for (int64_t c = chi; c >= (int64_t)tc.c0; --c) {
                const uint32_t word = wprev;
                if (c > (int64_t)tc.c0) wprev = bm[(size_t)(c - 1) * 512];
                __syncthreads();  // s_cand of the previous chunk is no longer read
                const int cnt = chunk_candidates<NT>(word, tc.item0 + ((uint32_t)c - tc.c0) * kChunkItems, maxl,
                                                     s_cand, s_ctot);
                for (int wend = cnt; wend > 0; wend -= BATCH) {
                    const int wstart = wend > BATCH ? wend - BATCH : 0;
                    round(wend - wstart, [&](int i, uint32_t& pos, uint32_t& g) {
                        pos = s_cand[wstart + i];
                        g = cl.cvals[pos];
                    });
                }
            }
        }
    }
}

}  // namespace

void launch_render_fwd(const float* proj, const ViewInfo* vt, int V, int64_t n, int tile, int tpr,
                       const uint32_t* vals, const uint32_t* ranges, float3 bg, float* image,
                       float* T_final, uint32_t* n_contrib, int64_t total_tiles, cudaStream_t st,
                       const CoarseLists* coarse, int rec4) {
    if (total_tiles <= 0) return;
    const float4* p = reinterpret_cast<const float4*>(proj);
    const uint2* r = reinterpret_cast<const uint2*>(ranges);
    const CoarseLists cl = coarse ? *coarse : CoarseLists{};
    const unsigned nb = (unsigned)(cl.sorder ? cl.n_super << (2 * kSuperShift) : total_tiles);
#define GS_FWD(BB, TT, NTH)                                                                                        \
    (cl.citems ? k_render_fwd<BB, TT, true><<<nb, NTH, 0, st>>>(p, vt, V, n, vals, r, cl, bg, image, T_final,      \
                                                                n_contrib, rec4)                                   \
               : k_render_fwd<BB, TT, false><<<nb, NTH, 0, st>>>(p, vt, V, n, vals, r, cl, bg, image, T_final,     \
                                                                 n_contrib, rec4))
    if (tile == 8)
        GS_FWD(8, 4, 32);
    else if (tpr == 2)
        GS_FWD(16, 2, 32);
    else
        GS_FWD(16, 4, 64);
#undef GS_FWD
}

void launch_raster_bwd(const float* proj, const ViewInfo* vt, int V, int64_t n, int tile, int tpr,
                       const uint32_t* vals, const uint32_t* ranges, float3 bg, const float* T_final,
                       const uint32_t* n_contrib, const float* dimage, float* grad2d,
                       int64_t total_tiles, cudaStream_t st, int64_t n_active, const CoarseLists* coarse,
                       int rec4) {
    if (n_active < 0) n_active = n;
    cudaMemsetAsync(grad2d, 0, sizeof(float) * kGradStride * (size_t)V * (size_t)n, st);
    if (total_tiles <= 0) return;
    const float4* p = reinterpret_cast<const float4*>(proj);
    const uint2* r = reinterpret_cast<const uint2*>(ranges);
    const CoarseLists cl = coarse ? *coarse : CoarseLists{};
    const unsigned nb = (unsigned)(cl.sorder ? cl.n_super << (2 * kSuperShift) : total_tiles);
#define GS_BWD(BB, TT, NTH)                                                                                        \
    (cl.citems ? k_raster_bwd<BB, TT, true><<<nb, NTH, 0, st>>>(p, vt, V, n, vals, r, cl, bg, T_final, n_contrib,  \
                                                                dimage, grad2d, n_active, rec4)                    \
               : k_raster_bwd<BB, TT, false><<<nb, NTH, 0, st>>>(p, vt, V, n, vals, r, cl, bg, T_final, n_contrib, \
                                                                 dimage, grad2d, n_active, rec4))
    if (tile == 8)
        GS_BWD(8, 4, 32);
    else if (tpr == 2)
        GS_BWD(16, 2, 32);
    else
        GS_BWD(16, 4, 64);
#undef GS_BWD
}

}  // namespace gs
