// Tile binning and the in-house onesweep LSD radix sort.
//
// Every (view, Gaussian, touched tile) becomes one entry ordered by (view,
// tile, float32 depth, Gaussian index) -- the per-tile front-to-back order
// that compositing needs (the differentiable splatting of the cited 3DGS
// method, Sec. 3.2.3).  Instead of one 64-bit (tile | depth) key sort of all K
// entries, the order is built in two stable sorts:
//   1. a 32-bit depth sort of the V*n projected Gaussians (values v*n + g, so
//      equal depths stay in (view, index) order);
//   2. key emission in that order, then a stable sort of the K entries by
//      their ceil(log2(total tiles))-bit tile key alone.
// Stability makes the result identical to the lexicographic order while the
// K-sized sort moves 8 bytes per entry per pass over 1-2 passes instead of
// 12 bytes over 6 passes.
//
// Emission is one pass: each block gathers 1024 depth-ordered Gaussians,
// finds its output offset by decoupled look-back over the preceding blocks,
// and expands the Gaussians' tile rectangles warp by warp into consecutive,
// coalesced (key, value) writes; it also accumulates the digit histograms of
// the tile-key sort, so that sort needs no counting pass of its own.
//
// The sort is a onesweep radix sort: per digit pass a single kernel ranks a
// tile of keys in shared memory (stable warp ranking from digit-bit ballots), publishes
// its per-digit counts, resolves its global digit offsets by decoupled
// look-back over the preceding tiles, and scatters.  The last pass of the
// tile-key sort writes the values (and the keys only if asked) and records
// each tile's [start, end) range with min/max atomics at run boundaries.
// Blocks take work from atomic counters in launch order, so a waited-on tile
// always belongs to a running block; every wait is bounded (about 1 s by
// default, the context's wait limit) and reports GS_ERR_TIMEOUT.
#include <algorithm>

#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kMinTileKeys = kThreads * 8;       // smallest onesweep tile (look-back sizing)
constexpr int kMaxPasses = 4;
// Digits of the widest pass: the super-tile sort takes a key of up to 9 bits
// (at most 512 super-tiles) in one pass.  Histograms and digit offsets keep
// kMaxR words per pass.
constexpr int kWideBits = 9;
constexpr int kWideItems = 12;  // keys per thread of a 9-bit pass (static shared memory below 48 KB)
constexpr int kMaxR = 1 << kWideBits;
__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ int64_t clamp_count(const uint32_t* d_count, int64_t cap) {
    const int64_t k = (int64_t)*d_count;
    return k < cap ? k : cap;
}

// ------------------------------------------------------------ histograms
// Items are packed (key << 32 | value); digits are taken from the key.
template <int BITS>
__global__ void __launch_bounds__(kThreads)
k_hist(const uint64_t* __restrict__ items, const uint32_t* d_count, int64_t cap, int passes,
       uint32_t* __restrict__ hist, const uint32_t* __restrict__ drange) {
    constexpr int R = 1 << BITS;
    __shared__ uint32_t sh[kWarps][kMaxPasses][R];
    for (int i = threadIdx.x; i < kWarps * kMaxPasses * R; i += kThreads) (&sh[0][0][0])[i] = 0;
    __syncthreads();
    const int64_t count = clamp_count(d_count, cap);
    const int w = threadIdx.x / 32;
    const DepthXform xf = depth_xform(drange);  // the keys the depth passes order
    // eight loads of a thread in flight per round: the pass is bound by
    // memory-level parallelism, not by the shared-memory atomics
    constexpr int U = 8;
    const int64_t stride = (int64_t)gridDim.x * kThreads * U;
    for (int64_t i0 = (int64_t)blockIdx.x * kThreads * U + threadIdx.x; i0 < count; i0 += stride) {
        uint32_t k[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t i = i0 + u * kThreads;
            k[u] = i < count ? xform_key((uint32_t)(items[i] >> 32), xf) : 0u;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (i0 + u * kThreads >= count) break;
            for (int p = 0; p < passes; ++p) atomicAdd(&sh[w][p][(k[u] >> (p * BITS)) & (R - 1)], 1u);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * R; i += kThreads) {
        const int p = i / R, d = i % R;
        uint32_t s = 0;
        for (int ww = 0; ww < kWarps; ++ww) s += sh[ww][p][d];
        if (s) atomicAdd(&hist[p * kMaxR + d], s);
    }
}

// Exclusive scan of each pass's histogram in place (one block of 256
// threads, each owning PER consecutive digits).
template <int BITS>
__global__ void k_hist_scan(uint32_t* hist, int passes) {
    constexpr int R = 1 << BITS;
    constexpr int PER = (R + 255) / 256;
    __shared__ uint32_t s_w[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int p = 0; p < passes; ++p) {
        uint32_t x[PER], sum = 0;
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int d = threadIdx.x * PER + i;
            x[i] = d < R ? hist[p * kMaxR + d] : 0u;
            sum += x[i];
        }
        uint32_t incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) s_w[warp] = incl;
        __syncthreads();
        uint32_t run = incl - sum;
        for (int w = 0; w < warp; ++w) run += s_w[w];
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int d = threadIdx.x * PER + i;
            if (d < R) hist[p * kMaxR + d] = run;
            run += x[i];
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------ onesweep pass
// ITEMS packed (key << 32 | value) items per thread, 256 threads: a tile of
// 256*ITEMS.  Outputs: out (packed, for the next pass) and/or, on the last
// pass of the tile-key sort, vout (values), kout (keys, may be null) and the
// per-key [start, end) ranges.  Depth sort (drange): dmode 1, the first pass,
// replaces each key by the key it orders (xform_key), which the later passes
// then read; dmode 2, the last pass, does nothing when the keys are narrow
// (their top digit is zero: the pass would not move an item).
template <int BITS, int ITEMS>
__global__ void __launch_bounds__(kThreads, 3)
k_onesweep(const uint64_t* __restrict__ in, uint64_t* __restrict__ out, uint32_t* __restrict__ kout,
           uint32_t* __restrict__ vout, const uint32_t* d_count, int64_t cap, int shift, uint32_t kmask,
           const uint32_t* __restrict__ digit_off, unsigned long long* __restrict__ lookback,
           uint32_t* tile_counter, uint32_t* __restrict__ ranges, DevStatus* status, long long spin,
           int64_t withhold, const uint32_t* __restrict__ drange, int dmode) {
    constexpr int R = 1 << BITS;
    const DepthXform xf = depth_xform(dmode ? drange : nullptr);
    if (dmode == 2 && xf.narrow) return;  // uniform over the grid
    constexpr uint32_t MASK = R - 1;
    constexpr int TILE = kThreads * ITEMS;
    __shared__ uint64_t s_items[TILE];
    __shared__ uint32_t s_whist[kWarps][R];   // per-warp digit counts, then warp prefixes
    __shared__ uint32_t s_local[R];           // tile-local start of each digit
    __shared__ uint32_t s_gbase[R];           // global start of this tile's digit run
    __shared__ uint32_t s_tile;
    __shared__ int s_abort;

    const int64_t count = clamp_count(d_count, cap);
    const int64_t n_tiles = (count + TILE - 1) / TILE;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt = lanemask_lt();

    for (;;) {
        if (threadIdx.x == 0) { s_tile = atomicAdd(tile_counter, 1u); s_abort = 0; }
        for (int i = lane; i < R; i += 32) s_whist[warp][i] = 0;
        __syncthreads();
        const int64_t tile = s_tile;
        if (tile >= n_tiles) break;
        // test hook (gs_ctx_set_wait_test): this tile publishes nothing and
        // scatters nothing, so the look-backs of the tiles after it run out
        const bool withheld = tile == withhold;

        // ---- load (warp-striped: warp w owns a contiguous run of 32*ITEMS);
        //      missing tail items get the all-ones key
        uint64_t item[ITEMS];
        uint32_t rank[ITEMS];
        const int64_t wbase = tile * TILE + (int64_t)warp * 32 * ITEMS;
        const uint64_t* src = in + wbase + lane;
        const int64_t wrem = count - wbase - lane;  // items this lane may read: j*32 < wrem
        if (wrem > 32 * (ITEMS - 1)) {
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) item[j] = src[j * 32];
        } else {
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) item[j] = (j * 32 < wrem) ? src[j * 32] : ~0ULL;
        }
        if (dmode == 1 && xf.narrow) {
            // (missing tail items become the culled key 2^24 - 1: still the
            // last run of every digit, at staged positions >= valid)
#pragma unroll
            for (int j = 0; j < ITEMS; ++j)
                item[j] = ((uint64_t)xform_key((uint32_t)(item[j] >> 32), xf) << 32) | (uint32_t)item[j];
        }
        // ---- stable rank within the warp, item order j*32 + lane: the lanes
        //      holding the same digit are found with one ballot per digit bit;
        //      the lowest of them adds the group size to the warp's counter
        //      and shares the old value with its group
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            const uint32_t d = (((uint32_t)(item[j] >> 32) & kmask) >> shift) & MASK;
            uint32_t peers = 0xFFFFFFFFu;
#pragma unroll
            for (int bit = 0; bit < BITS; ++bit) {
                const uint32_t b = __ballot_sync(0xFFFFFFFFu, (d >> bit) & 1u);
                peers &= ((d >> bit) & 1u) ? b : ~b;
            }
            const int leader = __ffs(peers) - 1;
            uint32_t before = 0;
            if (lane == leader) before = atomicAdd(&s_whist[warp][d], (uint32_t)__popc(peers));
            before = __shfl_sync(0xFFFFFFFFu, before, leader);
            rank[j] = before + __popc(peers & lt);
        }
        __syncthreads();

        // ---- per digit (thread t owns digits t, t + 256, ...): prefix over
        //      warps, tile count, publish
        constexpr int DPT = (R + kThreads - 1) / kThreads;
        uint32_t tile_cnt[DPT];
#pragma unroll
        for (int k = 0; k < DPT; ++k) {
            const int d = (int)threadIdx.x + k * kThreads;
            tile_cnt[k] = 0;
            if (d < R) {
                uint32_t acc = 0;
                for (int w = 0; w < kWarps; ++w) { const uint32_t c = s_whist[w][d]; s_whist[w][d] = acc; acc += c; }
                tile_cnt[k] = acc;
                if (!withheld)
                    st_volatile(lookback + tile * R + d, (tile == 0 ? kFlagInc : kFlagAgg) | (unsigned long long)acc);
                s_local[d] = acc;
            }
        }
        __syncthreads();
        // tile-local digit starts: exclusive scan of the tile counts (warp 0)
        if (threadIdx.x < 32) {
            constexpr int PER = (R + 31) / 32;
            uint32_t loc[PER], sum = 0;
#pragma unroll
            for (int i = 0; i < PER; ++i) {
                const int d = threadIdx.x * PER + i;
                loc[i] = d < R ? s_local[d] : 0u;
                sum += loc[i];
            }
            uint32_t incl = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                if (threadIdx.x >= o) incl += y;
            }
            uint32_t run = incl - sum;
#pragma unroll
            for (int i = 0; i < PER; ++i) {
                const int d = threadIdx.x * PER + i;
                if (d < R) s_local[d] = run;
                run += loc[i];
            }
        }
        // ---- look back over preceding tiles, per digit (after a wait that
        //      ran out the thread's further digits are not waited for)
        bool gave_up = withheld;
#pragma unroll
        for (int k = 0; k < DPT; ++k) {
            const int d = (int)threadIdx.x + k * kThreads;
            if (d < R) {
                unsigned long long excl = 0;
                if (!gave_up && !look_back(lookback + d, tile, R, tile_cnt[k], &excl, status, spin)) gave_up = true;
                s_gbase[d] = digit_off[d] + (uint32_t)excl;
            }
        }
        if (gave_up) s_abort = 1;
        __syncthreads();
        // ---- stage in shared memory in digit order
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            const uint32_t d = (((uint32_t)(item[j] >> 32) & kmask) >> shift) & MASK;
            s_items[s_local[d] + s_whist[warp][d] + rank[j]] = item[j];
        }
        __syncthreads();
        // ---- scatter (missing tail items are all-ones: they sit at the end of
        //      the last digit's run, i.e. at staged positions >= valid)
        const int64_t rem = count - tile * TILE;
        const int valid = rem < TILE ? (int)rem : TILE;
        if (!s_abort) {
            for (int i = threadIdx.x; i < valid; i += kThreads) {
                const uint64_t it = s_items[i];
                const uint32_t k = (uint32_t)(it >> 32) & kmask;
                const uint32_t d = (k >> shift) & MASK;
                const uint32_t pos = s_gbase[d] + (uint32_t)i - s_local[d];
                if ((int64_t)pos >= count) continue;  // unreachable when the histogram matches the keys
                if (out) out[pos] = it;
                if (vout) vout[pos] = (uint32_t)it;
                if (kout) kout[pos] = k;
                if (ranges) {
                    // runs of equal keys are contiguous both here and in the output
                    if (i == 0 || ((uint32_t)(s_items[i - 1] >> 32) & kmask) != k)
                        atomicMin(&ranges[2 * (size_t)k], pos);
                    if (i == valid - 1 || ((uint32_t)(s_items[i + 1] >> 32) & kmask) != k)
                        atomicMax(&ranges[2 * (size_t)k + 1], pos + 1);
                }
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------ utilities
__global__ void k_set_u32(uint32_t* p, uint32_t v) { *p = v; }
__global__ void k_range_reset(uint32_t* drange) {
    drange[0] = 0xFFFFFFFFu;
    drange[1] = 0u;
}

// Zero `radix` u64 words per look-back tile for each of `passes` arrays, for
// the tiles that the device count implies.
__global__ void k_clear_lookback(unsigned long long* lb, const uint32_t* d_count, int64_t cap,
                                 int radix, int passes, int64_t max_tiles, int tile_keys) {
    const int64_t count = clamp_count(d_count, cap);
    const int64_t tiles = (count + tile_keys - 1) / tile_keys;
    const int64_t words = tiles * radix;
    for (int p = 0; p < passes; ++p)
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words;
             i += (int64_t)gridDim.x * blockDim.x)
            lb[(int64_t)p * max_tiles * radix + i] = 0ULL;
}

// ranges := (0xFFFFFFFF, 0) so that min/max atomics can fill them.
__global__ void k_ranges_init(uint2* r, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        r[i] = make_uint2(0xFFFFFFFFu, 0u);
}

// tiles no entry reached become the empty range (0, 0).
__global__ void k_ranges_fix(uint2* r, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint2 x = r[i];
        if (x.x == 0xFFFFFFFFu) r[i] = make_uint2(0u, 0u);
    }
}

__global__ void k_clear_u32(uint32_t* p, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = 0u;
}

// Depth-sort input from projection records: key = float32 depth bits of a
// visible (view, Gaussian), all-ones when culled; value = record index.
// The range of the visible keys goes to drange (reset before).
__global__ void k_depth_keys(const uint4* __restrict__ proj, int64_t items, const ViewInfo* __restrict__ vt, int V,
                             uint64_t* __restrict__ kv, uint2* __restrict__ rects, uint32_t* __restrict__ drange) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= items) return;
    const uint4 r3 = proj[i * 4 + 3];
    const uint32_t key = r3.z ? proj[i * 4].z : 0xFFFFFFFFu;
    kv[i] = ((uint64_t)key << 32) | (uint32_t)i;
    depth_range_add(drange, r3.z ? key : 0xFFFFFFFFu, r3.z ? key : 0u);
    if (vt[V].rect32)
        st_hint(reinterpret_cast<uint32_t*>(rects) + i, r3.z ? rect32_pack(r3.x, r3.y) : 1u, l2_policy_evict_last());
    else
        st_hint(rects + i, make_uint2(r3.x, r3.y), l2_policy_evict_last());
}

// Compaction of depth-sort items: the items with a key other than all ones
// (Gaussians some earlier stage culled for every view, e.g. by preculling),
// in order.  Blocks of kKeepBlock items: count, scan of the block sums, emit.
constexpr int kKeepBlock = 1024;

__global__ void __launch_bounds__(256)
k_keep_count(const uint64_t* __restrict__ in, int64_t items, uint32_t* __restrict__ block_sums) {
    const int64_t b0 = (int64_t)blockIdx.x * kKeepBlock;
    uint32_t mine = 0;
#pragma unroll
    for (int r = 0; r < kKeepBlock / 256; ++r) {
        const int64_t i = b0 + r * 256 + threadIdx.x;
        mine += (i < items && (uint32_t)(in[i] >> 32) != 0xFFFFFFFFu) ? 1u : 0u;
    }
    __shared__ uint32_t s_w[8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xFFFFFFFFu, mine, o);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = mine;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < 8; ++w) t += s_w[w];
        block_sums[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(256)
k_keep_emit(const uint64_t* __restrict__ in, int64_t items, const uint32_t* __restrict__ block_off,
            uint64_t* __restrict__ out) {
    __shared__ uint32_t s_w[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t base = block_off[blockIdx.x];
    const int64_t b0 = (int64_t)blockIdx.x * kKeepBlock;
#pragma unroll
    for (int r = 0; r < kKeepBlock / 256; ++r) {
        const int64_t i = b0 + r * 256 + threadIdx.x;
        uint64_t it = 0;
        bool keep = false;
        if (i < items) {
            it = in[i];
            keep = (uint32_t)(it >> 32) != 0xFFFFFFFFu;
        }
        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, keep);
        if (lane == 0) s_w[warp] = __popc(bal);
        __syncthreads();
        uint32_t off = base;
        uint32_t tot = 0;
        for (int w = 0; w < 8; ++w) {
            if (w < warp) off += s_w[w];
            tot += s_w[w];
        }
        if (keep) out[off + __popc(bal & lanemask_lt())] = it;
        base += tot;
        __syncthreads();
    }
}

// ------------------------------------------------------------ emission
// Two-level entries carry their tile rectangle within the super-tile (local
// x0, x1 - 1, y0, y1 - 1, 3 bits each) in bits 52..63, above keys of up to
// 20 bits; sorts of such entries mask the key.
constexpr int kRectShift = 52;
constexpr int kMaxCoarseKeyBits = kRectShift - 32;
constexpr int kEmitThreads = 256;
constexpr int kEmitWarps = kEmitThreads / 32;
constexpr int kEmitRounds = 4;
constexpr int kEmitBlock = kEmitThreads * kEmitRounds;  // depth-ordered Gaussians per block

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// Item index within a block: warp w, round r, lane l -> w*128 + r*32 + l, so
// the 32 items of one (warp, round) are consecutive and their outputs form
// one contiguous range.  Each item's state (Gaussian, view, tile rectangle
// and the reciprocal of its key rectangle's width) waits in shared memory
// between the count and the expansion, where every output reads its owner's
// state from there; in registers the four rounds' state spilled to memory at
// the 32 registers that 8 blocks an SM allow.
// Compiled for 8 blocks an SM: the kernel waits on its gathers and barriers,
// and more resident blocks hide that better than fewer at 64 registers.
template <int BITS>
__global__ void __launch_bounds__(kEmitThreads, 8)
k_emit(const uint64_t* __restrict__ dsorted, const uint64_t* __restrict__ dsorted_narrow,
       const uint32_t* __restrict__ drange, int64_t total, int64_t n, const uint2* __restrict__ rects,
       const ViewInfo* __restrict__ vt, int64_t cap, uint64_t* __restrict__ kv,
       unsigned long long* __restrict__ lookback, uint32_t* block_counter, uint32_t* d_num_keys,
       int passes, uint32_t* __restrict__ hist, int sshift, unsigned long long* fine_total, uint32_t key_bound,
       const uint32_t* d_total, DevStatus* status, int V, long long spin) {
    constexpr int R = 1 << BITS;
    constexpr int HP = BITS > 8 ? 1 : kMaxPasses;  // a wide digit is a single pass
    __shared__ uint32_t s_hist[HP][R];
    __shared__ uint4 s_item[kEmitBlock];   // Gaussian, view, tile rectangle lo, hi
    __shared__ float s_rw[kEmitBlock];     // 1 / width of the key rectangle
    __shared__ int s_mark[kEmitWarps][32];
    __shared__ uint32_t s_wtot[kEmitWarps];
    __shared__ uint32_t s_blk;
    __shared__ unsigned long long s_excl;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool rect32 = vt[V].rect32 != 0;
    // narrow depth keys: the depth sort skipped its last pass and ended in
    // the other buffer
    if (depth_xform(drange).narrow) dsorted = dsorted_narrow;
    for (int i = threadIdx.x; i < HP * R; i += kEmitThreads) (&s_hist[0][0])[i] = 0;
    if (threadIdx.x == 0) s_blk = atomicAdd(block_counter, 1u);
    __syncthreads();
    const int64_t b = s_blk;
    const int64_t nblk = (total + kEmitBlock - 1) / kEmitBlock;
    // after a compaction only the first *d_total items are filled (the grid
    // still covers `total`; blocks past them publish empty counts)
    if (d_total && (int64_t)*d_total < total) total = (int64_t)*d_total;

    // the key rectangle of an item (the super-tile rectangle covering its
    // tile rectangle with two-level binning) and its entry count
    auto key_rect = [&](uint32_t flo, uint32_t fhi, uint32_t& lo, uint32_t& hi) -> uint32_t {
        const uint32_t rw = (fhi & 0xFFFFu) - (flo & 0xFFFFu), rh = (fhi >> 16) - (flo >> 16);
        lo = flo;
        hi = fhi;
        if (!sshift || rw * rh == 0) return rw * rh;
        const uint32_t sx0 = (flo & 0xFFFFu) >> sshift, sy0 = (flo >> 16) >> sshift;
        const uint32_t sx1 = (((fhi & 0xFFFFu) - 1u) >> sshift) + 1u;
        const uint32_t sy1 = (((fhi >> 16) - 1u) >> sshift) + 1u;
        lo = sx0 | (sy0 << 16);
        hi = sx1 | (sy1 << 16);
        return (sx1 - sx0) * (sy1 - sy0);
    };

    uint32_t incl[kEmitRounds];
    uint32_t wtot = 0;
    unsigned long long fine = 0;
#pragma unroll
    for (int r = 0; r < kEmitRounds; ++r) {
        const int slot = warp * (32 * kEmitRounds) + r * 32 + lane;
        const int64_t idx = b * kEmitBlock + slot;
        uint4 it = make_uint4(0u, 0u, 0u, 0u);
        uint32_t cnt = 0;
        float rw = 0.f;
        if (idx < total) {
            const uint32_t rr = (uint32_t)dsorted[idx];
            // the record's tile rectangle, left in L2 by the projection (its
            // last use: demoted for eviction)
            const uint2 rc = rect32 ? rect32_unpack(ld_hint(reinterpret_cast<const uint32_t*>(rects) + rr,
                                                            l2_policy_evict_first()))
                                    : ld_hint(rects + rr, l2_policy_evict_first());
            const uint32_t v = (uint32_t)(rr / (uint64_t)n);
            fine += ((rc.y & 0xFFFFu) - (rc.x & 0xFFFFu)) * ((rc.y >> 16) - (rc.x >> 16));
            uint32_t lo, hi;
            cnt = key_rect(rc.x, rc.y, lo, hi);
            const uint32_t w0 = (hi & 0xFFFFu) - (lo & 0xFFFFu);
            rw = w0 ? 1.0f / (float)w0 : 0.f;
            it = make_uint4(rr - v * (uint32_t)n, v, rc.x, rc.y);
        }
        s_item[slot] = it;
        s_rw[slot] = rw;
        incl[r] = warp_incl_scan(cnt, lane);
        wtot += __shfl_sync(0xFFFFFFFFu, incl[r], 31);
    }
    if (lane == 0) s_wtot[warp] = wtot;
    if (fine_total) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) fine += __shfl_xor_sync(0xFFFFFFFFu, fine, o);
        if (lane == 0 && fine) atomicAdd(fine_total, fine);
    }
    __syncthreads();
    uint32_t wexcl = 0, btot = 0;
    for (int w = 0; w < kEmitWarps; ++w) {
        if (w < warp) wexcl += s_wtot[w];
        btot += s_wtot[w];
    }
    if (threadIdx.x == 0) {
        st_volatile(lookback + b, (b == 0 ? kFlagInc : kFlagAgg) | (unsigned long long)btot);
        unsigned long long excl = 0;
        look_back(lookback, b, 1, btot, &excl, status, spin);
        s_excl = excl;
        if (b == nblk - 1) {
            const unsigned long long K = excl + btot;
            *d_num_keys = (uint32_t)(K > 0xFFFFFFFFull ? 0xFFFFFFFFull : K);
            // two-level: the fine total decides capacity (k_fine_total)
            if (!fine_total && (long long)K > cap) record_status(status, GS_ERR_CAPACITY, (long long)K);
        }
    }
    __syncthreads();

    // ---- expansion: 32 consecutive outputs per warp step, coalesced
    uint64_t base = s_excl + wexcl;
#pragma unroll
    for (int r = 0; r < kEmitRounds; ++r) {
        const int row = warp * (32 * kEmitRounds) + r * 32;  // this (warp, round)'s items
        const uint32_t rtot = __shfl_sync(0xFFFFFFFFu, incl[r], 31);
        uint32_t mlo, mhi;
        const uint4 mine = s_item[row + lane];
        const uint32_t cnt = key_rect(mine.z, mine.w, mlo, mhi);
        const uint32_t off = incl[r] - cnt;
        int carry = -1;
        for (uint32_t c = 0; c < rtot; c += 32) {
            s_mark[warp][lane] = -1;
            __syncwarp();
            if (cnt > 0 && off >= c && off < c + 32) s_mark[warp][off - c] = lane;
            __syncwarp();
            int m = s_mark[warp][lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xFFFFFFFFu, m, o);
                if (lane >= o) m = max(m, y);
            }
            m = max(m, carry);
            carry = __shfl_sync(0xFFFFFFFFu, m, 31);
            const int owner = m < 0 ? 0 : m;
            const uint32_t o_off = __shfl_sync(0xFFFFFFFFu, off, owner);
            const uint32_t o = c + lane;
            // only entries that fit the capacity are stored and counted, so the
            // sort's digit offsets always describe exactly the stored prefix
            const bool stored = o < rtot && base + o < (uint64_t)cap;
            uint32_t key = 0;
            if (stored) {
                const uint4 ow = s_item[row + owner];
                const float o_rw = s_rw[row + owner];
                uint32_t o_lo, o_hi;
                key_rect(ow.z, ow.w, o_lo, o_hi);
                const ViewInfo& vi = vt[ow.y];
                const uint32_t o_kb = (uint32_t)(sshift ? vi.stile_off : vi.tile_off);
                const uint32_t o_tx = (uint32_t)(sshift ? vi.stx : vi.tx);
                const uint32_t o_w = (o_hi & 0xFFFFu) - (o_lo & 0xFFFFu);
                const uint32_t j = o - o_off;
                // j / w exactly: j < 2^16 and w < 2^16, so (j + 0.5) / w stays
                // more than 0.5 / w away from an integer
                const uint32_t ty = (uint32_t)(((float)j + 0.5f) * o_rw);
                const uint32_t txx = j - ty * o_w;
                key = o_kb + ((o_lo >> 16) + ty) * o_tx + (o_lo & 0xFFFFu) + txx;
                // a view table larger than the caller's tile count (reported
                // by k_view_table) must not index past the ranges arrays
                if (key >= key_bound) key = key_bound - 1u;
                uint64_t extra = 0;
                if (sshift) {
                    // the tile rectangle clipped to this super-tile, in its
                    // local tile coordinates, above the key bits
                    const int ox = (int)(((o_lo & 0xFFFFu) + txx) << sshift);
                    const int oy = (int)(((o_lo >> 16) + ty) << sshift);
                    const int S = 1 << sshift;
                    const int x0 = max((int)(ow.z & 0xFFFFu) - ox, 0), x1 = min((int)(ow.w & 0xFFFFu) - ox, S);
                    const int y0 = max((int)(ow.z >> 16) - oy, 0), y1 = min((int)(ow.w >> 16) - oy, S);
                    extra = (uint64_t)((uint32_t)x0 | ((uint32_t)(x1 - 1) << 3) | ((uint32_t)y0 << 6) |
                                       ((uint32_t)(y1 - 1) << 9)) << kRectShift;
                }
                kv[base + o] = extra | ((uint64_t)key << 32) | ow.x;
            }
            const uint32_t act = __ballot_sync(0xFFFFFFFFu, stored);
            if (stored) {
                atomicAdd(&s_hist[0][key & (R - 1)], 1u);
                for (int p = 1; p < passes && p < HP; ++p) {
                    const uint32_t d = (key >> (p * BITS)) & (R - 1);
                    const uint32_t peers = __match_any_sync(act, d);
                    if (lane == __ffs(peers) - 1) atomicAdd(&s_hist[p][d], __popc(peers));
                }
            }
        }
        base += rtot;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * R && i < HP * R; i += kEmitThreads) {
        const uint32_t c = (&s_hist[0][0])[i];
        if (c) atomicAdd(&hist[(i / R) * kMaxR + (i % R)], c);
    }
}

// ------------------------------------------------------------ two-level binning
// Coarse entries (super-tile, Gaussian) are emitted in depth order and sorted
// stably by super-tile; each super-tile's depth-ordered list is then cut into
// chunks of kFineChunk entries and expanded into its kSuper x kSuper tiles'
// lists (one warp per chunk).  Per chunk, k_fine_count counts the entries of
// every tile; the counts are scanned over the chunks of a super-tile
// (k_fine_prefix) and over all tiles (k_tile_scan, which also writes the
// ranges); k_fine_write then
// writes each chunk's entries at its offsets, in chunk order and, within a
// chunk, in list order -- the stable (tile, depth, index) order.
constexpr int kFineThreads = 256;
constexpr int kFineChunk = kChunkItems;

// Fine total from the rectangles: number of stored entries, capacity check.
__global__ void k_fine_total(const unsigned long long* fine_total, int64_t cap, uint32_t* d_num_keys,
                             DevStatus* status) {
    const unsigned long long K = *fine_total;
    *d_num_keys = (uint32_t)(K > 0xFFFFFFFFull ? 0xFFFFFFFFull : K);
    if ((long long)K > cap) record_status(status, GS_ERR_CAPACITY, (long long)K);
}

__device__ __forceinline__ int find_super_view(const ViewInfo* __restrict__ vt, int V, int64_t s) {
    int lo = 0, hi = V - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (vt[mid].stile_off <= s) lo = mid; else hi = mid - 1;
    }
    return lo;
}

constexpr int kOrderMax = 2048;  // super-tiles the raster order ranks (above: identity order)

// Chunk table (one block): chunk_first[s] = first chunk of super-tile s,
// *d_n_chunks = total (clamped); k_chunk_owner then fills chunk_meta.  With
// `order` (n_order words): the raster order, super-tiles by decreasing list
// length, ties by index (each one's rank by counting); the identity order
// when the view table's count is not n_order or exceeds kOrderMax.
__global__ void __launch_bounds__(1024)
k_fine_chunks(const uint2* __restrict__ cranges, const ViewInfo* __restrict__ vt, int V, int64_t ns_bound,
              uint32_t* __restrict__ chunk_first, uint32_t* d_n_chunks, int64_t max_chunks, DevStatus* status,
              uint32_t* __restrict__ order, int n_order) {
    __shared__ uint32_t s_part[1024];
    __shared__ unsigned long long s_key[kOrderMax];
    if (order) {
        if (n_order > kOrderMax || vt[V].stile_off != (int64_t)n_order) {
            for (int i = threadIdx.x; i < n_order; i += blockDim.x) order[i] = (uint32_t)i;
        } else {
            for (int i = threadIdx.x; i < n_order; i += blockDim.x) {
                const uint2 r = cranges[i];
                s_key[i] = ((unsigned long long)(~(r.y - r.x)) << 32) | (uint32_t)i;
            }
            __syncthreads();
            for (int i = threadIdx.x; i < n_order; i += blockDim.x) {
                const unsigned long long k = s_key[i];
                int rank = 0;
                for (int j = 0; j < n_order; ++j) rank += s_key[j] < k;
                order[rank] = (uint32_t)i;
            }
        }
    }
    const int64_t ns = vt[V].stile_off < ns_bound ? vt[V].stile_off : ns_bound;
    const int64_t per = (ns + blockDim.x - 1) / blockDim.x;
    const int64_t a = (int64_t)threadIdx.x * per;
    const int64_t e = a + per < ns ? a + per : ns;
    uint32_t sum = 0;
    for (int64_t s = a; s < e; ++s) {
        const uint2 r = cranges[s];
        sum += (r.y > r.x ? r.y - r.x + kFineChunk - 1 : 0u) / kFineChunk;
    }
    s_part[threadIdx.x] = sum;
    __syncthreads();
    for (int o = 1; o < (int)blockDim.x; o <<= 1) {
        const uint32_t y = threadIdx.x >= (unsigned)o ? s_part[threadIdx.x - o] : 0u;
        __syncthreads();
        s_part[threadIdx.x] += y;
        __syncthreads();
    }
    uint32_t run = s_part[threadIdx.x] - sum;
    for (int64_t s = a; s < e; ++s) {
        const uint2 r = cranges[s];
        const uint32_t nc = (r.y > r.x ? r.y - r.x + kFineChunk - 1 : 0u) / kFineChunk;
        chunk_first[s] = run;
        run += nc;
    }
    if (threadIdx.x == blockDim.x - 1) {
        chunk_first[ns] = s_part[threadIdx.x];
        const uint32_t tot = s_part[threadIdx.x];
        *d_n_chunks = (int64_t)tot < max_chunks ? tot : (uint32_t)max_chunks;
        // more chunks than their tables hold: the caller's key capacity
        // (keys_cap / 256 chunks) is too small for them
        if ((int64_t)tot > max_chunks) record_status(status, GS_ERR_CAPACITY, (long long)tot * kFineChunk);
    }
}

// chunk_meta[c] := (first coarse entry, end entry, super-tile, view) of
// chunk c, one warp per super-tile (coalesced runs; chunks past the table
// are dropped, as k_fine_chunks reports), so that the passes over chunks
// find a chunk's geometry with one load.
__global__ void __launch_bounds__(256)
k_chunk_owner(const uint32_t* __restrict__ chunk_first, const uint2* __restrict__ cranges,
              const ViewInfo* __restrict__ vt, int V, int64_t ns_bound, uint4* __restrict__ chunk_meta,
              int64_t max_chunks) {
    const int64_t ns = vt[V].stile_off < ns_bound ? vt[V].stile_off : ns_bound;
    const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (s >= ns) return;
    const int64_t c0 = chunk_first[s];
    const int64_t c1 = min((int64_t)chunk_first[s + 1], max_chunks);
    const uint2 cr = cranges[s];
    const uint32_t v = (uint32_t)find_super_view(vt, V, s);
    for (int64_t c = c0 + (threadIdx.x & 31); c < c1; c += 32) {
        const uint32_t a = cr.x + (uint32_t)(c - c0) * (uint32_t)kFineChunk;
        chunk_meta[c] = make_uint4(a, min(cr.y, a + (uint32_t)kFineChunk), (uint32_t)s, v);
    }
}

// 32 x 32 bit-matrix transpose across a warp: on return bit j of lane k's
// word is bit k of lane j's input word (recursive block swaps, 5 rounds).
__device__ __forceinline__ uint32_t transpose32(uint32_t x, int lane) {
    const uint32_t masks[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int r = 0; r < 5; ++r) {
        const int sh = 16 >> r;
        const uint32_t m = masks[r];
        const uint32_t y = __shfl_xor_sync(0xFFFFFFFFu, x, sh);
        x = (lane & sh) ? ((x & ~m) | ((y & ~m) >> sh)) : ((x & m) | ((y & m) << sh));
    }
    return x;
}

// Chunk geometry shared by the count and write passes.
struct FineChunk {
    uint32_t a, e;          // coarse entries [a, e)
    int v, ox, oy;          // view, tile origin of the super-tile
    uint32_t t0, t1;        // this lane's tiles (k = lane, k = lane + 32)
    bool in0, in1;
    uint64_t valid;         // tiles of the super-tile inside the view
};

__device__ __forceinline__ FineChunk fine_chunk(uint32_t c, const uint4* __restrict__ chunk_meta,
                                                const ViewInfo* __restrict__ vt, int64_t total_tiles, int lane) {
    FineChunk f;
    const uint4 m = chunk_meta[c];
    f.a = m.x;
    f.e = m.y;
    const uint32_t s = m.z;
    f.v = (int)m.w;
    const ViewInfo vi = vt[f.v];
    const int ls = (int)(s - vi.stile_off);
    f.ox = (ls % vi.stx) << kSuperShift;
    f.oy = (ls / vi.stx) << kSuperShift;
    const int x = f.ox + (lane & (kSuper - 1));
    const int y0 = f.oy + (lane >> kSuperShift), y1 = y0 + 4;
    const int64_t tt0 = vi.tile_off + (int64_t)y0 * vi.tx + x, tt1 = vi.tile_off + (int64_t)y1 * vi.tx + x;
    f.in0 = x < vi.tx && y0 < vi.ty && tt0 < total_tiles;
    f.in1 = x < vi.tx && y1 < vi.ty && tt1 < total_tiles;
    f.t0 = f.in0 ? (uint32_t)tt0 : 0u;
    f.t1 = f.in1 ? (uint32_t)tt1 : 0u;
    f.valid = (uint64_t)__ballot_sync(0xFFFFFFFFu, f.in0) | ((uint64_t)__ballot_sync(0xFFFFFFFFu, f.in1) << 32);
    return f;
}

// Mask of the tiles (bit 8 * y + x) inside a packed local rectangle.
__device__ __forceinline__ uint64_t rect12_mask(uint32_t r) {
    const uint32_t x0 = r & 7u, x1 = ((r >> 3) & 7u) + 1u, y0 = (r >> 6) & 7u, y1 = ((r >> 9) & 7u) + 1u;
    const uint64_t row = (uint64_t)(((1u << x1) - 1u) & ~((1u << x0) - 1u)) * 0x0101010101010101ULL;
    const uint64_t below = y1 >= 8u ? ~0ULL : ((1ULL << (8u * y1)) - 1ULL);
    return row & below & ~((1ULL << (8u * y0)) - 1ULL);
}

// Group `grp` of a chunk: lane's entry value and its super-tile tile mask,
// transposed so that lane l holds the group's entries covering tile l (c0)
// and tile l + 32 (c1), bit j = group entry j.
__device__ __forceinline__ void fine_group(const FineChunk& f, uint32_t grp, const uint64_t* __restrict__ citems,
                                           int lane, uint32_t& gval, uint32_t& c0, uint32_t& c1) {
    const uint32_t i = f.a + grp * 32u + (uint32_t)lane;
    uint64_t m = 0;
    gval = 0;
    if (i < f.e) {
        const uint64_t it = citems[i];
        gval = (uint32_t)it;
        m = rect12_mask((uint32_t)(it >> kRectShift)) & f.valid;
    }
    c0 = transpose32((uint32_t)m, lane);
    c1 = transpose32((uint32_t)(m >> 32), lane);
}

// Count pass, one warp per chunk: chunk_off[c][k] := entries of chunk c in
// tile k of its super-tile.
__global__ void __launch_bounds__(kFineThreads)
k_fine_count(const uint64_t* __restrict__ citems, const uint2* __restrict__ cranges,
             const uint32_t* __restrict__ chunk_first, const uint4* __restrict__ chunk_meta,
             const uint32_t* __restrict__ d_n_chunks, const ViewInfo* __restrict__ vt, int V,
             int64_t total_tiles, uint32_t* __restrict__ chunk_off) {
    const int lane = threadIdx.x & 31;
    const uint32_t nchunks = *d_n_chunks;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < nchunks; c += nw) {
        const FineChunk f = fine_chunk(c, chunk_meta, vt, total_tiles, lane);
        uint32_t n0 = 0, n1 = 0;
        for (uint32_t grp = 0; f.a + grp * 32u < f.e; ++grp) {
            uint32_t gval, c0, c1;
            fine_group(f, grp, citems, lane, gval, c0, c1);
            n0 += __popc(c0);
            n1 += __popc(c1);
        }
        chunk_off[(size_t)c * 64 + lane] = n0;
        chunk_off[(size_t)c * 64 + 32 + lane] = n1;
    }
}

// Bitmap pass, one warp per chunk: the transposed column words of the
// chunk's groups, stored as bitmap[c][k][group] (two 32-byte rows a lane).
__global__ void __launch_bounds__(kFineThreads)
k_fine_mask(const uint64_t* __restrict__ citems, const uint2* __restrict__ cranges,
            const uint32_t* __restrict__ chunk_first, const uint4* __restrict__ chunk_meta,
            const uint32_t* __restrict__ d_n_chunks, const ViewInfo* __restrict__ vt, int V,
            int64_t total_tiles, uint32_t* __restrict__ bitmap) {
    const int lane = threadIdx.x & 31;
    const uint32_t nchunks = *d_n_chunks;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < nchunks; c += nw) {
        const FineChunk f = fine_chunk(c, chunk_meta, vt, total_tiles, lane);
        // the chunk's 8 items of this lane requested together, then decoded
        uint32_t rect[8];
#pragma unroll
        for (int grp = 0; grp < 8; ++grp) {
            const uint32_t i = f.a + (uint32_t)grp * 32u + (uint32_t)lane;
            rect[grp] = i < f.e ? (uint32_t)(citems[i] >> kRectShift) : 0xFFFFFFFFu;
        }
        uint32_t w0[8], w1[8];
#pragma unroll
        for (int grp = 0; grp < 8; ++grp) {
            const uint64_t m = rect[grp] == 0xFFFFFFFFu ? 0ull : rect12_mask(rect[grp]) & f.valid;
            w0[grp] = transpose32((uint32_t)m, lane);
            w1[grp] = transpose32((uint32_t)(m >> 32), lane);
        }
        uint4* out = reinterpret_cast<uint4*>(bitmap) + (size_t)c * 128;
        out[2 * lane] = make_uint4(w0[0], w0[1], w0[2], w0[3]);
        out[2 * lane + 1] = make_uint4(w0[4], w0[5], w0[6], w0[7]);
        out[64 + 2 * lane] = make_uint4(w1[0], w1[1], w1[2], w1[3]);
        out[64 + 2 * lane + 1] = make_uint4(w1[4], w1[5], w1[6], w1[7]);
    }
}

// Write pass, one block per chunk.  Warp w transposes group w (entries
// 32w .. 32w + 31 of the chunk) into shared memory: col[w][k] holds, bit j,
// whether entry 32w + j covers tile k.  Warp w then builds the runs of tiles
// k = w, w + 8, ..., w + 56: per tile, group by group, each lane whose entry
// is in the column writes it at run position + (set bits below it) into the
// warp's staging area, and the finished run (at most kFineChunk entries) is
// copied to the output with consecutive stores.
constexpr int kFineGroups = kFineChunk / 32;
constexpr int kFineWarps = kFineThreads / 32;
constexpr int kFineStage = kFineChunk;
static_assert(kFineWarps == kFineGroups, "one warp per group of the chunk");

template <bool KOUT>
__global__ void __launch_bounds__(kFineThreads)
k_fine_write(const uint64_t* __restrict__ citems, const uint2* __restrict__ cranges,
             const uint32_t* __restrict__ chunk_first, const uint4* __restrict__ chunk_meta,
             const uint32_t* __restrict__ d_n_chunks, const ViewInfo* __restrict__ vt, int V,
             int64_t total_tiles, const uint32_t* __restrict__ chunk_off,
             const uint2* __restrict__ ranges, int64_t cap, uint32_t* __restrict__ vout,
             uint32_t* __restrict__ kout) {
    __shared__ uint32_t s_col[kFineGroups][64];
    __shared__ uint32_t s_gv[kFineGroups][33];
    __shared__ uint32_t s_base[64], s_tile[64];
    __shared__ uint32_t s_stage[kFineWarps][4 * kFineStage];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t* stage = s_stage[warp];
    const uint32_t nchunks = *d_n_chunks;
    const uint32_t cap32 = cap < 0xFFFFFFFFll ? (uint32_t)cap : 0xFFFFFFFFu;  // keys_cap < 2^32
    for (uint32_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const FineChunk f = fine_chunk(c, chunk_meta, vt, total_tiles, lane);
        if (warp == 0) {
            s_base[lane] = f.in0 ? ranges[f.t0].x + chunk_off[(size_t)c * 64 + lane] : 0u;
            s_base[lane + 32] = f.in1 ? ranges[f.t1].x + chunk_off[(size_t)c * 64 + 32 + lane] : 0u;
            s_tile[lane] = f.t0;
            s_tile[lane + 32] = f.t1;
        }
        uint32_t gval = 0, c0 = 0, c1 = 0;
        if (f.a + (uint32_t)warp * 32u < f.e) fine_group(f, (uint32_t)warp, citems, lane, gval, c0, c1);
        s_col[warp][lane] = c0;
        s_col[warp][lane + 32] = c1;
        s_gv[warp][lane] = gval;
        __syncthreads();
        // Each warp writes 8 of the 64 tiles, 4 per round.  Lane (q, g) owns
        // the column word of tile q and group g: the 8 lanes of a tile scan
        // their counts for offsets, then each lane stages the entries of its
        // set bits in order, and the warp stores the 4 runs contiguously.
        const int q = lane >> 3, g = lane & 7;
#pragma unroll
        for (int rho = 0; rho < 2; ++rho) {
            const int k = warp * 8 + rho * 4 + q;
            uint32_t w = s_col[g][k];
            const uint32_t cw = __popc(w);
            uint32_t incl = cw;
#pragma unroll
            for (int o = 1; o < 8; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                if (g >= o) incl += y;
            }
            uint32_t off = incl - cw;
            const uint32_t tot = __shfl_sync(0xFFFFFFFFu, incl, lane | 7);
            uint32_t* st = stage + q * kFineStage;
            while (w) {
                const int b = __ffs(w) - 1;
                w &= w - 1u;
                st[off++] = s_gv[g][b];
            }
            __syncwarp();
            // the four runs as one sequence: item i of it is entry i - e_qq
            // of run qq, e_qq the runs' exclusive prefix
            const uint32_t e1 = __shfl_sync(0xFFFFFFFFu, tot, 0);
            const uint32_t e2 = e1 + __shfl_sync(0xFFFFFFFFu, tot, 8);
            const uint32_t e3 = e2 + __shfl_sync(0xFFFFFFFFu, tot, 16);
            const uint32_t all = e3 + __shfl_sync(0xFFFFFFFFu, tot, 24);
            const int k0 = warp * 8 + rho * 4;
            for (uint32_t i = (uint32_t)lane; i < all; i += 32) {
                const int qq = (int)(i >= e1) + (int)(i >= e2) + (int)(i >= e3);
                const uint32_t idx = i - (qq == 0 ? 0u : qq == 1 ? e1 : qq == 2 ? e2 : e3);
                const uint32_t o = s_base[k0 + qq] + idx;
                if (o < cap32) {
                    vout[o] = stage[qq * kFineStage + idx];
                    if (KOUT) kout[o] = s_tile[k0 + qq];
                }
            }
            __syncwarp();
        }
        __syncthreads();
    }
}

template <bool KOUT>
unsigned fine_write_grid(int sm_count) {
    static int per_sm = 0;
    if (per_sm == 0 &&
        (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fine_write<KOUT>, kFineThreads, 0) != cudaSuccess ||
         per_sm < 1))
        per_sm = 1;
    return (unsigned)(sm_count * per_sm);
}

// Per (super-tile, tile): exclusive prefix of the chunk counts in place, and
// the tile's total.
__global__ void k_fine_prefix(const uint32_t* __restrict__ chunk_first, const uint32_t* __restrict__ d_n_chunks,
                              const ViewInfo* __restrict__ vt, int V, int64_t total_tiles,
                              uint32_t* __restrict__ chunk_off, uint32_t* __restrict__ tile_count) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t ns = vt[V].stile_off < total_tiles ? vt[V].stile_off : total_tiles;
    if (idx >= ns * 64) return;
    const int64_t s = idx >> 6;
    const int k = (int)(idx & 63);
    const uint32_t nch = *d_n_chunks;
    const uint32_t c0 = chunk_first[s];
    const uint32_t c1 = min(chunk_first[s + 1], nch);
    uint32_t run = 0;
    uint32_t c = c0;
    for (; c + 8 <= c1; c += 8) {  // eight loads in flight
        uint32_t x[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) x[q] = chunk_off[(size_t)(c + q) * 64 + k];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            chunk_off[(size_t)(c + q) * 64 + k] = run;
            run += x[q];
        }
    }
    for (; c < c1; ++c) {
        const uint32_t x = chunk_off[(size_t)c * 64 + k];
        chunk_off[(size_t)c * 64 + k] = run;
        run += x;
    }
    const int v = find_super_view(vt, V, s);
    const ViewInfo vi = vt[v];
    const int ls = (int)(s - vi.stile_off);
    const int x = ((ls % vi.stx) << kSuperShift) + (k & (kSuper - 1));
    const int y = ((ls / vi.stx) << kSuperShift) + (k >> kSuperShift);
    const int64_t t = vi.tile_off + (int64_t)y * vi.tx + x;
    if (x < vi.tx && y < vi.ty && t < total_tiles) tile_count[t] = run;
}

// Exclusive scan of the tile counts (one block) into the ranges; empty
// tiles get (0, 0).  Ranges are clamped to the capacity: after an overflow
// (reported by k_fine_total) compositing reads only stored entries.
__global__ void __launch_bounds__(1024)
k_tile_scan(const uint32_t* __restrict__ tile_count, int64_t total_tiles, int64_t cap,
            uint2* __restrict__ ranges) {
    __shared__ unsigned long long s_part[1024];
    const int64_t per = (total_tiles + blockDim.x - 1) / blockDim.x;
    const int64_t a = (int64_t)threadIdx.x * per;
    const int64_t e = a + per < total_tiles ? a + per : total_tiles;
    unsigned long long sum = 0;
    for (int64_t t = a; t < e; ++t) sum += tile_count[t];
    s_part[threadIdx.x] = sum;
    __syncthreads();
    for (int o = 1; o < (int)blockDim.x; o <<= 1) {
        const unsigned long long y = threadIdx.x >= (unsigned)o ? s_part[threadIdx.x - o] : 0ULL;
        __syncthreads();
        s_part[threadIdx.x] += y;
        __syncthreads();
    }
    unsigned long long run = s_part[threadIdx.x] - sum;
    for (int64_t t = a; t < e; ++t) {
        const uint32_t k = tile_count[t];
        const uint32_t st = (uint32_t)min(run, (unsigned long long)cap);
        const uint32_t en = (uint32_t)min(run + k, (unsigned long long)cap);
        ranges[t] = k ? make_uint2(st, en) : make_uint2(0u, 0u);
        run += k;
    }
}

// ------------------------------------------------------------ drivers
// Passes over packed items: non-last passes ping-pong between buf[0] and
// buf[1] (input in buf[0]); the last pass writes `last_out` (packed) or the
// caller's value / key arrays and ranges.  wait.withhold applies to the last
// pass only.
template <int BITS, int ITEMS>
void onesweep_passes(uint64_t* const buf[2], uint64_t* last_out, uint32_t* kout, uint32_t* vout,
                     const uint32_t* d_count, int64_t cap, int passes, const SortScratch& s, uint32_t* ranges,
                     DevStatus* status, int sm_count, cudaStream_t st, WaitCfg wait,
                     uint32_t kmask = 0xFFFFFFFFu, const uint32_t* drange = nullptr) {
    constexpr int R = 1 << BITS;
    k_clear_lookback<<<sm_count * 4, 256, 0, st>>>(s.lookback, d_count, cap, R, passes, s.max_sort_tiles,
                                                   kThreads * ITEMS);
    k_hist_scan<BITS><<<1, 256, 0, st>>>(s.hist, passes);
    for (int p = 0; p < passes; ++p) {
        const bool last = p == passes - 1;
        const uint64_t* src = buf[p % 2];
        uint64_t* dst = last ? last_out : buf[(p + 1) % 2];
        k_onesweep<BITS, ITEMS><<<sm_count * 3, kThreads, 0, st>>>(
            src, dst, last ? kout : nullptr, last ? vout : nullptr, d_count, cap, p * BITS, kmask, s.hist + p * kMaxR,
            s.lookback + (int64_t)p * s.max_sort_tiles * R, s.counters + p, last ? ranges : nullptr, status,
            wait.spin, last ? wait.withhold : -1, drange,
            !drange ? 0 : (p == 0 ? 1 : (last && p == 3 ? 2 : 0)));
    }
}

// Emission + tile-key sort + ranges, for one digit width.
template <int BITS, int ITEMS>
void emit_and_sort(const uint64_t* dsorted, const uint64_t* dsorted_narrow, int64_t items, const uint32_t* d_items, int64_t n, const uint4* pr,
                   const ViewInfo* vt, int V,
                   int64_t keys_cap, int key_bits, const SortScratch& s, uint32_t* sorted_keys,
                   uint32_t* sorted_vals, uint32_t* ranges, int64_t total_tiles, uint32_t* d_num_keys,
                   DevStatus* status, int sm_count, cudaStream_t st,
                   void (*mark)(void* const*, int, cudaStream_t), void* const* events, int ev, WaitCfg wait) {
    const int passes = (key_bits + BITS - 1) / BITS;
    const int64_t nblk = (items + kEmitBlock - 1) / kEmitBlock;
    cudaMemsetAsync(s.hist, 0, sizeof(uint32_t) * kMaxPasses * kMaxR, st);
    cudaMemsetAsync(s.counters, 0, sizeof(uint32_t) * 8, st);
    cudaMemsetAsync(s.emit_lookback, 0, sizeof(unsigned long long) * (size_t)nblk, st);
    k_emit<BITS><<<(unsigned)nblk, kEmitThreads, 0, st>>>(dsorted, dsorted_narrow, s.drange, items, n, s.rects, vt, keys_cap, s.tkv[0],
                                                          s.emit_lookback, s.counters + 7, d_num_keys, passes,
                                                          s.hist, 0, nullptr, (uint32_t)total_tiles, d_items,
                                                          status, V, wait.spin);
    if (mark) mark(events, ev, st);
    k_ranges_init<<<sm_count * 2, 256, 0, st>>>(reinterpret_cast<uint2*>(ranges), total_tiles);
    uint64_t* const buf[2] = {s.tkv[0], s.tkv[1]};
    // the last pass writes the caller's arrays, which no later kernel of the
    // call reads: the one pass where the wait test hook applies
    onesweep_passes<BITS, ITEMS>(buf, nullptr, sorted_keys, sorted_vals, d_num_keys, keys_cap, passes, s, ranges,
                                 status, sm_count, st, wait);
    k_ranges_fix<<<sm_count * 2, 256, 0, st>>>(reinterpret_cast<uint2*>(ranges), total_tiles);
}

// Two-level binning: coarse emission and super-tile sort, then the fine
// expansion into the caller's arrays and ranges.
template <int BITS, int ITEMS>
void emit_two_level(const uint64_t* dsorted, const uint64_t* dsorted_narrow, int64_t items, const uint32_t* d_items, int64_t n, const uint4* pr,
                    const ViewInfo* vt, int V,
                    int64_t keys_cap, const SortScratch& s, uint32_t* sorted_keys,
                    uint32_t* sorted_vals, uint32_t* ranges, int64_t total_tiles, uint32_t* d_num_keys,
                    DevStatus* status, int sm_count, cudaStream_t st,
                    void (*mark)(void* const*, int, cudaStream_t), void* const* events, int ev,
                    CoarseLists* coarse, WaitCfg wait, int64_t n_super_exact, uint32_t* order) {
    wait.withhold = -1;  // later kernels read this sort's output
    // super-tiles never outnumber tiles: the tile count bounds the arrays
    // indexed by super-tile (the kernels read the exact count from vt[V]); the
    // key width comes from the exact count when the caller knows it
    const int64_t n_super = total_tiles;
    int bits = 1;
    while ((1LL << bits) < (n_super_exact > 0 ? n_super_exact : n_super)) ++bits;
    const int passes = (bits + BITS - 1) / BITS;
    const int64_t nblk = (items + kEmitBlock - 1) / kEmitBlock;
    cudaMemsetAsync(s.hist, 0, sizeof(uint32_t) * kMaxPasses * kMaxR, st);
    cudaMemsetAsync(s.counters, 0, sizeof(uint32_t) * 8, st);
    cudaMemsetAsync(s.emit_lookback, 0, sizeof(unsigned long long) * (size_t)nblk, st);
    cudaMemsetAsync(s.d_fine_total, 0, sizeof(unsigned long long), st);
    k_emit<BITS><<<(unsigned)nblk, kEmitThreads, 0, st>>>(dsorted, dsorted_narrow, s.drange, items, n, s.rects, vt, keys_cap, s.tkv[0],
                                                          s.emit_lookback, s.counters + 7, s.d_count_coarse,
                                                          passes, s.hist, kSuperShift, s.d_fine_total,
                                                          (uint32_t)n_super, d_items, status, V, wait.spin);
    k_fine_total<<<1, 1, 0, st>>>(s.d_fine_total, keys_cap, d_num_keys, status);
    if (mark) mark(events, ev, st);
    // stable sort by super-tile; the values land in the ping-pong buffer the
    // last pass does not read
    k_ranges_init<<<sm_count, 256, 0, st>>>(s.cranges, n_super);
    uint64_t* const buf[2] = {s.tkv[0], s.tkv[1]};
    const uint64_t* citems = buf[passes % 2];
    // chunk-bitmap lists: the last pass also writes the items' Gaussian
    // indices compactly (into the caller's value array, unused otherwise)
    onesweep_passes<BITS, ITEMS>(buf, buf[passes % 2], nullptr, coarse ? sorted_vals : nullptr, s.d_count_coarse,
                                 keys_cap, passes, s,
                                 reinterpret_cast<uint32_t*>(s.cranges), status, sm_count, st, wait,
                                 (uint32_t)((1ull << bits) - 1ull));
    k_ranges_fix<<<sm_count, 256, 0, st>>>(s.cranges, n_super);
    const unsigned fgrid = (unsigned)(sm_count * 8);
    if (coarse) {
        // chunk-bitmap lists: the bitmaps go to the ping-pong buffer the last
        // pass read and the room after it (2 KB for each of max_chunks)
        uint32_t* bitmap = reinterpret_cast<uint32_t*>(buf[1 - passes % 2]);
        const bool ordered = order && n_super_exact > 0;
        k_fine_chunks<<<1, 1024, 0, st>>>(s.cranges, vt, V, n_super, s.chunk_first, s.d_n_chunks,
                                          s.max_chunks, status, ordered ? order : nullptr,
                                          ordered ? (int)n_super_exact : 0);
        k_chunk_owner<<<(unsigned)((n_super + 7) / 8), 256, 0, st>>>(s.chunk_first, s.cranges, vt, V, n_super,
                                                                   s.chunk_meta, s.max_chunks);
        k_fine_mask<<<fgrid, kFineThreads, 0, st>>>(citems, s.cranges, s.chunk_first, s.chunk_meta, s.d_n_chunks, vt,
                                                    V, total_tiles, bitmap);
        coarse->citems = citems;
        coarse->cvals = sorted_vals;
        coarse->cranges = s.cranges;
        coarse->chunk_first = s.chunk_first;
        coarse->d_n_chunks = s.d_n_chunks;
        coarse->bitmap = bitmap;
        if (ordered) {
            coarse->sorder = order;
            coarse->n_super = n_super_exact;
        }
        return;
    }
    // fine expansion
    k_fine_chunks<<<1, 1024, 0, st>>>(s.cranges, vt, V, n_super, s.chunk_first, s.d_n_chunks,
                                      s.max_chunks, status, nullptr, 0);
    k_chunk_owner<<<(unsigned)((n_super + 7) / 8), 256, 0, st>>>(s.chunk_first, s.cranges, vt, V, n_super,
                                                               s.chunk_meta, s.max_chunks);
    k_fine_count<<<fgrid, kFineThreads, 0, st>>>(citems, s.cranges, s.chunk_first, s.chunk_meta, s.d_n_chunks, vt, V,
                                                 total_tiles, s.chunk_off);
    k_fine_prefix<<<(unsigned)((n_super * 64 + 255) / 256), 256, 0, st>>>(s.chunk_first, s.d_n_chunks, vt, V,
                                                                         total_tiles, s.chunk_off, s.tile_count);
    k_tile_scan<<<1, 1024, 0, st>>>(s.tile_count, total_tiles, keys_cap, reinterpret_cast<uint2*>(ranges));
    // one wave: a grid-stride loop over the chunks with as many blocks as are
    // resident (the staging buffers limit residency below 8 blocks an SM)
    if (sorted_keys)
        k_fine_write<true><<<fine_write_grid<true>(sm_count), kFineThreads, 0, st>>>(
            citems, s.cranges, s.chunk_first, s.chunk_meta, s.d_n_chunks, vt, V, total_tiles, s.chunk_off,
            reinterpret_cast<const uint2*>(ranges), keys_cap, sorted_vals, sorted_keys);
    else
        k_fine_write<false><<<fine_write_grid<false>(sm_count), kFineThreads, 0, st>>>(
            citems, s.cranges, s.chunk_first, s.chunk_meta, s.d_n_chunks, vt, V, total_tiles, s.chunk_off,
            reinterpret_cast<const uint2*>(ranges), keys_cap, sorted_vals, nullptr);
}

}  // namespace

size_t sort_scratch_bytes(int V, int64_t n, int64_t keys_cap, int64_t total_tiles) {
    SortScratch s;
    carve_sort_scratch(nullptr, V, n, keys_cap, total_tiles, &s);
    return s.bytes;
}

void carve_sort_scratch(char* base, int V, int64_t n, int64_t keys_cap, int64_t total_tiles, SortScratch* s) {
    Carver c(base);
    const int64_t items = (int64_t)V * n;
    s->dkv[0] = c.take<uint64_t>(items);
    s->dkv[1] = c.take<uint64_t>(items);
    s->emit_lookback = c.take<unsigned long long>((items + kEmitBlock - 1) / kEmitBlock + 1);
    // super-tiles never outnumber tiles
    const int64_t ns = total_tiles > 0 ? total_tiles : 1;
    // each ping-pong buffer is followed by room for ns + 1 chunk bitmaps, so
    // that the one the super-tile sort leaves free holds the bitmaps of all
    // keys_cap / 256 + ns + 1 chunks the chunk table allows
    const size_t bm_room = (size_t)(ns + 1) * kChunkItems * 8;
    s->tkv[0] = c.take<uint64_t>(keys_cap);
    c.take<char>(bm_room);
    s->tkv[1] = c.take<uint64_t>(keys_cap);
    c.take<char>(bm_room);
    s->hist = c.take<uint32_t>(kMaxPasses * kMaxR);
    s->counters = c.take<uint32_t>(8);
    s->max_sort_tiles = (std::max(items, keys_cap) + kMinTileKeys - 1) / kMinTileKeys + 1;
    s->lookback = c.take<unsigned long long>((size_t)kMaxPasses * s->max_sort_tiles * 256);
    s->d_count_depth = c.take<uint32_t>(1);
    s->drange = c.take<uint32_t>(2);
    s->rects = c.take<uint2>(items);
    s->keep_sums = c.take<uint32_t>((items + kKeepBlock - 1) / kKeepBlock + 1);
    s->max_chunks = keys_cap / kFineChunk + ns + 1;
    s->cranges = c.take<uint2>(ns);
    s->chunk_first = c.take<uint32_t>(ns + 1);
    s->chunk_meta = c.take<uint4>(s->max_chunks);
    s->chunk_off = c.take<uint32_t>((size_t)s->max_chunks * 64);
    s->tile_count = c.take<uint32_t>(ns);
    s->d_count_coarse = c.take<uint32_t>(1);
    s->d_n_chunks = c.take<uint32_t>(1);
    s->d_fine_total = c.take<unsigned long long>(1);
    s->bytes = c.off;
}

void launch_bin_sort(const float* proj, const ViewInfo* vt, int V, int64_t n, int64_t keys_cap,
                     int64_t total_tiles, int binning, int sort_bits, int sort_items, const SortScratch& s,
                     bool depth_ready,
                     uint32_t* sorted_keys, uint32_t* sorted_vals, uint32_t* ranges,
                     uint32_t* d_num_keys, DevStatus* status, int sm_count, cudaStream_t st,
                     void (*mark)(void* const*, int, cudaStream_t), void* const* events, int first_event,
                     bool compact, CoarseLists* coarse, WaitCfg wait, int64_t n_super, uint32_t* order) {
    if (coarse) *coarse = CoarseLists{};
    WaitCfg dwait = wait;
    dwait.withhold = -1;  // the depth sort's output feeds the emission
    const int64_t items = (int64_t)V * n;
    const uint4* pr = reinterpret_cast<const uint4*>(proj);
    if (items == 0) {
        k_clear_u32<<<sm_count * 2, 256, 0, st>>>(ranges, total_tiles * 2);
        k_set_u32<<<1, 1, 0, st>>>(d_num_keys, 0u);
        return;
    }
    // 1. depth sort of all (view, Gaussian) pairs: 32-bit keys, 4 passes of
    //    8-bit digits ending back in dkv[0] (with narrow keys the fourth
    //    launch returns at once and the sort ends in dkv[1])
    if (!depth_ready) {
        k_range_reset<<<1, 1, 0, st>>>(s.drange);
        k_depth_keys<<<(unsigned)((items + 255) / 256), 256, 0, st>>>(pr, items, vt, V, s.dkv[0], s.rects,
                                                                     s.drange);
    }
    // with compaction the kept items move to dkv[1] and the sort ends there;
    // with narrow keys (s.drange) the last pass is skipped and the sort ends
    // in the other buffer (dsorted_narrow)
    const uint64_t* dsorted = s.dkv[0];
    const uint64_t* dsorted_narrow = s.dkv[1];
    const uint32_t* d_items = nullptr;
    cudaMemsetAsync(s.hist, 0, sizeof(uint32_t) * kMaxPasses * kMaxR, st);
    cudaMemsetAsync(s.counters, 0, sizeof(uint32_t) * 8, st);
    if (compact) {
        const int64_t nb = (items + kKeepBlock - 1) / kKeepBlock;
        k_keep_count<<<(unsigned)nb, 256, 0, st>>>(s.dkv[0], items, s.keep_sums);
        launch_scan_sums(s.keep_sums, nb, s.d_count_depth, -1, nullptr, st);
        k_keep_emit<<<(unsigned)nb, 256, 0, st>>>(s.dkv[0], items, s.keep_sums, s.dkv[1]);
        k_hist<8><<<sm_count * 4, kThreads, 0, st>>>(s.dkv[1], s.d_count_depth, items, 4, s.hist, s.drange);
        uint64_t* const dbuf[2] = {s.dkv[1], s.dkv[0]};
        onesweep_passes<8, 16>(dbuf, s.dkv[1], nullptr, nullptr, s.d_count_depth, items, 4, s, nullptr, status,
                               sm_count, st, dwait, 0xFFFFFFFFu, s.drange);
        dsorted = s.dkv[1];
        dsorted_narrow = s.dkv[0];
        d_items = s.d_count_depth;
    } else {
        k_set_u32<<<1, 1, 0, st>>>(s.d_count_depth, (uint32_t)items);
        k_hist<8><<<sm_count * 4, kThreads, 0, st>>>(s.dkv[0], s.d_count_depth, items, 4, s.hist, s.drange);
        uint64_t* const dbuf[2] = {s.dkv[0], s.dkv[1]};
        onesweep_passes<8, 16>(dbuf, s.dkv[0], nullptr, nullptr, s.d_count_depth, items, 4, s, nullptr, status,
                               sm_count, st, dwait, 0xFFFFFFFFu, s.drange);
    }
    if (mark) mark(events, first_event, st);
    // 2. emission in depth order with the key histograms, 3. stable sort by
    //    tile key (direct) or by super-tile key followed by the expansion
    //    into tiles (two-level), into the caller's arrays with ranges
    int bits = 1;
    while ((1LL << bits) < total_tiles) ++bits;
    int sbits = 1;
    while ((1LL << sbits) < (n_super > 0 ? n_super : total_tiles)) ++sbits;
    if (binning != kBinDirect && bits <= kMaxCoarseKeyBits && sbits > sort_bits && sbits <= kWideBits) {
        // a super-tile key of 9 bits: one wide pass instead of two
        emit_two_level<kWideBits, kWideItems>(dsorted, dsorted_narrow, items, d_items, n, pr, vt, V, keys_cap, s, sorted_keys,
                                              sorted_vals, ranges, total_tiles, d_num_keys, status, sm_count, st,
                                              mark, events, first_event + 1, coarse, wait, n_super, order);
        return;
    }
#define GS_EMIT_SORT(B, I)                                                                                      \
    do {                                                                                                        \
        if (binning == kBinDirect || bits > kMaxCoarseKeyBits)                                                  \
            emit_and_sort<B, I>(dsorted, dsorted_narrow, items, d_items, n, pr, vt, V, keys_cap, bits, s, sorted_keys, sorted_vals, \
                                ranges,                                                                         \
                                total_tiles, d_num_keys, status, sm_count, st, mark, events, first_event + 1,   \
                                wait);                                                                          \
        else                                                                                                    \
            emit_two_level<B, I>(dsorted, dsorted_narrow, items, d_items, n, pr, vt, V, keys_cap, s, sorted_keys, sorted_vals,  \
                                 ranges,                                                                        \
                                 total_tiles, d_num_keys, status, sm_count, st, mark, events, first_event + 1,  \
                                 coarse, wait, n_super, order);                                                 \
    } while (0)
    const int it = sort_items == 8 ? 8 : (sort_items == 16 ? 16 : 12);
    switch (sort_bits * 100 + it) {
        case 408: GS_EMIT_SORT(4, 8); break;
        case 412: GS_EMIT_SORT(4, 12); break;
        case 416: GS_EMIT_SORT(4, 16); break;
        case 508: GS_EMIT_SORT(5, 8); break;
        case 512: GS_EMIT_SORT(5, 12); break;
        case 516: GS_EMIT_SORT(5, 16); break;
        case 608: GS_EMIT_SORT(6, 8); break;
        case 612: GS_EMIT_SORT(6, 12); break;
        case 616: GS_EMIT_SORT(6, 16); break;
        case 708: GS_EMIT_SORT(7, 8); break;
        case 712: GS_EMIT_SORT(7, 12); break;
        case 716: GS_EMIT_SORT(7, 16); break;
        case 808: GS_EMIT_SORT(8, 8); break;
        case 816: GS_EMIT_SORT(8, 16); break;
        default: GS_EMIT_SORT(8, 12); break;
    }
#undef GS_EMIT_SORT
}

}  // namespace gs
