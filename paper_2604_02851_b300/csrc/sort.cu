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
// The sort is a onesweep radix sort: one histogram pass over the keys for all
// digit passes, then per digit pass a single kernel that ranks a tile of keys
// in shared memory (warp match-any ranking, stable), publishes its per-digit
// counts, resolves its global digit offsets by decoupled look-back over the
// preceding tiles, and scatters.  Blocks are persistent and take tiles from
// an atomic counter in launch order, so a waited-on tile always belongs to a
// running block; every wait is bounded and reports GS_ERR_TIMEOUT.
#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kItems = 16;                       // keys per thread per tile
constexpr int kTileKeys = kThreads * kItems;     // 4096
constexpr int kMaxPasses = 4;
constexpr unsigned long long kFlagAgg = 1ULL << 62;
constexpr unsigned long long kFlagInc = 2ULL << 62;
constexpr unsigned long long kValMask = (1ULL << 62) - 1;

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ unsigned long long ld_volatile(const unsigned long long* p) {
    return *reinterpret_cast<const volatile unsigned long long*>(p);
}

__device__ __forceinline__ void st_volatile(unsigned long long* p, unsigned long long v) {
    *reinterpret_cast<volatile unsigned long long*>(p) = v;
}

__device__ __forceinline__ int64_t clamp_count(const uint32_t* d_count, int64_t cap) {
    const int64_t k = (int64_t)*d_count;
    return k < cap ? k : cap;
}

// ------------------------------------------------------------ histograms
template <int BITS>
__global__ void __launch_bounds__(kThreads)
k_hist(const uint32_t* __restrict__ keys, const uint32_t* d_count, int64_t cap, int begin_bit,
       int passes, uint32_t* __restrict__ hist) {
    constexpr int R = 1 << BITS;
    __shared__ uint32_t sh[kWarps][kMaxPasses][R];
    for (int i = threadIdx.x; i < kWarps * kMaxPasses * R; i += kThreads) (&sh[0][0][0])[i] = 0;
    __syncthreads();
    const int64_t count = clamp_count(d_count, cap);
    const int w = threadIdx.x / 32;
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * kThreads) {
        const uint32_t k = keys[i];
        for (int p = 0; p < passes; ++p) atomicAdd(&sh[w][p][(k >> (begin_bit + p * BITS)) & (R - 1)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * R; i += kThreads) {
        const int p = i / R, d = i % R;
        uint32_t s = 0;
        for (int ww = 0; ww < kWarps; ++ww) s += sh[ww][p][d];
        if (s) atomicAdd(&hist[p * 256 + d], s);
    }
}

// Exclusive scan of each pass's histogram in place (one block).
template <int BITS>
__global__ void k_hist_scan(uint32_t* hist, int passes) {
    constexpr int R = 1 << BITS;
    __shared__ uint32_t s[256];
    for (int p = 0; p < passes; ++p) {
        if (threadIdx.x < R) s[threadIdx.x] = hist[p * 256 + threadIdx.x];
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t acc = 0;
            for (int d = 0; d < R; ++d) { const uint32_t c = s[d]; s[d] = acc; acc += c; }
        }
        __syncthreads();
        if (threadIdx.x < R) hist[p * 256 + threadIdx.x] = s[threadIdx.x];
        __syncthreads();
    }
}

// ------------------------------------------------------------ onesweep pass
template <int BITS>
__global__ void __launch_bounds__(kThreads)
k_onesweep(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
           uint32_t* __restrict__ kout, uint32_t* __restrict__ vout, const uint32_t* d_count,
           int64_t cap, int shift, const uint32_t* __restrict__ digit_off,
           unsigned long long* __restrict__ lookback, uint32_t* tile_counter, DevStatus* status) {
    constexpr int R = 1 << BITS;
    constexpr uint32_t MASK = R - 1;
    __shared__ uint32_t s_keys[kTileKeys];
    __shared__ uint32_t s_vals[kTileKeys];
    __shared__ uint32_t s_whist[kWarps][R];   // per-warp digit counts, then warp prefixes
    __shared__ uint32_t s_local[R];           // tile-local start of each digit
    __shared__ uint32_t s_gbase[R];           // global start of this tile's digit run
    __shared__ uint32_t s_tile;
    __shared__ int s_abort;

    const int64_t count = clamp_count(d_count, cap);
    const int64_t n_tiles = (count + kTileKeys - 1) / kTileKeys;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt = lanemask_lt();

    for (;;) {
        if (threadIdx.x == 0) { s_tile = atomicAdd(tile_counter, 1u); s_abort = 0; }
        for (int i = lane; i < R; i += 32) s_whist[warp][i] = 0;
        __syncthreads();
        const int64_t tile = s_tile;
        if (tile >= n_tiles) break;

        // ---- load (warp-striped: warp w owns a contiguous run of 32*kItems keys)
        uint32_t key[kItems], val[kItems], rank[kItems];
        const int64_t wbase = tile * kTileKeys + (int64_t)warp * 32 * kItems;
#pragma unroll
        for (int j = 0; j < kItems; ++j) {
            const int64_t idx = wbase + j * 32 + lane;
            const bool ok = idx < count;
            key[j] = ok ? kin[idx] : 0xFFFFFFFFu;
            val[j] = ok ? vin[idx] : 0u;
        }
        // ---- stable rank within the warp, item order j*32 + lane
#pragma unroll
        for (int j = 0; j < kItems; ++j) {
            const uint32_t d = (key[j] >> shift) & MASK;
            const uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
            const uint32_t before = s_whist[warp][d];
            rank[j] = before + __popc(peers & lt);
            __syncwarp();
            if (lane == __ffs(peers) - 1) s_whist[warp][d] = before + __popc(peers);
            __syncwarp();
        }
        __syncthreads();

        // ---- per digit: prefix over warps, tile count, publish, look back
        uint32_t tile_cnt = 0;
        if (threadIdx.x < R) {
            const int d = threadIdx.x;
            uint32_t acc = 0;
            for (int w = 0; w < kWarps; ++w) { const uint32_t c = s_whist[w][d]; s_whist[w][d] = acc; acc += c; }
            tile_cnt = acc;
            unsigned long long* slot = lookback + tile * R + d;
            st_volatile(slot, (tile == 0 ? kFlagInc : kFlagAgg) | (unsigned long long)tile_cnt);
        }
        // tile-local digit starts: exclusive scan of tile_cnt over d (serial per warp chunk)
        if (threadIdx.x < R) s_local[threadIdx.x] = tile_cnt;
        __syncthreads();
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
        if (threadIdx.x < R) {
            const int d = threadIdx.x;
            unsigned long long excl = 0;
            if (tile > 0) {
                int64_t p = tile - 1;
                const long long t0 = clock64();
                for (;;) {
                    const unsigned long long x = ld_volatile(lookback + p * R + d);
                    if (x & (kFlagAgg | kFlagInc)) {
                        excl += x & kValMask;
                        if (x & kFlagInc) break;
                        --p;
                        continue;
                    }
                    if (clock64() - t0 > kSpinCycles) {
                        record_status(status, GS_ERR_TIMEOUT, tile);
                        s_abort = 1;
                        break;
                    }
                }
                st_volatile(lookback + tile * R + d, kFlagInc | (excl + tile_cnt));
            }
            s_gbase[d] = digit_off[d] + (uint32_t)excl;
        }
        __syncthreads();
        // ---- stage in shared memory in digit order
#pragma unroll
        for (int j = 0; j < kItems; ++j) {
            const uint32_t d = (key[j] >> shift) & MASK;
            const uint32_t lp = s_local[d] + s_whist[warp][d] + rank[j];
            s_keys[lp] = key[j];
            s_vals[lp] = val[j];
        }
        __syncthreads();
        // ---- scatter (invalid tail keys are all-ones: they sit at the end of
        //      the last digit's run, i.e. at staged positions >= valid)
        const int64_t rem = count - tile * kTileKeys;
        const int valid = rem < kTileKeys ? (int)rem : kTileKeys;
        if (!s_abort) {
            for (int i = threadIdx.x; i < valid; i += kThreads) {
                const uint32_t k = s_keys[i];
                const uint32_t d = (k >> shift) & MASK;
                const uint32_t pos = s_gbase[d] + (uint32_t)i - s_local[d];
                kout[pos] = k;
                vout[pos] = s_vals[i];
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------ utilities
__global__ void k_set_u32(uint32_t* p, uint32_t v) { *p = v; }

// Zero `per_tile` u64 words for each of `passes` look-back arrays, for the
// tiles that the device count implies.
__global__ void k_clear_lookback(unsigned long long* lb, const uint32_t* d_count, int64_t cap,
                                 int radix, int passes, int64_t max_tiles) {
    const int64_t count = clamp_count(d_count, cap);
    const int64_t tiles = (count + kTileKeys - 1) / kTileKeys;
    const int64_t words = tiles * radix;
    for (int p = 0; p < passes; ++p)
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words;
             i += (int64_t)gridDim.x * blockDim.x)
            lb[(int64_t)p * max_tiles * radix + i] = 0ULL;
}

__global__ void k_clear_u32(uint32_t* p, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = 0u;
}

// ------------------------------------------------------------ emission
constexpr int kEmitThreads = 256;
constexpr int kEmitItems = 4;
constexpr int kEmitBlock = kEmitThreads * kEmitItems;

__global__ void __launch_bounds__(kEmitThreads)
k_emit_count(const uint32_t* __restrict__ dvals, int64_t total, const uint4* __restrict__ proj,
             uint32_t* __restrict__ block_sums) {
    const int64_t base = (int64_t)blockIdx.x * kEmitBlock;
    uint32_t s = 0;
    for (int i = threadIdx.x; i < kEmitBlock; i += kEmitThreads) {
        const int64_t idx = base + i;
        if (idx < total) s += proj[(size_t)dvals[idx] * 4 + 3].z;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
    __shared__ uint32_t ws[kEmitThreads / 32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < kEmitThreads / 32; ++w) t += ws[w];
        block_sums[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(kEmitThreads)
k_emit_keys(const uint32_t* __restrict__ dvals, int64_t total, int64_t n,
            const uint4* __restrict__ proj, const ViewInfo* __restrict__ vt,
            const uint32_t* __restrict__ block_off, int64_t cap, uint32_t* __restrict__ keys,
            uint32_t* __restrict__ vals) {
    __shared__ uint32_t s_off[kEmitBlock + 1];
    __shared__ uint32_t s_lo[kEmitBlock], s_hi[kEmitBlock], s_g[kEmitBlock], s_kb[kEmitBlock],
        s_tx[kEmitBlock];
    __shared__ uint32_t s_wsum[kEmitThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kEmitBlock;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    // blocked: thread t owns items t*kEmitItems .. +kEmitItems-1
    uint32_t cnt[kEmitItems], tsum = 0;
#pragma unroll
    for (int j = 0; j < kEmitItems; ++j) {
        const int li = t * kEmitItems + j;
        const int64_t idx = base + li;
        cnt[j] = 0;
        if (idx < total) {
            const uint32_t r = dvals[idx];
            const uint4 pr = proj[(size_t)r * 4 + 3];
            cnt[j] = pr.z;
            const uint32_t v = (uint32_t)(r / (uint64_t)n);
            s_lo[li] = pr.x;
            s_hi[li] = pr.y;
            s_g[li] = r - v * (uint32_t)n;
            s_kb[li] = (uint32_t)vt[v].tile_off;
            s_tx[li] = (uint32_t)vt[v].tx;
        }
        tsum += cnt[j];
    }
    uint32_t incl = tsum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_wsum[warp] = incl;
    __syncthreads();
    uint32_t wbase = 0, btotal = 0;
    for (int w = 0; w < kEmitThreads / 32; ++w) {
        if (w < warp) wbase += s_wsum[w];
        btotal += s_wsum[w];
    }
    uint32_t run = wbase + incl - tsum;
#pragma unroll
    for (int j = 0; j < kEmitItems; ++j) {
        s_off[t * kEmitItems + j] = run;
        run += cnt[j];
    }
    if (t == 0) s_off[kEmitBlock] = btotal;
    __syncthreads();
    const int64_t out0 = block_off[blockIdx.x];
    for (uint32_t k = t; k < btotal; k += kEmitThreads) {
        // last item whose offset <= k (it has a non-zero count)
        int lo = 0, hi = kEmitBlock;  // s_off[lo] <= k < s_off[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (s_off[mid] <= k) lo = mid; else hi = mid;
        }
        const uint32_t li = k - s_off[lo];
        const uint32_t x0 = s_lo[lo] & 0xFFFFu, y0 = s_lo[lo] >> 16;
        const uint32_t w = (s_hi[lo] & 0xFFFFu) - x0;
        const uint32_t tx = x0 + li % w, ty = y0 + li / w;
        const int64_t pos = out0 + k;
        if (pos < cap) {
            keys[pos] = s_kb[lo] + ty * s_tx[lo] + tx;
            vals[pos] = s_g[lo];
        }
    }
}

// Depth-sort input from projection records: key = float32 depth bits of a
// visible (view, Gaussian), all-ones when culled; value = record index.
__global__ void k_depth_keys(const uint4* __restrict__ proj, int64_t items, uint32_t* __restrict__ keys,
                             uint32_t* __restrict__ vals) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= items) return;
    const uint32_t tiles = proj[i * 4 + 3].z;
    keys[i] = tiles ? proj[i * 4].z : 0xFFFFFFFFu;
    vals[i] = (uint32_t)i;
}

__global__ void k_ranges(const uint32_t* __restrict__ keys, const uint32_t* d_count, int64_t cap,
                         uint2* __restrict__ ranges) {
    const int64_t count = clamp_count(d_count, cap);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t k = keys[i];
        if (i == 0 || keys[i - 1] != k) ranges[k].x = (uint32_t)i;
        if (i == count - 1 || keys[i + 1] != k) ranges[k].y = (uint32_t)(i + 1);
    }
}

template <int BITS>
void sort_pairs_bits(const uint32_t* kin, const uint32_t* vin, uint32_t* ktmp, uint32_t* vtmp,
                     uint32_t* kout, uint32_t* vout, const uint32_t* d_count, int64_t cap,
                     int key_bits, const SortScratch& s, DevStatus* status, int sm_count,
                     cudaStream_t st) {
    constexpr int R = 1 << BITS;
    const int passes = (key_bits + BITS - 1) / BITS;
    const int grid_stream = sm_count * 4;
    cudaMemsetAsync(s.hist, 0, sizeof(uint32_t) * kMaxPasses * 256, st);
    cudaMemsetAsync(s.counters, 0, sizeof(uint32_t) * 8, st);
    k_clear_lookback<<<grid_stream, 256, 0, st>>>(s.lookback, d_count, cap, R, passes, s.max_sort_tiles);
    k_hist<BITS><<<grid_stream, kThreads, 0, st>>>(kin, d_count, cap, 0, passes, s.hist);
    k_hist_scan<BITS><<<1, 256, 0, st>>>(s.hist, passes);
    // destinations: the last pass writes (kout, vout); earlier ones alternate
    const uint32_t* src_k = kin;
    const uint32_t* src_v = vin;
    for (int p = 0; p < passes; ++p) {
        const bool to_out = ((passes - 1 - p) % 2) == 0;
        uint32_t* dk = to_out ? kout : ktmp;
        uint32_t* dv = to_out ? vout : vtmp;
        k_onesweep<BITS><<<sm_count * 2, kThreads, 0, st>>>(
            src_k, src_v, dk, dv, d_count, cap, p * BITS, s.hist + p * 256,
            s.lookback + (int64_t)p * s.max_sort_tiles * R, s.counters + p, status);
        src_k = dk;
        src_v = dv;
    }
}

}  // namespace

// Sort (key, value) pairs by the low `key_bits` bits of the key, stably.
void sort_pairs(const uint32_t* kin, const uint32_t* vin, uint32_t* ktmp, uint32_t* vtmp,
                uint32_t* kout, uint32_t* vout, const uint32_t* d_count, int64_t cap, int key_bits,
                int digit_bits, const SortScratch& s, DevStatus* status, int sm_count,
                cudaStream_t st) {
    if (key_bits < 1) key_bits = 1;
    switch (digit_bits) {
        case 4: sort_pairs_bits<4>(kin, vin, ktmp, vtmp, kout, vout, d_count, cap, key_bits, s, status, sm_count, st); break;
        case 5: sort_pairs_bits<5>(kin, vin, ktmp, vtmp, kout, vout, d_count, cap, key_bits, s, status, sm_count, st); break;
        case 6: sort_pairs_bits<6>(kin, vin, ktmp, vtmp, kout, vout, d_count, cap, key_bits, s, status, sm_count, st); break;
        case 7: sort_pairs_bits<7>(kin, vin, ktmp, vtmp, kout, vout, d_count, cap, key_bits, s, status, sm_count, st); break;
        default: sort_pairs_bits<8>(kin, vin, ktmp, vtmp, kout, vout, d_count, cap, key_bits, s, status, sm_count, st); break;
    }
}

size_t sort_scratch_bytes(int V, int64_t n, int64_t keys_cap) {
    Carver c(nullptr);
    const int64_t items = (int64_t)V * n;
    c.take<uint32_t>(items); c.take<uint32_t>(items); c.take<uint32_t>(items); c.take<uint32_t>(items);
    c.take<uint32_t>((items + kEmitBlock - 1) / kEmitBlock + 1);
    for (int i = 0; i < 5; ++i) c.take<uint32_t>(keys_cap);
    c.take<uint32_t>(kMaxPasses * 256);
    c.take<uint32_t>(8);
    const int64_t mx = (std::max(items, keys_cap) + kTileKeys - 1) / kTileKeys + 1;
    c.take<unsigned long long>((size_t)kMaxPasses * mx * 256);
    c.take<uint32_t>(1);
    return c.off;
}

void carve_sort_scratch(char* base, int V, int64_t n, int64_t keys_cap, SortScratch* s) {
    Carver c(base);
    const int64_t items = (int64_t)V * n;
    s->dkeys[0] = c.take<uint32_t>(items);
    s->dvals[0] = c.take<uint32_t>(items);
    s->dkeys[1] = c.take<uint32_t>(items);
    s->dvals[1] = c.take<uint32_t>(items);
    s->block_sums = c.take<uint32_t>((items + kEmitBlock - 1) / kEmitBlock + 1);
    s->tkeys[0] = c.take<uint32_t>(keys_cap);
    s->tvals[0] = c.take<uint32_t>(keys_cap);
    s->tkeys[1] = c.take<uint32_t>(keys_cap);
    s->tvals[1] = c.take<uint32_t>(keys_cap);
    s->tkeys[2] = c.take<uint32_t>(keys_cap);
    s->hist = c.take<uint32_t>(kMaxPasses * 256);
    s->counters = c.take<uint32_t>(8);
    s->max_sort_tiles = (std::max(items, keys_cap) + kTileKeys - 1) / kTileKeys + 1;
    s->lookback = c.take<unsigned long long>((size_t)kMaxPasses * s->max_sort_tiles * 256);
    s->d_count_depth = c.take<uint32_t>(1);
}

void launch_scan_sums(uint32_t* sums, int64_t count, uint32_t* d_total, long long cap,
                      DevStatus* status, cudaStream_t st);

void launch_bin_sort(const float* proj, const ViewInfo* vt, int V, int64_t n, int64_t keys_cap,
                     int64_t total_tiles, int sort_bits, const SortScratch& s, bool depth_ready,
                     uint32_t* sorted_keys, uint32_t* sorted_vals, uint32_t* ranges,
                     uint32_t* d_num_keys, DevStatus* status, int sm_count, cudaStream_t st) {
    const int64_t items = (int64_t)V * n;
    const uint4* pr = reinterpret_cast<const uint4*>(proj);
    // ranges start empty
    k_clear_u32<<<sm_count * 2, 256, 0, st>>>(ranges, total_tiles * 2);
    if (items == 0) {
        k_set_u32<<<1, 1, 0, st>>>(d_num_keys, 0u);
        return;
    }
    // 1. depth sort of all (view, Gaussian) pairs (32-bit keys, 8-bit digits)
    if (!depth_ready)
        k_depth_keys<<<(unsigned)((items + 255) / 256), 256, 0, st>>>(pr, items, s.dkeys[0], s.dvals[0]);
    k_set_u32<<<1, 1, 0, st>>>(s.d_count_depth, (uint32_t)items);
    // 4 passes (even): in -> tmp -> out -> tmp -> out, so out may alias in
    sort_pairs(s.dkeys[0], s.dvals[0], s.dkeys[1], s.dvals[1], s.dkeys[0], s.dvals[0],
               s.d_count_depth, items, 32, 8, s, status, sm_count, st);
    const uint32_t* dv_sorted = s.dvals[0];
    // 2. emission in depth order
    const int64_t nblk = (items + kEmitBlock - 1) / kEmitBlock;
    k_emit_count<<<(unsigned)nblk, kEmitThreads, 0, st>>>(dv_sorted, items, pr, s.block_sums);
    launch_scan_sums(s.block_sums, nblk, d_num_keys, (long long)keys_cap, status, st);
    k_emit_keys<<<(unsigned)nblk, kEmitThreads, 0, st>>>(dv_sorted, items, n, pr, vt, s.block_sums,
                                                         keys_cap, s.tkeys[0], s.tvals[0]);
    // 3. stable sort by tile key: input tkeys[0], temporary tkeys[1], output
    //    the caller's arrays (keys into tkeys[2] if the caller wants none)
    int bits = 1;
    while ((1LL << bits) < total_tiles) ++bits;
    uint32_t* kout = sorted_keys ? sorted_keys : s.tkeys[2];
    sort_pairs(s.tkeys[0], s.tvals[0], s.tkeys[1], s.tvals[1], kout, sorted_vals, d_num_keys,
               keys_cap, bits, sort_bits, s, status, sm_count, st);
    // 4. per-tile ranges
    k_ranges<<<sm_count * 4, 256, 0, st>>>(kout, d_num_keys, keys_cap, reinterpret_cast<uint2*>(ranges));
}

}  // namespace gs
