// Internal declarations of the sm_103a implementation behind include/gs.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gs.h"

namespace gs {

constexpr int kProjStride = 16;  // floats per (view, Gaussian) projection record
// float4s per record: the public 64-byte form, and the 48-byte form the fused
// calls keep in their workspace (the first three float4s; the tile rectangle,
// which only the depth-key pass of gs_bin_sort reads from a record, goes to
// the separate rectangle item there)
constexpr int kRecF4 = 4, kRecF4Compact = 3;
constexpr int kGradStride = 12;  // floats per (view, Gaussian) 2D-gradient record
constexpr int kParamPlanes = 15;
constexpr int kMaxViews = 4096;

// Compositing constants of the cited 3DGS method (Sec. 3.2.3 of the paper
// refits "the same parameters as in prior 3DGS work").
constexpr float kAlphaMax = 0.99f;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kTMin = 1e-4f;
constexpr float kDilation = 0.3f;
constexpr float kGuard = 1.3f;

// Per-view derived geometry, computed on the device from the camera array.
// Entry V holds the totals (tile_off = total tiles, pix_off = total pixels).
// Super-tiles group kSuper x kSuper tiles for the two-level binning.
constexpr int kSuperShift = 3;
constexpr int kSuper = 1 << kSuperShift;

struct ViewInfo {
    int32_t tx, ty;       // tiles along x / y
    int32_t width, height;
    int64_t tile_off;     // first global tile index of this view
    int64_t pix_off;      // first pixel (per channel) of this view
    int32_t stx, sty;     // super-tiles along x / y
    int64_t stile_off;    // first global super-tile index of this view
    int32_t rect32;       // totals entry vt[V] only: 1 when every view has at most 256 tiles
                          // along x and y, so the tile rectangles take their 4-byte form
    int32_t pad;
};

// Tile rectangle [x0, x1) x [y0, y1) in 4 bytes (x0, x1 - 1, y0, y1 - 1, a
// byte each; the empty rectangle is x0 = 1, x1 = 1, y0 = 0, y1 = 1).
__device__ __forceinline__ uint32_t rect32_pack(uint32_t lo, uint32_t hi) {
    const uint32_t x0 = lo & 0xFFFFu, y0 = lo >> 16, x1 = hi & 0xFFFFu, y1 = hi >> 16;
    if (x1 <= x0 || y1 <= y0) return 1u;
    return x0 | ((x1 - 1u) << 8) | (y0 << 16) | ((y1 - 1u) << 24);
}
__device__ __forceinline__ uint2 rect32_unpack(uint32_t r) {
    return make_uint2((r & 0xFFu) | (((r >> 16) & 0xFFu) << 16),
                      (((r >> 8) & 0xFFu) + 1u) | (((r >> 24) + 1u) << 16));
}

struct DevStatus {
    int32_t code;
    int32_t pad;
    long long detail;
};

__device__ __forceinline__ void record_status(DevStatus* s, int code, long long detail) {
    if (atomicCAS(&s->code, 0, code) == 0) s->detail = detail;
}

// Spin bound for inter-block waits: about one second at 2 GHz (the
// context's default; gs_ctx_set_wait_limit changes it).
constexpr long long kSpinCycles = 2000000000LL;

// Bounded-wait settings passed to the kernels that wait on other blocks:
// spin, the bound in clock cycles; withhold >= 0 (a test hook, honoured by
// gs_bin_sort alone): onesweep tile `withhold` of the last pass of the direct
// binning's tile-key sort publishes no digit counts, so that the waits of the
// tiles after it run out.
struct WaitCfg {
    long long spin = kSpinCycles;
    int64_t withhold = -1;
};

// ------------------------------------------------------------ decoupled look-back
// Slots of a look-back array hold (flag | count): kFlagAgg when a block has
// published its own count, kFlagInc when it has published the inclusive
// prefix through itself.
constexpr unsigned long long kFlagAgg = 1ULL << 62;
constexpr unsigned long long kFlagInc = 2ULL << 62;
constexpr unsigned long long kValMask = (1ULL << 62) - 1;

__device__ __forceinline__ unsigned long long ld_volatile(const unsigned long long* p) {
    return *reinterpret_cast<const volatile unsigned long long*>(p);
}

__device__ __forceinline__ void st_volatile(unsigned long long* p, unsigned long long v) {
    *reinterpret_cast<volatile unsigned long long*>(p) = v;
}

// Exclusive prefix of `mine` over the slots 0..slot-1 of a look-back array
// whose slots hold (flag | count); publishes this slot's inclusive value.
// Four predecessors are read per round trip.  Bounded: when a round finds
// no predecessor ready more than `spin` clock cycles after the wait began, it
// records GS_ERR_TIMEOUT, publishes the partial inclusive value (so that
// later slots need not wait as long) and returns false.
__device__ __forceinline__ bool look_back(unsigned long long* lb, int64_t slot, int stride,
                                          unsigned long long mine, unsigned long long* excl_out,
                                          DevStatus* status, long long spin) {
    unsigned long long excl = 0;
    bool ok = true;
    if (slot > 0) {
        int64_t p = slot - 1;
        const long long t0 = clock64();
        for (;;) {
            unsigned long long x[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) x[k] = (p - k >= 0) ? ld_volatile(lb + (p - k) * stride) : 0ULL;
            bool done = false;
            int used = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (done || used < k) break;  // stop at the first slot that is not ready
                if (!(x[k] & (kFlagAgg | kFlagInc))) break;
                excl += x[k] & kValMask;
                used = k + 1;
                if (x[k] & kFlagInc) done = true;
            }
            if (done) break;
            p -= used;
            // nothing ready: back off so that the polling does not take the
            // issue slots of the SM's other tiles (250 ns measured best of
            // 32-500 ns)
            if (used == 0) __nanosleep(250);
            if (used == 0 && clock64() - t0 > spin) {
                record_status(status, GS_ERR_TIMEOUT, slot);
                ok = false;
                break;
            }
        }
        st_volatile(lb + slot * stride, kFlagInc | (excl + mine));
    }
    *excl_out = excl;
    return ok;
}

// ------------------------------------------------------------ launchers
// Every launcher enqueues on `st`; none synchronises or allocates.

// expect_tiles / expect_super (>= 0): the tile and super-tile totals the
// caller planned for; a different total is reported as GS_ERR_ARG.
// drange (may be null): the depth-key range the projection then accumulates,
// reset here ({all ones, 0}).
void launch_view_table(const gs_camera* d_cams, int V, int tile, ViewInfo* vt,
                       long long expect_tiles, DevStatus* status, cudaStream_t st, long long expect_super = -1,
                       uint32_t* drange = nullptr);

// ------------------------------------------------------------ depth-key range
// drange[0] / drange[1]: the smallest / largest depth-sort key (float32 bits
// of the depth) of the visible (view, Gaussian) items, accumulated by the
// kernels that write the items.  When the keys span fewer than 2^24 - 1
// values ("narrow"), the depth sort orders key - smallest instead (culled
// items: 2^24 - 1): the same order, with a top byte of zero, so the fourth
// 8-bit pass would not move anything and is skipped.
struct DepthXform {
    uint32_t mn;
    bool narrow;
};
__device__ __forceinline__ DepthXform depth_xform(const uint32_t* drange) {
    DepthXform x;
    x.mn = 0;
    x.narrow = false;
    if (drange) {
        const uint32_t mn = drange[0], mx = drange[1];
        x.mn = mn;
        x.narrow = mn <= mx && mx - mn < 0xFFFFFFu;
    }
    return x;
}
__device__ __forceinline__ uint32_t xform_key(uint32_t k, DepthXform x) {
    return !x.narrow ? k : (k == 0xFFFFFFFFu ? 0xFFFFFFu : k - x.mn);
}
// Adds a thread's range [lo, hi] (lo > hi: none) of visible keys: reduced over
// the warp's live threads, then an atomic only where it widens the range.
__device__ __forceinline__ void depth_range_add(uint32_t* drange, uint32_t lo, uint32_t hi) {
    const unsigned am = __activemask();
    lo = __reduce_min_sync(am, lo);
    hi = __reduce_max_sync(am, hi);
    if ((int)(threadIdx.x & 31) == __ffs(am) - 1 && lo <= hi) {
        if (lo < *reinterpret_cast<volatile uint32_t*>(drange)) atomicMin(drange, lo);
        if (hi > *reinterpret_cast<volatile uint32_t*>(drange + 1)) atomicMax(drange + 1, hi);
    }
}

// Super-tiles of views of one size (kSuper x kSuper tiles each).
inline int64_t super_tiles_of(int V, int width, int height, int tile) {
    const int64_t tx = (width + tile - 1) / tile, ty = (height + tile - 1) / tile;
    return (int64_t)V * ((tx + kSuper - 1) / kSuper) * ((ty + kSuper - 1) / kSuper);
}

// Per-scene extras as the projection kernels take them (by value):
// dynamics (group == nullptr: static) and preculling (cell_vis == nullptr:
// none; fwd, when set, receives 1 for kept and 0 for culled Gaussians of the
// pool projected at offset 0).
struct Dyn {
    int n_groups;
    const uint8_t* group;
    const float4* poses;     // [G][2]: quaternion (w, x, y, z), translation (x, y, z, 0)
    const float4* normals;   // nullptr: no relighting
    const float4* light;
    float ambient, diffuse;
    const uint8_t* cell_vis;
    float grid_o[3];
    float grid_size;
    int grid_dims[3];
    uint8_t* fwd;
    const float* lit_tab;    // SH relighting: per group kLitTab floats (launch_light_table); nullptr: off
    const uint8_t* vis;      // light visibility, indexed like the dynamics arrays; nullptr: all lit
};

// Per-group relighting table: the environment coefficients rotated into the
// object's frame (e'[16][3]), then E_c Y_k(R_g^T l) ([16][3]).
constexpr int kLitTab = 96;
constexpr int kMaxGroups = 256;

inline Dyn make_dyn(const gs_dynamics* d, const gs_precull* pc = nullptr, uint8_t* fwd = nullptr,
                    const gs_lighting* lt = nullptr, const float* lit_tab = nullptr) {
    Dyn k{};
    if (lt && lt->light && lit_tab) {
        k.lit_tab = lit_tab;
        k.vis = lt->visibility;
    }
    if (pc && pc->cell_visible) {
        k.cell_vis = pc->cell_visible;
        for (int a = 0; a < 3; ++a) { k.grid_o[a] = pc->origin[a]; k.grid_dims[a] = pc->dims[a]; }
        k.grid_size = pc->cell_size;
        k.fwd = fwd;
    }
    if (d && d->n_groups > 0 && d->group && d->poses) {
        k.n_groups = d->n_groups;
        k.group = d->group;
        k.poses = reinterpret_cast<const float4*>(d->poses);
        k.normals = (d->normals && d->light) ? reinterpret_cast<const float4*>(d->normals) : nullptr;
        k.light = reinterpret_cast<const float4*>(d->light);
        k.ambient = d->ambient;
        k.diffuse = d->diffuse;
    }
    return k;
}

// depth_kv (may be null): packed (float32 depth bits << 32 | record index)
// per (view, Gaussian), all-ones depth when culled, for the depth sort.
// Records of Gaussian g of `params` (plane stride n) go to record v*n_out +
// g_off + g (n_out < 0: n_out = n), so that two pools can share one record
// array; dynamics arrays are indexed by g_off + g.
void launch_project(const float* params, int64_t n, int sh_degree, const Dyn& dyn, const gs_camera* d_cams,
                    const ViewInfo* vt, int V, int tile, float* proj, uint64_t* depth_kv, cudaStream_t st,
                    int64_t g_off = 0, int64_t n_out = -1, uint2* rects = nullptr, int rec4 = kRecF4,
                    uint32_t* drange = nullptr);

// L2 eviction-priority policies for cache-hinted loads and stores.
__device__ __forceinline__ uint64_t l2_policy_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t l2_policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ void st_hint(uint2* p, uint2 v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.v2.u32 [%0], {%1, %2}, %3;" ::"l"(p), "r"(v.x), "r"(v.y), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void st_hint(uint32_t* p, uint32_t v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.u32 [%0], %1, %2;" ::"l"(p), "r"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ uint32_t ld_hint(const uint32_t* p, uint64_t pol) {
    uint32_t v;
    asm volatile("ld.global.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ uint2 ld_hint(const uint2* p, uint64_t pol) {
    uint2 v;
    asm volatile("ld.global.L2::cache_hint.v2.u32 {%0, %1}, [%2], %3;" : "=r"(v.x), "=r"(v.y) : "l"(p), "l"(pol));
    return v;
}

// Adjoint of the first n records of each view (record stride n_out).
void launch_project_bwd(const float* params, int64_t n, int sh_degree, const Dyn& dyn, const gs_camera* d_cams,
                        int V, const float* proj, const float* grad2d, float* dparams,
                        int accumulate, cudaStream_t st, int64_t n_out = -1, int rec4 = kRecF4);

// Fills tab ([max(1, n_groups)][kLitTab]) from the device lighting buffer
// (gs_lighting.light) and the group poses of `dyn`.
void launch_light_table(const Dyn& dyn, const float* light, float* tab, cudaStream_t st);

// Light-space depth map and per-Gaussian visibility (gs_light_depth_map /
// gs_light_visibility); dynamics arrays are indexed by Gaussian.
void launch_light_depth(const float* params, int64_t n, const Dyn& dyn, const gs_light_camera& lc, float* depth,
                        int clear, cudaStream_t st);
void launch_light_visibility(const float* params, int64_t n, const Dyn& dyn, const gs_light_camera& lc,
                             const float* depth, uint8_t* vis, cudaStream_t st);

// Scratch of the bin/sort stage (all device pointers inside the workspace).
// Sorted items are packed (key << 32 | value).
struct SortScratch {
    uint64_t* dkv[2];          // depth sort ping-pong, V*n each
    unsigned long long* emit_lookback;  // emission block look-back (one word per block)
    uint64_t* tkv[2];          // tile-key sort ping-pong, keys_cap each
    uint32_t* hist;            // [4][256]
    uint32_t* counters;        // [8] onesweep tile counters (+ emission block counter)
    unsigned long long* lookback;  // [4][max_tiles][256]
    int64_t max_sort_tiles;    // per pass
    uint32_t* d_count_depth;   // depth-sort items (V*n, or those kept by the compaction)
    uint32_t* drange;          // [2] range of the visible depth keys (depth_xform)
    uint2* rects;              // [V*n] tile rectangle of each record: (x0 | y0 << 16, x1 | y1 << 16),
                               // or as uint32 [V*n] in the 4-byte form when vt[V].rect32; kept in
                               // L2 (evict-last) from the projection to the emission
    uint32_t* keep_sums;       // block sums of the depth-item compaction
    // two-level binning (super-tile lists, then per-tile lists)
    uint2* cranges;            // [total_tiles] bound on super-tiles: coarse [start, end)
    uint32_t* chunk_first;     // [total_tiles + 1] first chunk of each super-tile
    uint4* chunk_meta;         // [max_chunks] per chunk: first and end coarse entry, super-tile, view
    uint32_t* chunk_off;       // [max_chunks][64] per-tile counts, then offsets
    uint32_t* tile_count;      // [total_tiles]
    uint32_t* d_count_coarse;  // coarse entries stored
    uint32_t* d_n_chunks;
    unsigned long long* d_fine_total;  // fine entries implied by the rectangles
    int64_t max_chunks;
    size_t bytes;              // total scratch size
};

size_t sort_scratch_bytes(int V, int64_t n, int64_t keys_cap, int64_t total_tiles);
void carve_sort_scratch(char* base, int V, int64_t n, int64_t keys_cap, int64_t total_tiles, SortScratch* s);

// Binning modes (gs_ctx_set_binning).
constexpr int kBinTwoLevel = 0;
constexpr int kBinDirect = 1;

// Full bin + sort: depth sort, key emission, tile-key sort, ranges.
// Per-tile lists in chunk-bitmap form: two-level binning without the
// expansion into per-tile arrays.  Super-tile s's depth-ordered coarse items
// citems[cranges[s].x, cranges[s].y) are cut into chunks of kChunkItems
// (chunk_first[s] .. chunk_first[s + 1], clamped to *d_n_chunks); the 8
// words bitmap[c][k][0..7] of chunk c and local tile k (8 y + x within the
// super-tile) mark, bit j of word w, whether item 32 w + j of the chunk is an
// entry of that tile.  A tile's list is its marked items in chunk order, the
// order of the expanded list.
constexpr int kChunkItems = 256;
struct CoarseLists {
    const uint64_t* citems = nullptr;  // null: the call produced expanded lists
    const uint32_t* cvals = nullptr;   // the items' Gaussian indices (low words), compact
    const uint2* cranges = nullptr;
    const uint32_t* chunk_first = nullptr;
    const uint32_t* d_n_chunks = nullptr;
    const uint32_t* bitmap = nullptr;
    // super-tiles in the order the raster kernels take them (null: tile
    // order); then their grid is n_super x 64 blocks, one per tile slot of a
    // super-tile (slots outside the view exit)
    const uint32_t* sorder = nullptr;
    int64_t n_super = 0;
};

// coarse: when non-null and the two-level path is taken, the per-tile lists
// are left in chunk-bitmap form (*coarse filled; sorted_keys, sorted_vals and
// ranges untouched); otherwise coarse->citems stays null.
// n_super (> 0): the exact super-tile total, which the view table checks; it
// sizes the super-tile key (one 9-bit pass instead of two 8-bit ones for up
// to 512 super-tiles).  0: unknown, bounded by the tile count.
// order (with n_super > 0 and chunk-bitmap lists; room for n_super words):
// receives the super-tiles by decreasing list length (ties by index), the
// order in which the raster kernels then take them, so that the longest
// lists start first instead of ending the launch (coarse->sorder).
void launch_bin_sort(const float* proj, const ViewInfo* vt, int V, int64_t n, int64_t keys_cap,
                     int64_t total_tiles, int binning, int sort_bits, int sort_items, const SortScratch& s,
                     bool depth_ready,
                     uint32_t* sorted_keys, uint32_t* sorted_vals, uint32_t* ranges,
                     uint32_t* d_num_keys, DevStatus* status, int sm_count, cudaStream_t st,
                     void (*mark)(void* const*, int, cudaStream_t) = nullptr, void* const* events = nullptr,
                     int first_event = 0, bool compact = false, CoarseLists* coarse = nullptr,
                     WaitCfg wait = WaitCfg{}, int64_t n_super = 0, uint32_t* order = nullptr);

// tpr: threads per pixel row of a 16 x 16 tile (2 or 4); 8 x 8 tiles use 4.
// Adjoint: Gaussians with index >= n_active (a frozen pool appended after the
// active one) get no 2D gradient (n_active < 0: all of them do).
// coarse: lists in chunk-bitmap form (then vals and ranges are not read, and
// n_contrib holds citems positions + 1), or null for expanded lists.
void launch_render_fwd(const float* proj, const ViewInfo* vt, int V, int64_t n, int tile, int tpr,
                       const uint32_t* vals, const uint32_t* ranges, float3 bg, float* image,
                       float* T_final, uint32_t* n_contrib, int64_t total_tiles,
                       cudaStream_t st, const CoarseLists* coarse = nullptr, int rec4 = kRecF4);

void launch_raster_bwd(const float* proj, const ViewInfo* vt, int V, int64_t n, int tile, int tpr,
                       const uint32_t* vals, const uint32_t* ranges, float3 bg,
                       const float* T_final, const uint32_t* n_contrib, const float* dimage,
                       float* grad2d, int64_t total_tiles, cudaStream_t st, int64_t n_active = -1,
                       const CoarseLists* coarse = nullptr, int rec4 = kRecF4);

size_t loss_scratch_bytes(int V, int H, int W);
void launch_loss(const float* image, const float* target, int V, int H, int W, float w_l1,
                 float w_ssim, float* d_loss, float* dimage, char* scratch, cudaStream_t st);

// fwd (may be null): Gaussians with fwd[g] == 0 are left untouched.
void launch_adam(float* theta, const float* grad, float* m, float* v, int64_t n,
                 const gs_adam_cfg& cfg, cudaStream_t st, const uint8_t* fwd = nullptr);

// Preculling visibility: max pyramids of the views' depth buffers in
// `scratch` (precull_scratch_bytes), then one thread per cell.
size_t precull_scratch_bytes(const gs_camera* host_cams, int V);
void launch_cell_visibility(const gs_camera* d_cams, const gs_camera* host_cams, int V, const float* depth,
                            const gs_precull& grid, uint8_t* vis, char* scratch, cudaStream_t st);

size_t delta_scratch_bytes(int64_t n);
void launch_delta(const float* theta, float* baseline, int64_t n, float thr, uint32_t* d_idx,
                  uint8_t* d_records, uint32_t* d_count, char* scratch, cudaStream_t st);
// The training step's Adam update and delta extraction: Adam fused with the
// changed test (k_adam_flags), the step counter increment, then (after the
// optional phase mark) the scan and the record emission.
void launch_adam_delta(float* theta, const float* grad, float* m, float* v, int64_t n, const gs_adam_cfg& cfg,
                       const uint8_t* fwd, float* baseline, float thr, uint32_t* d_idx, uint8_t* d_records,
                       uint32_t* d_count, char* scratch, cudaStream_t st, void (*mark)(void* const*, int, cudaStream_t),
                       void* const* events, int event);

// Tensor deltas of one attribute group (GS_ATTR_*) and client-side replay.
bool attr_group(int attr, int* lo, int* hi, int* f32);
void launch_tensor_delta(const float* theta, float* baseline, int64_t n, int attr, float thr, uint32_t* d_idx,
                         uint8_t* d_vals, uint32_t* d_count, char* scratch, cudaStream_t st);
void launch_apply_tensor_delta(float* params, int64_t n, int attr, const uint32_t* d_idx, const uint8_t* d_vals,
                               const uint32_t* d_count, DevStatus* status, int sm_count, cudaStream_t st);
void launch_apply_delta(float* params, int64_t n, const uint8_t* d_records, const uint32_t* d_count,
                        DevStatus* status, int sm_count, cudaStream_t st);

// Exclusive scan of `count` uint32 block sums in place (one block); the total
// goes to *d_total; if cap >= 0 and the total exceeds it, GS_ERR_CAPACITY.
void launch_scan_sums(uint32_t* sums, int64_t count, uint32_t* d_total, long long cap,
                      DevStatus* status, cudaStream_t st);

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Bump allocator over the workspace; with base == nullptr it only measures.
struct Carver {
    char* base;
    size_t off = 0;
    explicit Carver(void* b) : base(static_cast<char*>(b)) {}
    template <class T>
    T* take(size_t count) {
        off = align_up(off, 256);
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

}  // namespace gs

struct gs_ctx {
    int device = 0;
    int sm_count = 148;
    int tile = 16;
    int sort_bits = 8;
    int sort_items = 16;
    int binning = gs::kBinTwoLevel;
    int raster_tpr = 4;       // compositing: threads per pixel row
    int raster_bwd_tpr = 4;   // its adjoint
    void* ws = nullptr;
    size_t ws_bytes = 0;
    gs::DevStatus* d_status = nullptr;
    float* d_light_tab = nullptr;   // [kMaxGroups][kLitTab] relighting table
    long long wait_cycles = gs::kSpinCycles;  // bound of every inter-block wait
    int64_t wait_test_tile = -1;              // gs_ctx_set_wait_test (test hook; -1: off)
    cudaStream_t capture_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
};
