// extern "C" entry points declared in include/gs.h.
//
// Host-side argument checks happen before anything is enqueued; kernels
// report their own errors through the context's device status word.  Scratch
// comes from the context workspace, carved per call from its start (calls on
// one context are stream-ordered, so a later call may reuse the region).
#include <algorithm>
#include <cstring>
#include <new>

#include "gs_internal.cuh"

using namespace gs;

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

inline cudaStream_t S(void* s) { return static_cast<cudaStream_t>(s); }

gs_status_t launch_check() {
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

int64_t tiles_of(const gs_camera* cams, int V, int tile) {
    int64_t t = 0;
    for (int v = 0; v < V; ++v)
        t += (int64_t)((cams[v].width + tile - 1) / tile) * ((cams[v].height + tile - 1) / tile);
    return t;
}

bool bad_views(int V) { return V < 1 || V > kMaxViews; }

bool bad_precull(const gs_precull* p) {
    return p && (!p->cell_visible || !(p->cell_size > 0.f) || p->dims[0] < 1 || p->dims[1] < 1 || p->dims[2] < 1 ||
                 (int64_t)p->dims[0] * p->dims[1] * p->dims[2] >= (1LL << 40));
}

bool bad_dyn(const gs_dynamics* d) {
    return d && (d->n_groups < 0 || d->n_groups > 256 || (d->n_groups > 0 && (!d->group || !d->poses)) ||
                 (d->normals && !d->light));
}

bool bad_lighting(const gs_lighting* lt, const gs_dynamics* d) {
    return lt && (!lt->light || (d && d->normals));
}

bool bad_light_cam(const gs_light_camera* c) {
    return !c || !(c->texel > 0.f) || !(c->texel < 3.0e38f) || c->width < 1 || c->width > 16384 || c->height < 1 ||
           c->height > 16384 || !(c->alpha_min > 0.f) || !(c->alpha_min <= 0.99f) || !(c->bias >= 0.f) ||
           !(c->bias < 3.0e38f);
}

// Projection extras of a scene; fills the context's relighting table first
// when the scene is relit.
Dyn scene_dyn(gs_ctx* ctx, const gs_dynamics* d, const gs_precull* pc, uint8_t* fwd, const gs_lighting* lt,
              cudaStream_t st) {
    const Dyn k = make_dyn(d, pc, fwd, lt, ctx->d_light_tab);
    if (k.lit_tab) launch_light_table(k, lt->light, ctx->d_light_tab, st);
    return k;
}

// Workspace plan of the fused calls (render_batch, train_step).
struct FusedPlan {
    ViewInfo* vt;
    float* proj;
    char* sort;
    uint32_t* vals;
    uint32_t* ranges;
    uint32_t* n_keys;
    float* T_final;
    uint32_t* n_contrib;
    float* dimage;
    char* loss;
    float* grad2d;
    char* delta;
    uint8_t* fwd;
    uint32_t* order;  // super-tiles in raster order
    size_t bytes;
};

FusedPlan plan_fused(void* base, int V, int64_t n, int64_t keys_cap, int64_t total_tiles,
                     int64_t total_pixels, int H, int W, bool train) {
    Carver c(base);
    FusedPlan p{};
    p.vt = c.take<ViewInfo>(V + 1);
    p.proj = c.take<float>((size_t)V * n * kProjStride);
    p.sort = c.take<char>(sort_scratch_bytes(V, n, keys_cap, total_tiles));
    p.vals = c.take<uint32_t>(keys_cap);
    p.ranges = c.take<uint32_t>(total_tiles * 2);
    p.n_keys = c.take<uint32_t>(1);
    if (train) {
        p.T_final = c.take<float>(total_pixels);
        p.n_contrib = c.take<uint32_t>(total_pixels);
        p.dimage = c.take<float>(3 * total_pixels);
        p.loss = c.take<char>(loss_scratch_bytes(V, H, W));
        p.grad2d = c.take<float>((size_t)V * n * kGradStride);
        p.delta = c.take<char>(delta_scratch_bytes(n));
        p.fwd = c.take<uint8_t>(n > 0 ? n : 1);
    }
    p.order = c.take<uint32_t>(total_tiles > 0 ? total_tiles : 1);  // super-tiles never outnumber tiles
    p.bytes = c.off;
    return p;
}

gs_status_t check_ws(const gs_ctx* ctx, size_t need) {
    return need <= ctx->ws_bytes ? GS_OK : GS_ERR_CAPACITY;
}

// The context's wait bound without the test hook (fused calls read their
// sorts' outputs).
WaitCfg spin_only(const gs_ctx* ctx) {
    WaitCfg w;
    w.spin = ctx->wait_cycles;
    return w;
}

}  // namespace

extern "C" {

gs_status_t gs_ctx_create(gs_ctx** out, int device, size_t workspace_bytes) {
    if (!out) return GS_ERR_ARG;
    *out = nullptr;
    gs_ctx* c = new (std::nothrow) gs_ctx();
    if (!c) return GS_ERR_OOM;
    c->device = device;
    DeviceGuard g(device);
    if (cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        delete c;
        return GS_ERR_CUDA;
    }
    if (cudaMalloc(&c->d_status, sizeof(DevStatus)) != cudaSuccess) {
        delete c;
        return GS_ERR_OOM;
    }
    if (cudaMalloc(&c->d_light_tab, sizeof(float) * kMaxGroups * kLitTab) != cudaSuccess) {
        cudaFree(c->d_status);
        delete c;
        return GS_ERR_OOM;
    }
    cudaMemset(c->d_status, 0, sizeof(DevStatus));
    if (cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaFree(c->d_light_tab);
        cudaFree(c->d_status);
        delete c;
        return GS_ERR_CUDA;
    }
    *out = c;
    if (workspace_bytes) {
        const gs_status_t s = gs_ctx_reserve(c, workspace_bytes);
        if (s != GS_OK) {
            gs_ctx_destroy(c);
            *out = nullptr;
            return s;
        }
    }
    return GS_OK;
}

gs_status_t gs_ctx_destroy(gs_ctx* ctx) {
    if (!ctx) return GS_ERR_ARG;
    DeviceGuard g(ctx->device);
    cudaDeviceSynchronize();
    if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
    if (ctx->graph) cudaGraphDestroy(ctx->graph);
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->d_status) cudaFree(ctx->d_status);
    if (ctx->d_light_tab) cudaFree(ctx->d_light_tab);
    if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
    delete ctx;
    return GS_OK;
}

gs_status_t gs_ctx_reserve(gs_ctx* ctx, size_t bytes) {
    if (!ctx) return GS_ERR_ARG;
    if (bytes <= ctx->ws_bytes) return GS_OK;
    DeviceGuard g(ctx->device);
    cudaDeviceSynchronize();
    if (ctx->ws) cudaFree(ctx->ws);
    ctx->ws = nullptr;
    ctx->ws_bytes = 0;
    if (cudaMalloc(&ctx->ws, bytes) != cudaSuccess) {
        cudaGetLastError();
        return GS_ERR_OOM;
    }
    ctx->ws_bytes = bytes;
    return GS_OK;
}

gs_status_t gs_ctx_set_tile(gs_ctx* ctx, int32_t tile) {
    if (!ctx || (tile != 8 && tile != 16)) return GS_ERR_ARG;
    ctx->tile = tile;
    return GS_OK;
}

gs_status_t gs_ctx_set_sort_bits(gs_ctx* ctx, int32_t bits) {
    if (!ctx || bits < 4 || bits > 8) return GS_ERR_ARG;
    ctx->sort_bits = bits;
    return GS_OK;
}

gs_status_t gs_ctx_set_sort_items(gs_ctx* ctx, int32_t items) {
    if (!ctx || (items != 8 && items != 12 && items != 16)) return GS_ERR_ARG;
    ctx->sort_items = items;
    return GS_OK;
}

gs_status_t gs_ctx_set_binning(gs_ctx* ctx, int32_t mode) {
    if (!ctx || (mode != GS_BINNING_TWO_LEVEL && mode != GS_BINNING_DIRECT)) return GS_ERR_ARG;
    ctx->binning = mode == GS_BINNING_DIRECT ? kBinDirect : kBinTwoLevel;
    return GS_OK;
}

gs_status_t gs_ctx_set_raster_threads(gs_ctx* ctx, int32_t threads_per_row) {
    if (!ctx || (threads_per_row != 2 && threads_per_row != 4)) return GS_ERR_ARG;
    ctx->raster_tpr = threads_per_row;
    ctx->raster_bwd_tpr = threads_per_row;
    return GS_OK;
}

gs_status_t gs_ctx_set_raster_bwd_threads(gs_ctx* ctx, int32_t threads_per_row) {
    if (!ctx || (threads_per_row != 2 && threads_per_row != 4)) return GS_ERR_ARG;
    ctx->raster_bwd_tpr = threads_per_row;
    return GS_OK;
}

gs_status_t gs_ctx_set_wait_limit(gs_ctx* ctx, int64_t cycles) {
    if (!ctx || cycles < 0) return GS_ERR_ARG;
    ctx->wait_cycles = cycles == 0 ? kSpinCycles : (long long)cycles;
    return GS_OK;
}

gs_status_t gs_ctx_set_wait_test(gs_ctx* ctx, int64_t tile) {
    if (!ctx || tile < -1) return GS_ERR_ARG;
    ctx->wait_test_tile = tile;
    return GS_OK;
}

gs_status_t gs_ctx_get_tuning(const gs_ctx* ctx, int32_t* binning, int32_t* sort_bits, int32_t* sort_items,
                              int32_t* raster_threads, int32_t* raster_bwd_threads) {
    if (!ctx) return GS_ERR_ARG;
    if (binning) *binning = ctx->binning == kBinDirect ? GS_BINNING_DIRECT : GS_BINNING_TWO_LEVEL;
    if (sort_bits) *sort_bits = ctx->sort_bits;
    if (sort_items) *sort_items = ctx->sort_items;
    if (raster_threads) *raster_threads = ctx->raster_tpr;
    if (raster_bwd_threads) *raster_bwd_threads = ctx->raster_bwd_tpr;
    return GS_OK;
}

gs_status_t gs_get_status(gs_ctx* ctx, void* stream, int32_t* status, int64_t* detail) {
    if (!ctx || !status) return GS_ERR_ARG;
    DeviceGuard g(ctx->device);
    DevStatus h{};
    if (cudaMemcpyAsync(&h, ctx->d_status, sizeof(h), cudaMemcpyDeviceToHost, S(stream)) != cudaSuccess)
        return GS_ERR_CUDA;
    if (cudaStreamSynchronize(S(stream)) != cudaSuccess) return GS_ERR_CUDA;
    cudaMemsetAsync(ctx->d_status, 0, sizeof(DevStatus), S(stream));
    if (cudaStreamSynchronize(S(stream)) != cudaSuccess) return GS_ERR_CUDA;
    *status = h.code;
    if (detail) *detail = h.detail;
    return GS_OK;
}

int64_t gs_total_tiles(const gs_ctx* ctx, const gs_camera* host_cams, int32_t n_views) {
    if (!ctx || !host_cams || bad_views(n_views)) return -1;
    return tiles_of(host_cams, n_views, ctx->tile);
}

size_t gs_workspace_size(const gs_ctx* ctx, const gs_camera* host_cams, int32_t n_views, int64_t n,
                         int64_t keys_cap) {
    if (!ctx || !host_cams || bad_views(n_views) || n < 0 || keys_cap < 0) return 0;
    const int64_t tt = tiles_of(host_cams, n_views, ctx->tile);
    int64_t px = 0;
    for (int v = 0; v < n_views; ++v) px += (int64_t)host_cams[v].width * host_cams[v].height;
    const FusedPlan p = plan_fused(nullptr, n_views, n, keys_cap, tt, px, host_cams[0].height,
                                   host_cams[0].width, true);
    return p.bytes + 4096;
}

gs_status_t gs_project(gs_ctx* ctx, const gs_scene* scene, const gs_camera* d_cams, int32_t n_views,
                       float* proj, void* stream) {
    if (!ctx || !scene || !d_cams || !proj || bad_views(n_views) || scene->n < 0 ||
        scene->sh_degree < 0 || scene->sh_degree > 3 || (scene->n > 0 && !scene->params))
        return GS_ERR_ARG;
    if ((int64_t)n_views * scene->n >= (1LL << 32) || bad_dyn(scene->dyn) || bad_precull(scene->precull) ||
        bad_lighting(scene->lighting, scene->dyn))
        return GS_ERR_ARG;
    Carver c(ctx->ws);
    ViewInfo* vt = c.take<ViewInfo>(n_views + 1);
    if (check_ws(ctx, c.off)) return GS_ERR_CAPACITY;
    DeviceGuard g(ctx->device);
    launch_view_table(d_cams, n_views, ctx->tile, vt, -1, ctx->d_status, S(stream));
    const Dyn dyn = scene_dyn(ctx, scene->dyn, scene->precull, nullptr, scene->lighting, S(stream));
    launch_project(scene->params, scene->n, scene->sh_degree, dyn, d_cams, vt, n_views, ctx->tile, proj, nullptr,
                   S(stream));
    return launch_check();
}

gs_status_t gs_bin_sort(gs_ctx* ctx, const float* proj, const gs_camera* d_cams, int32_t n_views, int64_t n,
                        int64_t total_tiles, int64_t keys_cap, uint32_t* sorted_keys, uint32_t* sorted_vals,
                        uint32_t* ranges, uint32_t* d_num_keys, void* stream) {
    if (!ctx || !proj || !d_cams || !sorted_vals || !ranges || !d_num_keys || bad_views(n_views) || n < 0 ||
        total_tiles < 1 || keys_cap < 0 || keys_cap >= (1LL << 32) || (int64_t)n_views * n >= (1LL << 32))
        return GS_ERR_ARG;
    Carver c(ctx->ws);
    ViewInfo* vt = c.take<ViewInfo>(n_views + 1);
    char* ss = c.take<char>(sort_scratch_bytes(n_views, n, keys_cap, total_tiles));
    if (check_ws(ctx, c.off)) return GS_ERR_CAPACITY;
    DeviceGuard g(ctx->device);
    SortScratch s;
    carve_sort_scratch(ss, n_views, n, keys_cap, total_tiles, &s);
    launch_view_table(d_cams, n_views, ctx->tile, vt, total_tiles, ctx->d_status, S(stream));
    WaitCfg wait;
    wait.spin = ctx->wait_cycles;
    wait.withhold = ctx->wait_test_tile;  // the test hook applies to this call only
    launch_bin_sort(proj, vt, n_views, n, keys_cap, total_tiles, ctx->binning, ctx->sort_bits, ctx->sort_items, s, false, sorted_keys,
                    sorted_vals, ranges, d_num_keys, ctx->d_status, ctx->sm_count, S(stream), nullptr, nullptr, 0,
                    false, nullptr, wait);
    return launch_check();
}

gs_status_t gs_render_fwd(gs_ctx* ctx, const float* proj, const gs_camera* d_cams, int32_t n_views, int64_t n,
                          int64_t total_tiles, const uint32_t* sorted_vals, const uint32_t* ranges,
                          const float* bg, float* image, float* T_final, uint32_t* n_contrib, void* stream) {
    if (!ctx || !proj || !d_cams || !sorted_vals || !ranges || !image || bad_views(n_views) || n < 0 ||
        total_tiles < 1)
        return GS_ERR_ARG;
    Carver c(ctx->ws);
    ViewInfo* vt = c.take<ViewInfo>(n_views + 1);
    if (check_ws(ctx, c.off)) return GS_ERR_CAPACITY;
    DeviceGuard g(ctx->device);
    const float3 b = bg ? make_float3(bg[0], bg[1], bg[2]) : make_float3(0.f, 0.f, 0.f);
    launch_view_table(d_cams, n_views, ctx->tile, vt, total_tiles, ctx->d_status, S(stream));
    launch_render_fwd(proj, vt, n_views, n, ctx->tile, ctx->raster_tpr, sorted_vals, ranges, b, image, T_final, n_contrib,
                      total_tiles, S(stream));
    return launch_check();
}

gs_status_t gs_loss(gs_ctx* ctx, const float* image, const float* target, int32_t n_views, int32_t height,
                    int32_t width, float w_l1, float w_ssim, float* d_loss, float* dimage, void* stream) {
    if (!ctx || !image || !target || !d_loss || !dimage || bad_views(n_views) || height < 1 || width < 1)
        return GS_ERR_ARG;
    Carver c(ctx->ws);
    char* ls = c.take<char>(loss_scratch_bytes(n_views, height, width));
    if (check_ws(ctx, c.off)) return GS_ERR_CAPACITY;
    DeviceGuard g(ctx->device);
    launch_loss(image, target, n_views, height, width, w_l1, w_ssim, d_loss, dimage, ls, S(stream));
    return launch_check();
}

gs_status_t gs_raster_bwd(gs_ctx* ctx, const float* proj, const gs_camera* d_cams, int32_t n_views, int64_t n,
                          int64_t total_tiles, const uint32_t* sorted_vals, const uint32_t* ranges,
                          const float* bg, const float* T_final, const uint32_t* n_contrib,
                          const float* dimage, float* grad2d, void* stream) {
    if (!ctx || !proj || !d_cams || !sorted_vals || !ranges || !T_final || !n_contrib || !dimage || !grad2d ||
        bad_views(n_views) || n < 0 || total_tiles < 1)
        return GS_ERR_ARG;
    Carver c(ctx->ws);
    ViewInfo* vt = c.take<ViewInfo>(n_views + 1);
    if (check_ws(ctx, c.off)) return GS_ERR_CAPACITY;
    DeviceGuard g(ctx->device);
    const float3 b = bg ? make_float3(bg[0], bg[1], bg[2]) : make_float3(0.f, 0.f, 0.f);
    launch_view_table(d_cams, n_views, ctx->tile, vt, total_tiles, ctx->d_status, S(stream));
    launch_raster_bwd(proj, vt, n_views, n, ctx->tile, ctx->raster_bwd_tpr, sorted_vals, ranges, b, T_final, n_contrib, dimage,
                      grad2d, total_tiles, S(stream));
    return launch_check();
}

gs_status_t gs_project_bwd(gs_ctx* ctx, const gs_scene* scene, const gs_camera* d_cams, int32_t n_views,
                           const float* proj, const float* grad2d, float* dparams, int32_t accumulate,
                           void* stream) {
    if (!ctx || !scene || !d_cams || !proj || !grad2d || !dparams || bad_views(n_views) || scene->n < 0 ||
        scene->sh_degree < 0 || scene->sh_degree > 3 || (scene->n > 0 && !scene->params) || bad_dyn(scene->dyn) ||
        bad_precull(scene->precull) || bad_lighting(scene->lighting, scene->dyn))
        return GS_ERR_ARG;
    DeviceGuard g(ctx->device);
    const Dyn dyn = scene_dyn(ctx, scene->dyn, scene->precull, nullptr, scene->lighting, S(stream));
    launch_project_bwd(scene->params, scene->n, scene->sh_degree, dyn, d_cams, n_views, proj, grad2d, dparams,
                       accumulate, S(stream));
    return launch_check();
}

gs_status_t gs_render_bwd(gs_ctx* ctx, const gs_scene* scene, const gs_camera* d_cams, int32_t n_views,
                          int64_t total_tiles, const float* proj, const uint32_t* sorted_vals,
                          const uint32_t* ranges, const float* bg, const float* T_final,
                          const uint32_t* n_contrib, const float* dimage, float* grad2d, float* dparams,
                          void* stream) {
    if (!scene) return GS_ERR_ARG;
    gs_status_t s = gs_raster_bwd(ctx, proj, d_cams, n_views, scene->n, total_tiles, sorted_vals, ranges, bg,
                                  T_final, n_contrib, dimage, grad2d, stream);
    if (s != GS_OK) return s;
    return gs_project_bwd(ctx, scene, d_cams, n_views, proj, grad2d, dparams, 0, stream);
}

gs_status_t gs_adam_step(gs_ctx* ctx, float* theta, const float* grad, float* m, float* v, int64_t n,
                         const gs_adam_cfg* cfg, void* stream) {
    if (!ctx || !cfg || n < 0 || (n > 0 && (!theta || !grad || !m || !v)) || (!cfg->d_step && cfg->step < 1))
        return GS_ERR_ARG;
    DeviceGuard g(ctx->device);
    launch_adam(theta, grad, m, v, n, *cfg, S(stream));
    return launch_check();
}

gs_status_t gs_extract_delta(gs_ctx* ctx, const float* theta, float* baseline, int64_t n, float thr,
                             uint32_t* d_idx, uint8_t* d_records, uint32_t* d_count, void* stream) {
    if (!ctx || n < 0 || !d_count || (n > 0 && (!theta || !baseline || !d_idx || !d_records)) ||
        n >= (1LL << 32) || !(thr >= 0.f))
        return GS_ERR_ARG;
    Carver c(ctx->ws);
    char* ds = c.take<char>(delta_scratch_bytes(n));
    if (check_ws(ctx, c.off)) return GS_ERR_CAPACITY;
    DeviceGuard g(ctx->device);
    launch_delta(theta, baseline, n, thr, d_idx, d_records, d_count, ds, S(stream));
    return launch_check();
}

int32_t gs_tensor_record_bytes(int32_t attr) {
    int lo, hi, f32;
    if (!attr_group(attr, &lo, &hi, &f32)) return -1;
    return (hi - lo) * (f32 ? 4 : 2);
}

gs_status_t gs_extract_tensor_delta(gs_ctx* ctx, const float* theta, float* baseline, int64_t n, int32_t attr,
                                    float thr, uint32_t* d_idx, void* d_vals, uint32_t* d_count, void* stream) {
    int lo, hi, f32;
    if (!ctx || n < 0 || !d_count || (n > 0 && (!theta || !baseline || !d_idx || !d_vals)) ||
        n >= (1LL << 32) || !(thr >= 0.f) || !attr_group(attr, &lo, &hi, &f32))
        return GS_ERR_ARG;
    Carver c(ctx->ws);
    char* ds = c.take<char>(delta_scratch_bytes(n));
    if (check_ws(ctx, c.off)) return GS_ERR_CAPACITY;
    DeviceGuard g(ctx->device);
    launch_tensor_delta(theta, baseline, n, attr, thr, d_idx, static_cast<uint8_t*>(d_vals), d_count, ds,
                        S(stream));
    return launch_check();
}

gs_status_t gs_apply_tensor_delta(gs_ctx* ctx, float* params, int64_t n, int32_t attr, const uint32_t* d_idx,
                                  const void* d_vals, const uint32_t* d_count, void* stream) {
    int lo, hi, f32;
    if (!ctx || n < 0 || !d_count || (n > 0 && (!params || !d_idx || !d_vals)) || !attr_group(attr, &lo, &hi, &f32))
        return GS_ERR_ARG;
    if (n == 0) return GS_OK;
    DeviceGuard g(ctx->device);
    launch_apply_tensor_delta(params, n, attr, d_idx, static_cast<const uint8_t*>(d_vals), d_count, ctx->d_status,
                              ctx->sm_count, S(stream));
    return launch_check();
}

gs_status_t gs_apply_delta(gs_ctx* ctx, float* params, int64_t n, const uint8_t* d_records,
                           const uint32_t* d_count, void* stream) {
    if (!ctx || n < 0 || !d_count || (n > 0 && (!params || !d_records))) return GS_ERR_ARG;
    if (n == 0) return GS_OK;
    DeviceGuard g(ctx->device);
    launch_apply_delta(params, n, d_records, d_count, ctx->d_status, ctx->sm_count, S(stream));
    return launch_check();
}

// n_super (> 0): the exact super-tile total of the views (checked by the view
// table): the super-tile sort takes no more digits than it needs and the
// compositing takes the longest tile lists first.
static gs_status_t render_batch(gs_ctx* ctx, const gs_scene* scene, const gs_camera* d_cams, int32_t n_requests,
                                int64_t total_tiles, int64_t n_super, int64_t keys_cap, const float* bg,
                                float* image, void* stream) {
    if (!ctx || !scene || !d_cams || !image || bad_views(n_requests) || scene->n < 0 || total_tiles < 1 ||
        keys_cap < 0 || keys_cap >= (1LL << 32) || scene->sh_degree < 0 || scene->sh_degree > 3 ||
        (scene->n > 0 && !scene->params) || (int64_t)n_requests * scene->n >= (1LL << 32) || bad_dyn(scene->dyn) ||
        bad_precull(scene->precull) || bad_lighting(scene->lighting, scene->dyn))
        return GS_ERR_ARG;
    const FusedPlan p0 = plan_fused(nullptr, n_requests, scene->n, keys_cap, total_tiles, 0, 0, 0, false);
    if (check_ws(ctx, p0.bytes)) return GS_ERR_CAPACITY;
    const FusedPlan p = plan_fused(ctx->ws, n_requests, scene->n, keys_cap, total_tiles, 0, 0, 0, false);
    DeviceGuard g(ctx->device);
    cudaStream_t st = S(stream);
    SortScratch s;
    carve_sort_scratch(p.sort, n_requests, scene->n, keys_cap, total_tiles, &s);
    const float3 b = bg ? make_float3(bg[0], bg[1], bg[2]) : make_float3(0.f, 0.f, 0.f);
    launch_view_table(d_cams, n_requests, ctx->tile, p.vt, total_tiles, ctx->d_status, st,
                      n_super > 0 ? n_super : -1, s.drange);
    const Dyn dyn = scene_dyn(ctx, scene->dyn, scene->precull, nullptr, scene->lighting, st);
    launch_project(scene->params, scene->n, scene->sh_degree, dyn, d_cams, p.vt, n_requests, ctx->tile, p.proj,
                   s.dkv[0], st, 0, -1, s.rects, kRecF4Compact, s.drange);
    // two-level binning leaves the per-tile lists in chunk-bitmap form
    CoarseLists cl;
    launch_bin_sort(p.proj, p.vt, n_requests, scene->n, keys_cap, total_tiles, ctx->binning, ctx->sort_bits, ctx->sort_items, s, true, nullptr,
                    p.vals, p.ranges, p.n_keys, ctx->d_status, ctx->sm_count, st, nullptr, nullptr, 0,
                    scene->precull != nullptr, &cl, spin_only(ctx), n_super > 0 ? n_super : 0,
                    n_super > 0 ? p.order : nullptr);
    launch_render_fwd(p.proj, p.vt, n_requests, scene->n, ctx->tile, ctx->raster_tpr, p.vals, p.ranges, b, image, nullptr,
                      nullptr, total_tiles, st, &cl, kRecF4Compact);
    return launch_check();
}

gs_status_t gs_render_batch(gs_ctx* ctx, const gs_scene* scene, const gs_camera* d_cams, int32_t n_requests,
                            int64_t total_tiles, int64_t keys_cap, const float* bg, float* image,
                            void* stream) {
    return render_batch(ctx, scene, d_cams, n_requests, total_tiles, 0, keys_cap, bg, image, stream);
}

gs_status_t gs_render_batch_sized(gs_ctx* ctx, const gs_scene* scene, const gs_camera* d_cams,
                                  const gs_camera* host_cams, int32_t n_requests, int64_t keys_cap,
                                  const float* bg, float* image, void* stream) {
    if (!ctx || !host_cams || bad_views(n_requests)) return GS_ERR_ARG;
    int64_t ns = 0;
    for (int v = 0; v < n_requests; ++v) {
        if (host_cams[v].width < 1 || host_cams[v].height < 1) return GS_ERR_ARG;
        ns += super_tiles_of(1, host_cams[v].width, host_cams[v].height, ctx->tile);
    }
    return render_batch(ctx, scene, d_cams, n_requests, tiles_of(host_cams, n_requests, ctx->tile), ns, keys_cap,
                        bg, image, stream);
}

static void mark(void* const* events, int i, cudaStream_t st) {
    // phase boundary i of gs_train_step_events (null events: nothing recorded)
    if (!events || !events[i]) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cs);
    if (cs == cudaStreamCaptureStatusActive)
        cudaEventRecordWithFlags(static_cast<cudaEvent_t>(events[i]), st, cudaEventRecordExternal);
    else
        cudaEventRecord(static_cast<cudaEvent_t>(events[i]), st);
}

gs_status_t gs_train_step(gs_ctx* ctx, const gs_camera* d_cams, const gs_train_io* io, const gs_train_cfg* cfg,
                          void* stream) {
    return gs_train_step_events(ctx, d_cams, io, cfg, nullptr, stream);
}

gs_status_t gs_train_step_events(gs_ctx* ctx, const gs_camera* d_cams, const gs_train_io* io,
                                 const gs_train_cfg* cfg, void* const* ev, void* stream) {
    if (!ctx || !d_cams || !io || !cfg || bad_views(cfg->n_views) || cfg->n < 0 || cfg->sh_degree < 0 ||
        cfg->sh_degree > 3 || cfg->width < 1 || cfg->height < 1 || cfg->keys_cap < 0 ||
        cfg->keys_cap >= (1LL << 32) || (int64_t)cfg->n_views * cfg->n >= (1LL << 32) || !io->params ||
        !io->grads || !io->adam_m || !io->adam_v || !io->baseline || !io->targets || !io->image ||
        !io->d_loss || !io->d_delta_idx || !io->d_delta_records || !io->d_delta_count || !io->d_step ||
        bad_dyn(cfg->dyn) || bad_precull(cfg->precull) || bad_lighting(cfg->lighting, cfg->dyn) ||
        cfg->n_frozen < 0 || (cfg->n_frozen > 0 && !io->frozen) ||
        (int64_t)cfg->n_views * (cfg->n + cfg->n_frozen) >= (1LL << 32) || cfg->phases < 0 ||
        cfg->phases > GS_TRAIN_ALL)
        return GS_ERR_ARG;
    const int phases = cfg->phases ? cfg->phases : GS_TRAIN_ALL;
    const int V = cfg->n_views;
    const int64_t na = cfg->n;                  // active pool
    const int64_t n = cfg->n + cfg->n_frozen;   // every rendered Gaussian
    const int B = ctx->tile;
    const int64_t tt = (int64_t)V * ((cfg->width + B - 1) / B) * ((cfg->height + B - 1) / B);
    const int64_t ns = super_tiles_of(V, cfg->width, cfg->height, B);
    const int64_t px = (int64_t)V * cfg->width * cfg->height;
    const FusedPlan p0 = plan_fused(nullptr, V, n, cfg->keys_cap, tt, px, cfg->height, cfg->width, true);
    if (check_ws(ctx, p0.bytes)) return GS_ERR_CAPACITY;
    const FusedPlan p = plan_fused(ctx->ws, V, n, cfg->keys_cap, tt, px, cfg->height, cfg->width, true);
    DeviceGuard g(ctx->device);
    cudaStream_t st = S(stream);
    SortScratch s;
    carve_sort_scratch(p.sort, V, n, cfg->keys_cap, tt, &s);
    const float3 b = make_float3(cfg->bg[0], cfg->bg[1], cfg->bg[2]);
    mark(ev, 0, st);
    launch_view_table(d_cams, V, B, p.vt, tt, ctx->d_status, st, ns, s.drange);
    const Dyn dyn = scene_dyn(ctx, cfg->dyn, cfg->precull, p.fwd, cfg->lighting, st);
    if (!(phases & GS_TRAIN_GRADIENT)) {
        // update only: the gradient of the caller's io->grads; the phase marks
        // of the skipped part are recorded together.  Preculling still marks
        // the Gaussians it keeps (Adam leaves the others).
        if (cfg->precull)
            launch_project(io->params, na, cfg->sh_degree, dyn, d_cams, p.vt, V, B, p.proj, s.dkv[0], st, 0, n,
                           s.rects, kRecF4Compact, s.drange);
        for (int e = 1; e <= 8; ++e) mark(ev, e, st);
        gs_adam_cfg ac = cfg->adam;
        ac.d_step = io->d_step;
        ac.increment = 1;
        launch_adam_delta(io->params, io->grads, io->adam_m, io->adam_v, na, ac, cfg->precull ? p.fwd : nullptr,
                          io->baseline, cfg->delta_thr, io->d_delta_idx, io->d_delta_records, io->d_delta_count,
                          p.delta, st, ev ? mark : nullptr, ev, 9);
        return launch_check();
    }
    launch_project(io->params, na, cfg->sh_degree, dyn, d_cams, p.vt, V, B, p.proj, s.dkv[0], st, 0, n, s.rects,
                   kRecF4Compact, s.drange);
    if (cfg->n_frozen > 0)
        launch_project(io->frozen, cfg->n_frozen, cfg->sh_degree, dyn, d_cams, p.vt, V, B, p.proj, s.dkv[0], st,
                       na, n, s.rects, kRecF4Compact, s.drange);
    mark(ev, 1, st);
    // two-level binning leaves the per-tile lists in chunk-bitmap form, which
    // both raster kernels walk
    CoarseLists cl;
    launch_bin_sort(p.proj, p.vt, V, n, cfg->keys_cap, tt, ctx->binning, ctx->sort_bits, ctx->sort_items, s, true, nullptr,
                    p.vals, p.ranges, p.n_keys, ctx->d_status, ctx->sm_count, st, ev ? mark : nullptr, ev, 2,
                    cfg->precull != nullptr, &cl, spin_only(ctx), ns, p.order);
    mark(ev, 4, st);
    launch_render_fwd(p.proj, p.vt, V, n, B, ctx->raster_tpr, p.vals, p.ranges, b, io->image, p.T_final, p.n_contrib, tt,
                      st, &cl, kRecF4Compact);
    mark(ev, 5, st);
    launch_loss(io->image, io->targets, V, cfg->height, cfg->width, cfg->w_l1, cfg->w_ssim, io->d_loss, p.dimage,
                p.loss, st);
    mark(ev, 6, st);
    launch_raster_bwd(p.proj, p.vt, V, n, B, ctx->raster_bwd_tpr, p.vals, p.ranges, b, p.T_final, p.n_contrib, p.dimage, p.grad2d, tt,
                      st, na, &cl, kRecF4Compact);
    mark(ev, 7, st);
    launch_project_bwd(io->params, na, cfg->sh_degree, dyn, d_cams, V, p.proj, p.grad2d, io->grads, 0, st, n,
                       kRecF4Compact);
    mark(ev, 8, st);
    if (!(phases & GS_TRAIN_UPDATE)) {
        mark(ev, 9, st);
        mark(ev, 10, st);
        return launch_check();
    }
    gs_adam_cfg ac = cfg->adam;
    ac.d_step = io->d_step;
    ac.increment = 1;
    // Adam with the delta's changed test (phase 9 ends after it), then the
    // delta's scan and records
    launch_adam_delta(io->params, io->grads, io->adam_m, io->adam_v, na, ac, cfg->precull ? p.fwd : nullptr,
                      io->baseline, cfg->delta_thr, io->d_delta_idx, io->d_delta_records, io->d_delta_count,
                      p.delta, st, ev ? mark : nullptr, ev, 9);
    mark(ev, 10, st);
    return launch_check();
}

gs_status_t gs_autotune(gs_ctx* ctx, const gs_scene* scene, const gs_camera* d_cams, const gs_camera* host_cams,
                        int32_t n_views, int64_t keys_cap, int32_t reps, gs_tune_entry* results,
                        int32_t max_results, int32_t* n_results, void* stream) {
    if (!ctx || !scene || !d_cams || !host_cams || bad_views(n_views) || scene->n < 0 || scene->sh_degree < 0 ||
        scene->sh_degree > 3 || (scene->n > 0 && !scene->params) || keys_cap < 0 || keys_cap >= (1LL << 32) ||
        (int64_t)n_views * scene->n >= (1LL << 32) || reps < 1 || max_results < 0 ||
        (max_results > 0 && !results) || bad_dyn(scene->dyn) || bad_precull(scene->precull) ||
        bad_lighting(scene->lighting, scene->dyn))
        return GS_ERR_ARG;
    const int V = n_views;
    const int64_t n = scene->n;
    const int B = ctx->tile;
    const int64_t tt = tiles_of(host_cams, V, B);
    int64_t px = 0, ns = 0;
    for (int v = 0; v < V; ++v) {
        px += (int64_t)host_cams[v].width * host_cams[v].height;
        ns += super_tiles_of(1, host_cams[v].width, host_cams[v].height, B);
    }
    const FusedPlan p0 = plan_fused(nullptr, V, n, keys_cap, tt, px, host_cams[0].height, host_cams[0].width, true);
    if (check_ws(ctx, p0.bytes)) return GS_ERR_CAPACITY;
    const FusedPlan p = plan_fused(ctx->ws, V, n, keys_cap, tt, px, host_cams[0].height, host_cams[0].width, true);
    DeviceGuard g(ctx->device);
    cudaStream_t st = S(stream);
    SortScratch s;
    carve_sort_scratch(p.sort, V, n, keys_cap, tt, &s);
    const Dyn dyn = scene_dyn(ctx, scene->dyn, scene->precull, nullptr, scene->lighting, st);
    // the image is not read back: it goes to the image-gradient buffer, which
    // the adjoint then reads (its cost does not depend on the values)
    float* image = p.dimage;
    const float3 bg = make_float3(0.f, 0.f, 0.f);
    // ev (may be null): recorded before compositing, between compositing and
    // its adjoint, and after the adjoint
    auto run = [&](cudaEvent_t* ev) {
        launch_view_table(d_cams, V, B, p.vt, tt, ctx->d_status, st, ns, s.drange);
        launch_project(scene->params, n, scene->sh_degree, dyn, d_cams, p.vt, V, B, p.proj, s.dkv[0], st, 0, -1, s.rects,
                       kRecF4Compact, s.drange);
        CoarseLists cl;
        launch_bin_sort(p.proj, p.vt, V, n, keys_cap, tt, ctx->binning, ctx->sort_bits, ctx->sort_items, s, true,
                        nullptr, p.vals, p.ranges, p.n_keys, ctx->d_status, ctx->sm_count, st, nullptr, nullptr, 0,
                        scene->precull != nullptr, &cl, spin_only(ctx), ns, p.order);
        if (ev) cudaEventRecord(ev[0], st);
        launch_render_fwd(p.proj, p.vt, V, n, B, ctx->raster_tpr, p.vals, p.ranges, bg, image, p.T_final,
                          p.n_contrib, tt, st, &cl, kRecF4Compact);
        if (ev) cudaEventRecord(ev[1], st);
        launch_raster_bwd(p.proj, p.vt, V, n, B, ctx->raster_bwd_tpr, p.vals, p.ranges, bg, p.T_final, p.n_contrib,
                          p.dimage, p.grad2d, tt, st, -1, &cl, kRecF4Compact);
        if (ev) cudaEventRecord(ev[2], st);
    };
    constexpr int kMaxReps = 16;
    const int nrep = reps < kMaxReps ? reps : kMaxReps;
    cudaEvent_t ev[2 + 3 * kMaxReps];
    int made = 0;
    while (made < 2 + 3 * nrep && cudaEventCreate(&ev[made]) == cudaSuccess) ++made;
    auto destroy_events = [&]() {
        for (int i = 0; i < made; ++i) cudaEventDestroy(ev[i]);
    };
    if (made < 2 + 3 * nrep) {
        destroy_events();
        return GS_ERR_CUDA;
    }
    cudaEvent_t e0 = ev[0], e1 = ev[1];
    cudaEvent_t(*er)[3] = reinterpret_cast<cudaEvent_t(*)[3]>(ev + 2);
    const int keep_bin = ctx->binning, keep_bits = ctx->sort_bits, keep_items = ctx->sort_items,
              keep_tpr = ctx->raster_tpr, keep_btpr = ctx->raster_bwd_tpr;
    const int bins[2] = {kBinTwoLevel, kBinDirect};
    const int bitss[3] = {8, 7, 6};
    const int itemss[3] = {16, 12, 8};
    const int tprs[2] = {4, 2};
    // per binning mode (its raster kernels read different list forms): the
    // sort settings with the least time outside compositing, and per layout
    // the best compositing and adjoint times seen
    float best_pre[2] = {-1.f, -1.f}, best_fwd[2][2] = {{-1.f, -1.f}, {-1.f, -1.f}},
          best_bwd[2][2] = {{-1.f, -1.f}, {-1.f, -1.f}};
    int bbits[2] = {keep_bits, keep_bits}, bitems[2] = {keep_items, keep_items};
    int32_t count = 0;
    gs_status_t rc = GS_OK;
    for (int ib = 0; ib < 2 && rc == GS_OK; ++ib)
        for (int ibits = 0; ibits < 3 && rc == GS_OK; ++ibits)
            for (int iit = 0; iit < 3 && rc == GS_OK; ++iit)
                for (int itp = 0; itp < 2 && rc == GS_OK; ++itp) {
                    if (B == 8 && tprs[itp] != 4) continue;  // 8-px tiles have one layout
                    ctx->binning = bins[ib];
                    ctx->sort_bits = bitss[ibits];
                    ctx->sort_items = itemss[iit];
                    ctx->raster_tpr = tprs[itp];
                    ctx->raster_bwd_tpr = tprs[itp];
                    run(nullptr);  // warm-up
                    cudaEventRecord(e0, st);
                    for (int r = 0; r < reps; ++r) run(r < nrep ? er[r] : nullptr);
                    cudaEventRecord(e1, st);
                    if (cudaEventSynchronize(e1) != cudaSuccess) { rc = GS_ERR_CUDA; break; }
                    DevStatus h{};
                    if (cudaMemcpy(&h, ctx->d_status, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) {
                        rc = GS_ERR_CUDA;
                        break;
                    }
                    if (h.code != GS_OK) { rc = (gs_status_t)h.code; break; }  // left in the status word
                    float ms = 0.f, fwd = 0.f, bwd = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    ms /= (float)reps;
                    for (int r = 0; r < nrep; ++r) {
                        float a = 0.f, b = 0.f;
                        cudaEventElapsedTime(&a, er[r][0], er[r][1]);
                        cudaEventElapsedTime(&b, er[r][1], er[r][2]);
                        fwd += a;
                        bwd += b;
                    }
                    fwd /= (float)nrep;
                    bwd /= (float)nrep;
                    if (count < max_results) {
                        gs_tune_entry& t = results[count];
                        t.binning = bins[ib] == kBinDirect ? GS_BINNING_DIRECT : GS_BINNING_TWO_LEVEL;
                        t.sort_bits = bitss[ibits];
                        t.sort_items = itemss[iit];
                        t.raster_threads = tprs[itp];
                        t.ms = ms;
                        t.ms_render_fwd = fwd;
                        t.ms_render_bwd = bwd;
                    }
                    ++count;
                    const float pre = ms - fwd - bwd;
                    if (best_pre[ib] < 0.f || pre < best_pre[ib]) {
                        best_pre[ib] = pre;
                        bbits[ib] = bitss[ibits]; bitems[ib] = itemss[iit];
                    }
                    if (best_fwd[ib][itp] < 0.f || fwd < best_fwd[ib][itp]) best_fwd[ib][itp] = fwd;
                    if (best_bwd[ib][itp] < 0.f || bwd < best_bwd[ib][itp]) best_bwd[ib][itp] = bwd;
                }
    destroy_events();
    if (n_results) *n_results = count < max_results ? count : max_results;
    if (rc != GS_OK) {
        ctx->binning = keep_bin; ctx->sort_bits = keep_bits; ctx->sort_items = keep_items;
        ctx->raster_tpr = keep_tpr; ctx->raster_bwd_tpr = keep_btpr;
        return rc;
    }
    // a layout never timed (8-px tiles) keeps -1 and loses
    auto best_of = [](const float (&t)[2]) { return (t[1] >= 0.f && t[1] < t[0]) ? 1 : 0; };
    float total[2];
    for (int ib = 0; ib < 2; ++ib)
        total[ib] = best_pre[ib] + best_fwd[ib][best_of(best_fwd[ib])] + best_bwd[ib][best_of(best_bwd[ib])];
    const int b = total[1] < total[0] ? 1 : 0;
    ctx->binning = bins[b]; ctx->sort_bits = bbits[b]; ctx->sort_items = bitems[b];
    ctx->raster_tpr = tprs[best_of(best_fwd[b])];
    ctx->raster_bwd_tpr = tprs[best_of(best_bwd[b])];
    return launch_check();
}

gs_status_t gs_light_depth_map(gs_ctx* ctx, const gs_scene* scene, const gs_light_camera* lcam, float* depth,
                               int32_t accumulate, void* stream) {
    if (!ctx || !scene || !depth || bad_light_cam(lcam) || scene->n < 0 || (scene->n > 0 && !scene->params) ||
        bad_dyn(scene->dyn))
        return GS_ERR_ARG;
    DeviceGuard g(ctx->device);
    launch_light_depth(scene->params, scene->n, make_dyn(scene->dyn), *lcam, depth, accumulate ? 0 : 1, S(stream));
    return launch_check();
}

gs_status_t gs_light_visibility(gs_ctx* ctx, const gs_scene* scene, const gs_light_camera* lcam,
                                const float* depth, uint8_t* visibility, void* stream) {
    if (!ctx || !scene || !depth || bad_light_cam(lcam) || scene->n < 0 ||
        (scene->n > 0 && (!scene->params || !visibility)) || bad_dyn(scene->dyn))
        return GS_ERR_ARG;
    if (scene->n == 0) return GS_OK;
    DeviceGuard g(ctx->device);
    launch_light_visibility(scene->params, scene->n, make_dyn(scene->dyn), *lcam, depth, visibility, S(stream));
    return launch_check();
}

size_t gs_precull_workspace_size(const gs_camera* host_cams, int32_t n_views) {
    if (!host_cams || bad_views(n_views)) return 0;
    return precull_scratch_bytes(host_cams, n_views) + 4096;
}

gs_status_t gs_cell_visibility(gs_ctx* ctx, const gs_camera* d_cams, const gs_camera* host_cams, int32_t n_views,
                               const float* d_depth, const gs_precull* grid, uint8_t* d_cell_visible,
                               void* stream) {
    if (!ctx || !d_cams || !host_cams || bad_views(n_views) || !d_depth || !grid || !d_cell_visible ||
        !(grid->cell_size > 0.f) || grid->dims[0] < 1 || grid->dims[1] < 1 || grid->dims[2] < 1 ||
        (int64_t)grid->dims[0] * grid->dims[1] * grid->dims[2] >= (1LL << 40))
        return GS_ERR_ARG;
    for (int v = 0; v < n_views; ++v)
        if (host_cams[v].width < 1 || host_cams[v].height < 1) return GS_ERR_ARG;
    if (check_ws(ctx, precull_scratch_bytes(host_cams, n_views))) return GS_ERR_CAPACITY;
    DeviceGuard g(ctx->device);
    launch_cell_visibility(d_cams, host_cams, n_views, d_depth, *grid, d_cell_visible,
                           static_cast<char*>(ctx->ws), S(stream));
    return launch_check();
}

gs_status_t gs_train_graph_capture(gs_ctx* ctx, const gs_camera* d_cams, const gs_train_io* io,
                                   const gs_train_cfg* cfg, void* stream) {
    return gs_train_graph_capture_events(ctx, d_cams, io, cfg, nullptr, stream);
}

gs_status_t gs_train_graph_capture_events(gs_ctx* ctx, const gs_camera* d_cams, const gs_train_io* io,
                                          const gs_train_cfg* cfg, void* const* events, void* stream) {
    if (!ctx) return GS_ERR_ARG;
    DeviceGuard g(ctx->device);
    if (cudaStreamSynchronize(S(stream)) != cudaSuccess) return GS_ERR_CUDA;
    if (ctx->graph_exec) { cudaGraphExecDestroy(ctx->graph_exec); ctx->graph_exec = nullptr; }
    if (ctx->graph) { cudaGraphDestroy(ctx->graph); ctx->graph = nullptr; }
    if (cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return GS_ERR_CUDA;
    const gs_status_t s = gs_train_step_events(ctx, d_cams, io, cfg, events, ctx->capture_stream);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(ctx->capture_stream, &graph);
    if (s != GS_OK) {
        if (graph) cudaGraphDestroy(graph);
        return s;
    }
    if (e != cudaSuccess || !graph) return GS_ERR_CUDA;
    if (cudaGraphInstantiate(&ctx->graph_exec, graph, 0) != cudaSuccess) {
        cudaGraphDestroy(graph);
        return GS_ERR_CUDA;
    }
    ctx->graph = graph;
    return GS_OK;
}

gs_status_t gs_graph_launch(gs_ctx* ctx, void* stream) {
    if (!ctx || !ctx->graph_exec) return GS_ERR_ARG;
    DeviceGuard g(ctx->device);
    return cudaGraphLaunch(ctx->graph_exec, S(stream)) == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

}  // extern "C"
