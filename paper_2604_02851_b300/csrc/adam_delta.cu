// Adam update and changed-set extraction for the incremental stream.
//
// Adam: Sec. 3.1 ("updates the trainable Gaussian parameters using the
// configured loss and learning rates"), Sec. 3.3 (optimiser state is rebuilt
// or extended with the model).  Bias-corrected Adam, one float4 per thread,
// learning rate per element of a Gaussian's 60 floats.
//
// Delta: Sec. 3.5 -- between snapshots the server sends tensor-delta packets,
// with residuals against the previously transmitted state and fresh baselines
// after a snapshot.  A Gaussian is sent when any of its 60 floats moved by
// more than thr from its last transmitted value; the sent set is compacted in
// index order (block sums, one-block scan, ordered emit) and packed as
// 128-byte records: uint32 index, float32 mean, 56 float16 (RNE) attributes.
#include <cuda_fp16.h>
#include <math.h>

#include "gs_internal.cuh"

namespace gs {
namespace {

struct LrTable { float lr[60]; };

// One bias-corrected Adam update of a float4 of parameters (learning rates
// l[0..3]); bc1 = 1 - b1^t, sbc2 = sqrt(1 - b2^t).
__device__ __forceinline__ void adam4(float4& th, float4& mm, float4& vv, const float4 g, const float* l, float b1,
                                      float b2, float eps, float bc1, float sbc2) {
#define ADAM_LANE(c, k)                                                   \
    mm.c = b1 * mm.c + (1.f - b1) * g.c;                                  \
    vv.c = b2 * vv.c + (1.f - b2) * g.c * g.c;                            \
    th.c -= (l[k] / bc1) * mm.c / (sqrtf(vv.c) / sbc2 + eps);
    ADAM_LANE(x, 0)
    ADAM_LANE(y, 1)
    ADAM_LANE(z, 2)
    ADAM_LANE(w, 3)
#undef ADAM_LANE
}

__global__ void __launch_bounds__(256)
k_adam(float4* __restrict__ theta, const float4* __restrict__ grad, float4* __restrict__ m,
       float4* __restrict__ v, int64_t n, LrTable lr, float b1, float b2, float eps, int host_step,
       const int32_t* __restrict__ d_step, const uint8_t* __restrict__ fwd) {
    const int step = d_step ? *d_step : host_step;
    const float bc1 = 1.f - powf(b1, (float)step);
    const float bc2 = 1.f - powf(b2, (float)step);
    const float sbc2 = sqrtf(bc2);
    const int64_t total = 15 * n;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int plane = (int)(i / n);
        if (fwd && !fwd[i - (int64_t)plane * n]) continue;  // preculled: no update
        const float4 g = grad[i];
        float4 mm = m[i], vv = v[i], th = theta[i];
        adam4(th, mm, vv, g, lr.lr + 4 * plane, b1, b2, eps, bc1, sbc2);
        m[i] = mm;
        v[i] = vv;
        theta[i] = th;
    }
}

__global__ void k_inc_step(int32_t* d_step) { *d_step += 1; }

// ---------------------------------------------------------------- delta
constexpr int kDeltaThreads = 256;

__global__ void __launch_bounds__(kDeltaThreads)
k_delta_flags(const float4* __restrict__ theta, const float4* __restrict__ base, int64_t n, float thr,
              uint8_t* __restrict__ flags, uint32_t* __restrict__ block_sums) {
    const int64_t g = (int64_t)blockIdx.x * kDeltaThreads + threadIdx.x;
    uint32_t changed = 0;
    if (g < n) {
#pragma unroll
        for (int p = 0; p < 15; ++p) {
            const float4 a = theta[p * n + g], b = base[p * n + g];
            const float m = fmaxf(fmaxf(fabsf(a.x - b.x), fabsf(a.y - b.y)), fmaxf(fabsf(a.z - b.z), fabsf(a.w - b.w)));
            changed |= (m > thr) ? 1u : 0u;
        }
        flags[g] = (uint8_t)changed;
    }
    const uint32_t cnt = __syncthreads_count(changed);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = cnt;
}

// The training step's Adam update fused with the changed test of the delta
// extraction: one thread per Gaussian walks its 15 planes, updates them and
// compares the new values with the baseline, so that the parameters are read
// once.  Same arithmetic as k_adam and k_delta_flags.  Six blocks an SM (40
// registers, the learning rates in shared memory) keep enough loads in
// flight; unrolling the plane loop, or 5 and 8 blocks, measured slower.
__global__ void __launch_bounds__(kDeltaThreads, 6)
k_adam_flags(float4* __restrict__ theta, const float4* __restrict__ grad, float4* __restrict__ m,
             float4* __restrict__ v, const float4* __restrict__ base, int64_t n, LrTable lr, float b1, float b2,
             float eps, int host_step, const int32_t* __restrict__ d_step, const uint8_t* __restrict__ fwd,
             float thr, uint8_t* __restrict__ flags, uint32_t* __restrict__ block_sums) {
    __shared__ float s_lr[60];
    if (threadIdx.x < 60) s_lr[threadIdx.x] = lr.lr[threadIdx.x];
    __syncthreads();
    const int step = d_step ? *d_step : host_step;
    const float bc1 = 1.f - powf(b1, (float)step);
    const float sbc2 = sqrtf(1.f - powf(b2, (float)step));
    const int64_t g = (int64_t)blockIdx.x * kDeltaThreads + threadIdx.x;
    uint32_t changed = 0;
    if (g < n) {
        const bool upd = !fwd || fwd[g];  // preculled: no update
#pragma unroll 1
        for (int p = 0; p < 15; ++p) {
            const int64_t i = p * n + g;
            float4 th = theta[i];
            const float4 b = base[i];
            if (upd) {
                const float4 gr = grad[i];
                float4 mm = m[i], vv = v[i];
                adam4(th, mm, vv, gr, s_lr + 4 * p, b1, b2, eps, bc1, sbc2);
                m[i] = mm;
                v[i] = vv;
                theta[i] = th;
            }
            const float d = fmaxf(fmaxf(fabsf(th.x - b.x), fabsf(th.y - b.y)), fmaxf(fabsf(th.z - b.z), fabsf(th.w - b.w)));
            changed |= (d > thr) ? 1u : 0u;
        }
        flags[g] = (uint8_t)changed;
    }
    const uint32_t cnt = __syncthreads_count(changed);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = cnt;
}

__global__ void __launch_bounds__(kDeltaThreads)
k_delta_emit(const float4* __restrict__ theta, float4* __restrict__ base, int64_t n,
             const uint8_t* __restrict__ flags, const uint32_t* __restrict__ block_off,
             uint32_t* __restrict__ d_idx, uint8_t* __restrict__ d_records) {
    const int64_t g = (int64_t)blockIdx.x * kDeltaThreads + threadIdx.x;
    const bool ch = g < n && flags[g];
    const uint32_t ballot = __ballot_sync(0xFFFFFFFFu, ch);
    __shared__ uint32_t s_w[kDeltaThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) s_w[warp] = __popc(ballot);
    __syncthreads();
    uint32_t off = block_off[blockIdx.x];
    for (int w = 0; w < warp; ++w) off += s_w[w];
    off += __popc(ballot & ((1u << lane) - 1u));
    if (!ch) return;
    d_idx[off] = (uint32_t)g;
    float t[60];
#pragma unroll
    for (int p = 0; p < 15; ++p) {
        const float4 a = theta[p * n + g];
        t[4 * p] = a.x; t[4 * p + 1] = a.y; t[4 * p + 2] = a.z; t[4 * p + 3] = a.w;
        base[p * n + g] = a;
    }
    // record: [0] index, [1..3] mean, then float16: log-scale (4..6),
    // quaternion (8..11), opacity logit (3), SH (12..59)
    uint32_t w[32];
    w[0] = (uint32_t)g;
    w[1] = __float_as_uint(t[0]);
    w[2] = __float_as_uint(t[1]);
    w[3] = __float_as_uint(t[2]);
    uint16_t h[56];
    int k = 0;
#pragma unroll
    for (int i = 4; i < 7; ++i) h[k++] = __half_as_ushort(__float2half_rn(t[i]));
#pragma unroll
    for (int i = 8; i < 12; ++i) h[k++] = __half_as_ushort(__float2half_rn(t[i]));
    h[k++] = __half_as_ushort(__float2half_rn(t[3]));
#pragma unroll
    for (int i = 12; i < 60; ++i) h[k++] = __half_as_ushort(__float2half_rn(t[i]));
#pragma unroll
    for (int i = 0; i < 28; ++i) w[4 + i] = (uint32_t)h[2 * i] | ((uint32_t)h[2 * i + 1] << 16);
    uint4* rec = reinterpret_cast<uint4*>(d_records + (size_t)off * 128);
#pragma unroll
    for (int i = 0; i < 8; ++i) rec[i] = make_uint4(w[4 * i], w[4 * i + 1], w[4 * i + 2], w[4 * i + 3]);
}

// ---------------------------------------------------------------- tensor deltas
// One attribute group of the 60 floats of a Gaussian (flat indices [lo, hi),
// planes lo/4 .. (hi-1)/4), sent as float32 (mean) or float16 RNE.
struct Group {
    int lo, hi, f32;
};

__device__ __forceinline__ float lane_of(const float4& a, int l) {
    return l == 0 ? a.x : (l == 1 ? a.y : (l == 2 ? a.z : a.w));
}
__device__ __forceinline__ void set_lane(float4& a, int l, float v) {
    if (l == 0) a.x = v; else if (l == 1) a.y = v; else if (l == 2) a.z = v; else a.w = v;
}

__global__ void __launch_bounds__(kDeltaThreads)
k_tdelta_flags(const float4* __restrict__ theta, const float4* __restrict__ base, int64_t n, Group gr, float thr,
               uint8_t* __restrict__ flags, uint32_t* __restrict__ block_sums) {
    const int64_t g = (int64_t)blockIdx.x * kDeltaThreads + threadIdx.x;
    uint32_t changed = 0;
    if (g < n) {
        for (int p = gr.lo >> 2; p <= (gr.hi - 1) >> 2; ++p) {
            const float4 a = theta[p * n + g], b = base[p * n + g];
#pragma unroll
            for (int l = 0; l < 4; ++l) {
                const int f = 4 * p + l;
                if (f >= gr.lo && f < gr.hi && fabsf(lane_of(a, l) - lane_of(b, l)) > thr) changed = 1u;
            }
        }
        flags[g] = (uint8_t)changed;
    }
    const uint32_t cnt = __syncthreads_count(changed);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = cnt;
}

__global__ void __launch_bounds__(kDeltaThreads)
k_tdelta_emit(const float4* __restrict__ theta, float4* __restrict__ base, int64_t n, Group gr,
              const uint8_t* __restrict__ flags, const uint32_t* __restrict__ block_off,
              uint32_t* __restrict__ d_idx, uint8_t* __restrict__ d_vals) {
    const int64_t g = (int64_t)blockIdx.x * kDeltaThreads + threadIdx.x;
    const bool ch = g < n && flags[g];
    const uint32_t ballot = __ballot_sync(0xFFFFFFFFu, ch);
    __shared__ uint32_t s_w[kDeltaThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) s_w[warp] = __popc(ballot);
    __syncthreads();
    uint32_t off = block_off[blockIdx.x];
    for (int w = 0; w < warp; ++w) off += s_w[w];
    off += __popc(ballot & ((1u << lane) - 1u));
    if (!ch) return;
    d_idx[off] = (uint32_t)g;
    const int rb = (gr.hi - gr.lo) * (gr.f32 ? 4 : 2);
    uint8_t* rec = d_vals + (size_t)off * rb;
    for (int p = gr.lo >> 2; p <= (gr.hi - 1) >> 2; ++p) {
        const float4 a = theta[p * n + g];
        float4 b = base[p * n + g];
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            const int f = 4 * p + l;
            if (f < gr.lo || f >= gr.hi) continue;
            const float v = lane_of(a, l);
            if (gr.f32) reinterpret_cast<float*>(rec)[f - gr.lo] = v;
            else reinterpret_cast<__half*>(rec)[f - gr.lo] = __float2half_rn(v);
            set_lane(b, l, v);
        }
        base[p * n + g] = b;
    }
}

// Client-side replay: decoded values of the first *d_count records into
// the params planes; an index >= n records GS_ERR_ARG and is skipped.
__global__ void __launch_bounds__(256)
k_apply_tdelta(float4* __restrict__ params, int64_t n, Group gr, const uint32_t* __restrict__ d_idx,
               const uint8_t* __restrict__ d_vals, const uint32_t* __restrict__ d_count, DevStatus* status) {
    const int64_t m = *d_count;
    const int rb = (gr.hi - gr.lo) * (gr.f32 ? 4 : 2);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t g = d_idx[i];
        if ((int64_t)g >= n) { record_status(status, GS_ERR_ARG, (long long)g); continue; }
        const uint8_t* rec = d_vals + (size_t)i * rb;
        for (int p = gr.lo >> 2; p <= (gr.hi - 1) >> 2; ++p) {
            float4 a = params[p * n + g];
#pragma unroll
            for (int l = 0; l < 4; ++l) {
                const int f = 4 * p + l;
                if (f < gr.lo || f >= gr.hi) continue;
                const float v = gr.f32 ? reinterpret_cast<const float*>(rec)[f - gr.lo]
                                       : __half2float(reinterpret_cast<const __half*>(rec)[f - gr.lo]);
                set_lane(a, l, v);
            }
            params[p * n + g] = a;
        }
    }
}

// Replay of the full 128-byte records (gs_extract_delta's layout).
__global__ void __launch_bounds__(256)
k_apply_delta(float4* __restrict__ params, int64_t n, const uint4* __restrict__ recs,
              const uint32_t* __restrict__ d_count, DevStatus* status) {
    const int64_t m = *d_count;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t w[32];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const uint4 u = recs[i * 8 + q];
            w[4 * q] = u.x; w[4 * q + 1] = u.y; w[4 * q + 2] = u.z; w[4 * q + 3] = u.w;
        }
        const uint32_t g = w[0];
        if ((int64_t)g >= n) { record_status(status, GS_ERR_ARG, (long long)g); continue; }
        float h[56];
#pragma unroll
        for (int k = 0; k < 28; ++k) {
            h[2 * k] = __half2float(__ushort_as_half((unsigned short)(w[4 + k] & 0xFFFFu)));
            h[2 * k + 1] = __half2float(__ushort_as_half((unsigned short)(w[4 + k] >> 16)));
        }
        // h: log-scale (3), quaternion (4), opacity logit (1), SH (48)
        params[g] = make_float4(__uint_as_float(w[1]), __uint_as_float(w[2]), __uint_as_float(w[3]), h[7]);
        float4 sc = params[n + g];
        sc.x = h[0]; sc.y = h[1]; sc.z = h[2];
        params[n + g] = sc;
        params[2 * n + g] = make_float4(h[3], h[4], h[5], h[6]);
#pragma unroll
        for (int p = 0; p < 12; ++p)
            params[(3 + p) * n + g] = make_float4(h[8 + 4 * p], h[9 + 4 * p], h[10 + 4 * p], h[11 + 4 * p]);
    }
}

// ---------------------------------------------------------------- scan
__global__ void __launch_bounds__(1024)
k_scan_sums(uint32_t* sums, int64_t count, uint32_t* d_total, long long cap, DevStatus* status) {
    __shared__ uint32_t s_w[32];
    __shared__ unsigned long long s_carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < count; base += 1024) {
        const int64_t i = base + threadIdx.x;
        const uint32_t x = i < count ? sums[i] : 0u;
        uint32_t incl = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) s_w[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            uint32_t w = s_w[lane];
            uint32_t wi = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, wi, o);
                if (lane >= o) wi += y;
            }
            s_w[lane] = wi - w;
        }
        __syncthreads();
        const unsigned long long carry = s_carry;
        if (i < count) sums[i] = (uint32_t)(carry + s_w[warp] + incl - x);
        __syncthreads();
        if (threadIdx.x == 1023) s_carry = carry + s_w[warp] + incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const unsigned long long total = s_carry;
        *d_total = (uint32_t)(total > 0xFFFFFFFFull ? 0xFFFFFFFFull : total);
        if (cap >= 0 && (long long)total > cap) record_status(status, GS_ERR_CAPACITY, (long long)total);
    }
}

}  // namespace

void launch_scan_sums(uint32_t* sums, int64_t count, uint32_t* d_total, long long cap, DevStatus* status,
                      cudaStream_t st) {
    k_scan_sums<<<1, 1024, 0, st>>>(sums, count, d_total, cap, status);
}

void launch_adam(float* theta, const float* grad, float* m, float* v, int64_t n, const gs_adam_cfg& cfg,
                 cudaStream_t st, const uint8_t* fwd) {
    if (n > 0) {
        LrTable lr;
        for (int i = 0; i < 60; ++i) lr.lr[i] = cfg.lr[i];
        const int64_t total = 15 * n;
        int64_t blocks = (total + 255) / 256;
        if (blocks > 148 * 16) blocks = 148 * 16;
        k_adam<<<(unsigned)blocks, 256, 0, st>>>(
            reinterpret_cast<float4*>(theta), reinterpret_cast<const float4*>(grad),
            reinterpret_cast<float4*>(m), reinterpret_cast<float4*>(v), n, lr, cfg.beta1, cfg.beta2,
            cfg.eps, cfg.step, cfg.d_step, fwd);
    }
    if (cfg.d_step && cfg.increment) k_inc_step<<<1, 1, 0, st>>>(const_cast<int32_t*>(cfg.d_step));
}

size_t delta_scratch_bytes(int64_t n) {
    Carver c(nullptr);
    c.take<uint8_t>(n > 0 ? n : 1);
    c.take<uint32_t>((n + kDeltaThreads - 1) / kDeltaThreads + 1);
    return c.off;
}

void launch_delta(const float* theta, float* baseline, int64_t n, float thr, uint32_t* d_idx,
                  uint8_t* d_records, uint32_t* d_count, char* scratch, cudaStream_t st) {
    Carver c(scratch);
    uint8_t* flags = c.take<uint8_t>(n > 0 ? n : 1);
    const int64_t nblk = (n + kDeltaThreads - 1) / kDeltaThreads;
    uint32_t* sums = c.take<uint32_t>(nblk + 1);
    if (n <= 0) {
        cudaMemsetAsync(d_count, 0, sizeof(uint32_t), st);
        return;
    }
    const float4* th = reinterpret_cast<const float4*>(theta);
    float4* b = reinterpret_cast<float4*>(baseline);
    k_delta_flags<<<(unsigned)nblk, kDeltaThreads, 0, st>>>(th, b, n, thr, flags, sums);
    k_scan_sums<<<1, 1024, 0, st>>>(sums, nblk, d_count, -1, nullptr);
    k_delta_emit<<<(unsigned)nblk, kDeltaThreads, 0, st>>>(th, b, n, flags, sums, d_idx, d_records);
}

void launch_adam_delta(float* theta, const float* grad, float* m, float* v, int64_t n, const gs_adam_cfg& cfg,
                       const uint8_t* fwd, float* baseline, float thr, uint32_t* d_idx, uint8_t* d_records,
                       uint32_t* d_count, char* scratch, cudaStream_t st, void (*mark)(void* const*, int, cudaStream_t),
                       void* const* events, int event) {
    Carver c(scratch);
    uint8_t* flags = c.take<uint8_t>(n > 0 ? n : 1);
    const int64_t nblk = (n + kDeltaThreads - 1) / kDeltaThreads;
    uint32_t* sums = c.take<uint32_t>(nblk + 1);
    if (n > 0) {
        LrTable lr;
        for (int i = 0; i < 60; ++i) lr.lr[i] = cfg.lr[i];
        k_adam_flags<<<(unsigned)nblk, kDeltaThreads, 0, st>>>(
            reinterpret_cast<float4*>(theta), reinterpret_cast<const float4*>(grad), reinterpret_cast<float4*>(m),
            reinterpret_cast<float4*>(v), reinterpret_cast<const float4*>(baseline), n, lr, cfg.beta1, cfg.beta2,
            cfg.eps, cfg.step, cfg.d_step, fwd, thr, flags, sums);
    }
    if (cfg.d_step && cfg.increment) k_inc_step<<<1, 1, 0, st>>>(const_cast<int32_t*>(cfg.d_step));
    if (mark) mark(events, event, st);
    if (n <= 0) {
        cudaMemsetAsync(d_count, 0, sizeof(uint32_t), st);
        return;
    }
    k_scan_sums<<<1, 1024, 0, st>>>(sums, nblk, d_count, -1, nullptr);
    k_delta_emit<<<(unsigned)nblk, kDeltaThreads, 0, st>>>(reinterpret_cast<const float4*>(theta),
                                                          reinterpret_cast<float4*>(baseline), n, flags, sums, d_idx,
                                                          d_records);
}

bool attr_group(int attr, int* lo, int* hi, int* f32) {
    switch (attr) {
        case GS_ATTR_MEAN: *lo = 0; *hi = 3; *f32 = 1; return true;
        case GS_ATTR_OPACITY: *lo = 3; *hi = 4; *f32 = 0; return true;
        case GS_ATTR_SCALE: *lo = 4; *hi = 7; *f32 = 0; return true;
        case GS_ATTR_ROTATION: *lo = 8; *hi = 12; *f32 = 0; return true;
        case GS_ATTR_DC: *lo = 12; *hi = 15; *f32 = 0; return true;
        case GS_ATTR_SH_REST: *lo = 15; *hi = 60; *f32 = 0; return true;
        default: return false;
    }
}

void launch_tensor_delta(const float* theta, float* baseline, int64_t n, int attr, float thr, uint32_t* d_idx,
                         uint8_t* d_vals, uint32_t* d_count, char* scratch, cudaStream_t st) {
    Group gr;
    attr_group(attr, &gr.lo, &gr.hi, &gr.f32);
    Carver c(scratch);
    uint8_t* flags = c.take<uint8_t>(n > 0 ? n : 1);
    const int64_t nblk = (n + kDeltaThreads - 1) / kDeltaThreads;
    uint32_t* sums = c.take<uint32_t>(nblk + 1);
    if (n <= 0) {
        cudaMemsetAsync(d_count, 0, sizeof(uint32_t), st);
        return;
    }
    const float4* th = reinterpret_cast<const float4*>(theta);
    float4* b = reinterpret_cast<float4*>(baseline);
    k_tdelta_flags<<<(unsigned)nblk, kDeltaThreads, 0, st>>>(th, b, n, gr, thr, flags, sums);
    k_scan_sums<<<1, 1024, 0, st>>>(sums, nblk, d_count, -1, nullptr);
    k_tdelta_emit<<<(unsigned)nblk, kDeltaThreads, 0, st>>>(th, b, n, gr, flags, sums, d_idx, d_vals);
}

void launch_apply_tensor_delta(float* params, int64_t n, int attr, const uint32_t* d_idx, const uint8_t* d_vals,
                               const uint32_t* d_count, DevStatus* status, int sm_count, cudaStream_t st) {
    Group gr;
    attr_group(attr, &gr.lo, &gr.hi, &gr.f32);
    k_apply_tdelta<<<(unsigned)(sm_count * 4), 256, 0, st>>>(reinterpret_cast<float4*>(params), n, gr, d_idx, d_vals,
                                                              d_count, status);
}

void launch_apply_delta(float* params, int64_t n, const uint8_t* d_records, const uint32_t* d_count,
                        DevStatus* status, int sm_count, cudaStream_t st) {
    k_apply_delta<<<(unsigned)(sm_count * 4), 256, 0, st>>>(reinterpret_cast<float4*>(params), n,
                                                             reinterpret_cast<const uint4*>(d_records), d_count,
                                                             status);
}

}  // namespace gs
