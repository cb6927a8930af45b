// EWA projection with spherical-harmonics colour, and its adjoint.
//
// Sec. 3.2.3: the model is refined by differentiable rendering of "the same
// parameters as in prior 3DGS work" (means, scales, rotations, opacities, SH
// coefficients -- Sec. 3.1); Sec. 3.2.2 / 3.4.1: appearance is a diffuse SH
// representation of degree <= 3.
//
// One thread owns one Gaussian: its 60 parameters are read once (coalesced
// float4 planes) and every view is projected from registers, so the model is
// read from HBM once per step however many reference views there are.
#include "gauss.cuh"

namespace gs {
namespace {

// Geometry of one Gaussian in one view; returns false when culled by the
// near plane or a non-positive 2D determinant.
struct ViewGeom {
    float tx, ty, tz;
    float xt, yt;        // guard-band clamped t_x, t_y used in J
    int clx, cly;
    float limx, limy;
    float J00, J02, J11, J12;
    float M0[3], M1[3];  // rows of J W
    float a, b, c, det;
    float3 dir;
    float len;
    float iz;            // 1 / t_z
};

__device__ __forceinline__ bool view_geom(const Gauss& G, const Cam& C, ViewGeom& V) {
    const float* W = C.R;
    V.tx = W[0] * G.mu.x + W[1] * G.mu.y + W[2] * G.mu.z + C.t[0];
    V.ty = W[3] * G.mu.x + W[4] * G.mu.y + W[5] * G.mu.z + C.t[1];
    V.tz = W[6] * G.mu.x + W[7] * G.mu.y + W[8] * G.mu.z + C.t[2];
    if (!(V.tz > C.near)) return false;
    V.limx = kGuard * ((float)C.W / (2.f * C.fx));
    V.limy = kGuard * ((float)C.H / (2.f * C.fy));
    const float iz = 1.f / V.tz, iz2 = iz * iz;
    V.iz = iz;
    const float rx = V.tx * iz, ry = V.ty * iz;
    V.clx = rx < -V.limx ? -1 : (rx > V.limx ? 1 : 0);
    V.cly = ry < -V.limy ? -1 : (ry > V.limy ? 1 : 0);
    V.xt = fminf(fmaxf(rx, -V.limx), V.limx) * V.tz;
    V.yt = fminf(fmaxf(ry, -V.limy), V.limy) * V.tz;
    V.J00 = C.fx * iz;
    V.J02 = -C.fx * V.xt * iz2;
    V.J11 = C.fy * iz;
    V.J12 = -C.fy * V.yt * iz2;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        V.M0[i] = V.J00 * W[i] + V.J02 * W[6 + i];
        V.M1[i] = V.J11 * W[3 + i] + V.J12 * W[6 + i];
    }
    const float* S = G.S;
    const float SM0x = S[0] * V.M0[0] + S[1] * V.M0[1] + S[2] * V.M0[2];
    const float SM0y = S[1] * V.M0[0] + S[3] * V.M0[1] + S[4] * V.M0[2];
    const float SM0z = S[2] * V.M0[0] + S[4] * V.M0[1] + S[5] * V.M0[2];
    const float SM1x = S[0] * V.M1[0] + S[1] * V.M1[1] + S[2] * V.M1[2];
    const float SM1y = S[1] * V.M1[0] + S[3] * V.M1[1] + S[4] * V.M1[2];
    const float SM1z = S[2] * V.M1[0] + S[4] * V.M1[1] + S[5] * V.M1[2];
    V.a = V.M0[0] * SM0x + V.M0[1] * SM0y + V.M0[2] * SM0z + kDilation;
    V.b = V.M0[0] * SM1x + V.M0[1] * SM1y + V.M0[2] * SM1z;
    V.c = V.M1[0] * SM1x + V.M1[1] * SM1y + V.M1[2] * SM1z + kDilation;
    V.det = V.a * V.c - V.b * V.b;
    if (!(V.det > 0.f)) return false;
    // camera centre = -W^T t
    const float cx = -(W[0] * C.t[0] + W[3] * C.t[1] + W[6] * C.t[2]);
    const float cy = -(W[1] * C.t[0] + W[4] * C.t[1] + W[7] * C.t[2]);
    const float cz = -(W[2] * C.t[0] + W[5] * C.t[1] + W[8] * C.t[2]);
    const float dx = G.mu.x - cx, dy = G.mu.y - cy, dz = G.mu.z - cz;
    V.len = sqrtf(dx * dx + dy * dy + dz * dz);
    const float il = 1.f / V.len;
    V.dir = make_float3(dx * il, dy * il, dz * il);
    return true;
}

// Tile rectangle of the square of half-side r around (u, v).  The clamp is
// applied in float before the conversion so that huge coordinates stay safe.
// The tile size is a power of two (8 or 16), so multiplying by its reciprocal
// is the exact quotient.
__device__ __forceinline__ void tile_rect(float u, float v, float r, int TX, int TY, int tile,
                                          int& x0, int& y0, int& x1, int& y1) {
    const float ft = (float)tile, ift = 1.f / ft;
    x0 = (int)fminf(fmaxf(floorf((u - r) * ift), 0.f), (float)TX);
    y0 = (int)fminf(fmaxf(floorf((v - r) * ift), 0.f), (float)TY);
    x1 = (int)fminf(fmaxf(floorf((u + r + ft - 1.f) * ift), 0.f), (float)TX);
    y1 = (int)fminf(fmaxf(floorf((v + r + ft - 1.f) * ift), 0.f), (float)TY);
}

// ------------------------------------------------------------ relighting
// Per-group relighting table (Sec. 3.4.1).  The environment seen from the
// object's frame is Lenv'(w) = Lenv(R_g w); rotation keeps each SH band, so
// band l of e' is the least-squares fit of Lenv restricted to band l, sampled
// at R_g w_j, over the band's basis at 20 spiral directions w_j (the fit is
// exact: the rotated band lies in the band's span; its normal matrices have
// condition numbers below 2).  The directional light enters as
// E_c Y_k(R_g^T l).  One thread per group; float32 throughout.
constexpr int kFitDirs = 20;

__device__ __forceinline__ void spiral_dir(int j, float* w) {
    const float z = 1.f - (2.f * j + 1.f) / (float)kFitDirs;
    const float r = sqrtf(fmaxf(0.f, 1.f - z * z));
    float sn, cs;
    sincosf(2.3999632297286533f * (float)j, &sn, &cs);  // golden angle
    w[0] = r * cs; w[1] = r * sn; w[2] = z;
}

__global__ void k_light_table(Dyn d, const float* __restrict__ light, float* __restrict__ tab, int G) {
    const int grp = blockIdx.x * blockDim.x + threadIdx.x;
    if (grp >= G) return;
    float R[9] = {1.f, 0.f, 0.f, 0.f, 1.f, 0.f, 0.f, 0.f, 1.f};
    if (d.group) {
        const float4 q = d.poses[2 * grp];
        quat_rot(q.x, q.y, q.z, q.w, R);
    }
    float* out = tab + (size_t)grp * kLitTab;
    for (int c = 0; c < 3; ++c) out[c] = light[c];  // band 0 is rotation invariant
    for (int l = 1; l <= 3; ++l) {
        const int nb = 2 * l + 1, o = l * l;
        float M[7][7], rhs[7][3];
        for (int a = 0; a < nb; ++a) {
            for (int b = 0; b < nb; ++b) M[a][b] = 0.f;
            rhs[a][0] = rhs[a][1] = rhs[a][2] = 0.f;
        }
        for (int j = 0; j < kFitDirs; ++j) {
            float w[3], Y[16], Yr[16];
            spiral_dir(j, w);
            sh_basis<3>(w[0], w[1], w[2], Y);
            sh_basis<3>(R[0] * w[0] + R[1] * w[1] + R[2] * w[2], R[3] * w[0] + R[4] * w[1] + R[5] * w[2],
                        R[6] * w[0] + R[7] * w[1] + R[8] * w[2], Yr);
            float Lb[3] = {0.f, 0.f, 0.f};
            for (int m = 0; m < nb; ++m)
                for (int c = 0; c < 3; ++c) Lb[c] += light[3 * (o + m) + c] * Yr[o + m];
            for (int a = 0; a < nb; ++a) {
                for (int b = 0; b < nb; ++b) M[a][b] += Y[o + a] * Y[o + b];
                for (int c = 0; c < 3; ++c) rhs[a][c] += Y[o + a] * Lb[c];
            }
        }
        // Gaussian elimination with partial pivoting
        for (int col = 0; col < nb; ++col) {
            int piv = col;
            for (int r = col + 1; r < nb; ++r)
                if (fabsf(M[r][col]) > fabsf(M[piv][col])) piv = r;
            if (piv != col) {
                for (int b = 0; b < nb; ++b) { const float t = M[col][b]; M[col][b] = M[piv][b]; M[piv][b] = t; }
                for (int c = 0; c < 3; ++c) { const float t = rhs[col][c]; rhs[col][c] = rhs[piv][c]; rhs[piv][c] = t; }
            }
            const float inv = 1.f / M[col][col];
            for (int r = col + 1; r < nb; ++r) {
                const float f = M[r][col] * inv;
                for (int b = col; b < nb; ++b) M[r][b] -= f * M[col][b];
                for (int c = 0; c < 3; ++c) rhs[r][c] -= f * rhs[col][c];
            }
        }
        for (int r = nb - 1; r >= 0; --r)
            for (int c = 0; c < 3; ++c) {
                float acc = rhs[r][c];
                for (int b = r + 1; b < nb; ++b) acc -= M[r][b] * out[3 * (o + b) + c];
                out[3 * (o + r) + c] = acc / M[r][r];
            }
    }
    // directional light in the object frame: R_g^T l
    const float lx = light[48], ly = light[49], lz = light[50];
    float Y[16];
    sh_basis<3>(R[0] * lx + R[3] * ly + R[6] * lz, R[1] * lx + R[4] * ly + R[7] * lz,
                R[2] * lx + R[5] * ly + R[8] * lz, Y);
    for (int k = 0; k < 16; ++k)
        for (int c = 0; c < 3; ++c) out[48 + 3 * k + c] = light[52 + c] * Y[k];
}

// Relit colour of one Gaussian (view-independent): weights w_j = e'_j + v E Y_j.
// lt: the group's table row, in shared or global memory.
template <int NB>
__device__ __forceinline__ void relit_rgb(const float* sh, const float* lt, float v, float* rgb, uint32_t& mask) {
    mask = 0;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < NB; ++k) acc += sh[3 * k + ch] * (lt[3 * k + ch] + v * lt[48 + 3 * k + ch]);
        acc += 0.5f;
        if (acc < 0.f) { acc = 0.f; mask |= 1u << ch; }
        rgb[ch] = acc;
    }
}

__device__ __forceinline__ uint32_t lit_group(const Dyn& d, int64_t g) {
    return d.group ? min((uint32_t)d.group[g], (uint32_t)(d.n_groups - 1)) : 0u;
}

__device__ __forceinline__ const float* lit_row(const Dyn& d, int64_t g) {
    return d.lit_tab + (size_t)lit_group(d, g) * kLitTab;
}

// Groups whose table rows the relit projection stages in shared memory (row
// stride 97 floats: the rows of a warp's groups fall in different banks).
constexpr int kStageGroups = 64;
constexpr int kStageStride = kLitTab + 1;

inline int lit_groups(const Dyn& d) { return d.group ? d.n_groups : 1; }

__device__ __forceinline__ float lit_vis(const Dyn& d, int64_t g) {
    return d.vis ? (float)d.vis[g] * (1.f / 255.f) : 1.f;
}

// Four blocks an SM (64 registers).  View-dependent colour: the coefficients
// wait in shared memory; relit colour: a few spills, measured faster than
// three blocks at 78 registers.  Both measured faster than two blocks with the
// coefficients in 116 registers.
template <int D, bool LIT>
__global__ void __launch_bounds__(256, 4)
k_project(const float4* __restrict__ P, int64_t n, int64_t g_off, int64_t n_out, Dyn dyn,
          const gs_camera* __restrict__ cams, const ViewInfo* __restrict__ vt, int V, int tile,
          float4* __restrict__ proj, uint64_t* __restrict__ dkv, uint2* __restrict__ rects, int rec4,
          uint32_t* __restrict__ drange) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    extern __shared__ float s_lt[];
    bool staged = false;
    if (LIT) {
        const int Gs = dyn.group ? dyn.n_groups : 1;
        staged = Gs <= kStageGroups;
        if (staged) {
            for (int i = threadIdx.x; i < Gs * kLitTab; i += blockDim.x)
                s_lt[(i / kLitTab) * kStageStride + i % kLitTab] = __ldg(&dyn.lit_tab[i]);
            __syncthreads();
        }
    }
    if (g >= n) return;
    constexpr int NB = (D + 1) * (D + 1);
    constexpr int NPL = (3 * NB + 3) / 4;
    const bool rect32 = rects && vt[V].rect32;
    Gauss G;
    load_gauss(P, n, g, G);
    apply_dyn(dyn, g_off + g, G);
    // preculling: the Gaussian takes part only when its (world) cell is kept
    bool kept = true;
    if (dyn.cell_vis) {
        const float pm[3] = {G.mu.x, G.mu.y, G.mu.z};
        int cidx[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float d = (pm[a] - dyn.grid_o[a]) / dyn.grid_size;
            long long k = (long long)floorf(d);
            k = k < 0 ? 0 : (k > dyn.grid_dims[a] - 1 ? dyn.grid_dims[a] - 1 : k);
            cidx[a] = (int)k;
        }
        const int64_t cell = ((int64_t)cidx[2] * dyn.grid_dims[1] + cidx[1]) * dyn.grid_dims[0] + cidx[0];
        kept = dyn.cell_vis[cell] != 0;
        if (dyn.fwd && g_off == 0) dyn.fwd[g] = kept ? 1 : 0;
    }
    // relit colour: the coefficients in registers, used once; view-dependent
    // colour: in shared memory (this thread's column, the DC term scaled),
    // read per view
    float lrgb[3] = {0.f, 0.f, 0.f};
    uint32_t lmask = 0;
    const float tau = 2.f * (logf(G.opac) + 5.5412635f);  // 2 ln(255 o): the alpha >= 1/255 ellipse
    float4* s_sh = reinterpret_cast<float4*>(s_lt);
    if constexpr (!LIT) {
#pragma unroll
        for (int pl = 0; pl < NPL; ++pl) {
            float4 c = P[(3 + pl) * n + g];
            if (pl == 0) { c.x *= G.L; c.y *= G.L; c.z *= G.L; }
            s_sh[pl * blockDim.x + threadIdx.x] = c;
        }
    } else {
        float sh[NPL * 4];
#pragma unroll
        for (int pl = 0; pl < NPL; ++pl) {
            const float4 c = P[(3 + pl) * n + g];
            sh[4 * pl] = c.x; sh[4 * pl + 1] = c.y; sh[4 * pl + 2] = c.z; sh[4 * pl + 3] = c.w;
        }
        sh[0] *= G.L; sh[1] *= G.L; sh[2] *= G.L;
        const float* lt = staged ? s_lt + lit_group(dyn, g_off + g) * kStageStride : lit_row(dyn, g_off + g);
        relit_rgb<NB>(sh, lt, lit_vis(dyn, g_off + g), lrgb, lmask);
    }
    uint32_t klo = 0xFFFFFFFFu, khi = 0u;  // range of this thread's visible depth keys
    for (int v = 0; v < V; ++v) {
        const Cam C = load_cam(cams + v);
        const int64_t rec = (int64_t)v * n_out + g_off + g;
        float4* out = proj + rec * rec4;
        ViewGeom Vg;
        bool ok = kept && view_geom(G, C, Vg);
        float u = 0.f, vv = 0.f, r = 0.f;
        int x0 = 0, y0 = 0, x1 = 0, y1 = 0;
        if (ok) {
            const float mid = 0.5f * (Vg.a + Vg.c);
            const float lam = mid + sqrtf(fmaxf(0.1f, mid * mid - Vg.det));
            r = ceilf(3.f * sqrtf(lam));
            u = C.fx * (Vg.tx * Vg.iz) + C.cx;
            vv = C.fy * (Vg.ty * Vg.iz) + C.cy;
            const ViewInfo vi = vt[v];
            tile_rect(u, vv, r, vi.tx, vi.ty, tile, x0, y0, x1, y1);
            // cut the square down to the tiles of pixel centres inside the
            // box of the ellipse where alpha reaches 1/255 (q <= tau =
            // 2 ln(255 o), half-widths sqrt(tau a), sqrt(tau c)): compositing
            // takes the splat nowhere else, so the image is the square's
            if (tau >= 0.f) {
                const float rx = sqrtf(tau * Vg.a) * 1.001f + 0.01f, ry = sqrtf(tau * Vg.c) * 1.001f + 0.01f;
                const float ift = 1.f / (float)tile;  // exact: the tile size is a power of two
                const int ex0 = (int)fminf(fmaxf(floorf(ceilf(u - rx - 0.5f) * ift), 0.f), (float)vi.tx);
                const int ex1 = (int)fminf(fmaxf(floorf((u + rx - 0.5f) * ift) + 1.f, 0.f), (float)vi.tx);
                const int ey0 = (int)fminf(fmaxf(floorf(ceilf(vv - ry - 0.5f) * ift), 0.f), (float)vi.ty);
                const int ey1 = (int)fminf(fmaxf(floorf((vv + ry - 0.5f) * ift) + 1.f, 0.f), (float)vi.ty);
                x0 = max(x0, ex0); x1 = min(x1, ex1); y0 = max(y0, ey0); y1 = min(y1, ey1);
            } else {
                x1 = x0;  // a splat fainter than 1/255 takes no pixel
            }
            ok = x1 > x0 && y1 > y0;
        }
        if (!ok) {
            const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
            out[0] = z; out[1] = z; out[2] = z;
            if (rec4 == kRecF4) out[3] = z;
            if (dkv) dkv[rec] = (0xFFFFFFFFull << 32) | (uint32_t)rec;
            if (rects) {
                if (rect32) st_hint(reinterpret_cast<uint32_t*>(rects) + rec, 1u, l2_policy_evict_last());
                else st_hint(rects + rec, make_uint2(0u, 0u), l2_policy_evict_last());
            }
            continue;
        }
        float rgb[3] = {lrgb[0], lrgb[1], lrgb[2]};
        uint32_t mask = lmask;
        if (!LIT) {
            float Y[16];
            const float3 ds = sh_dir(G, Vg.dir);
            sh_basis<D>(ds.x, ds.y, ds.z, Y);
            float acc[3] = {0.f, 0.f, 0.f};  // each channel summed over k in order
#pragma unroll
            for (int pl = 0; pl < NPL; ++pl) {
                const float4 c4 = s_sh[pl * blockDim.x + threadIdx.x];
                const float cv[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int j = 4 * pl + e;
                    if (j < 3 * NB) acc[j % 3] += cv[e] * Y[j / 3];
                }
            }
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                float a = acc[ch] + 0.5f;
                if (a < 0.f) { a = 0.f; mask |= 1u << ch; }
                rgb[ch] = a;
            }
        }
        const float idet = 1.f / Vg.det;
        out[0] = make_float4(u, vv, Vg.tz, G.opac);
        out[1] = make_float4(Vg.c * idet, -Vg.b * idet, Vg.a * idet, r);
        out[2] = make_float4(rgb[0], rgb[1], rgb[2], __uint_as_float(mask));
        const uint32_t lo = (uint32_t)x0 | ((uint32_t)y0 << 16), hi = (uint32_t)x1 | ((uint32_t)y1 << 16);
        if (rec4 == kRecF4)
            out[3] = make_float4(__uint_as_float(lo), __uint_as_float(hi),
                                 __uint_as_float((uint32_t)((x1 - x0) * (y1 - y0))), 0.f);
        if (dkv) dkv[rec] = ((uint64_t)__float_as_uint(Vg.tz) << 32) | (uint32_t)rec;
        klo = min(klo, __float_as_uint(Vg.tz));
        khi = max(khi, __float_as_uint(Vg.tz));
        // the emission gathers the rectangle in depth order: kept in L2
        if (rects) {
            if (rect32) st_hint(reinterpret_cast<uint32_t*>(rects) + rec, rect32_pack(lo, hi), l2_policy_evict_last());
            else st_hint(rects + rec, make_uint2(lo, hi), l2_policy_evict_last());
        }
    }
    if (drange) depth_range_add(drange, klo, khi);
}

// ------------------------------------------------------------------ adjoint
// 4 blocks an SM.  View-dependent colour: 128 registers, the SH coefficients
// and their gradient accumulators in shared memory (48 KB a block); relit:
// 123 registers, no spills (measured faster than 3 blocks at 130).
template <int D, bool LIT>
__global__ void __launch_bounds__(128, 4)
k_project_bwd(const float4* __restrict__ P, int64_t n, int64_t n_out, Dyn dyn, const gs_camera* __restrict__ cams,
              int V,
              const float4* __restrict__ proj, const float4* __restrict__ g2d,
              float4* __restrict__ dP, int accumulate, int rec4) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    constexpr int NB = (D + 1) * (D + 1);
    constexpr int NPL = (3 * NB + 3) / 4;
    // the SH coefficients are staged in shared memory once and re-read per
    // view from there, rather than held in registers next to their gradient
    __shared__ float4 s_sh[LIT ? 1 : NPL][128];
    if (!LIT) {
#pragma unroll
        for (int pl = 0; pl < NPL; ++pl) s_sh[pl][threadIdx.x] = __ldg(&P[(3 + pl) * n + g]);
    }
    Gauss G;
    load_gauss(P, n, g, G);
    apply_dyn(dyn, g, G);
    // view-dependent colour: the SH gradient accumulates in shared memory
    // (this thread's column), next to the coefficients
    __shared__ float4 s_dsh[LIT ? 1 : NPL][128];
    if (!LIT) {
#pragma unroll
        for (int pl = 0; pl < NPL; ++pl) s_dsh[pl][threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    float dmx = 0.f, dmy = 0.f, dmz = 0.f, dlogit = 0.f;
    float gsum[3] = {0.f, 0.f, 0.f};  // relit: colour gradient summed over the views
    float D00 = 0.f, D01 = 0.f, D02 = 0.f, D11 = 0.f, D12 = 0.f, D22 = 0.f;  // dSigma + dSigma^T
    for (int v = 0; v < V; ++v) {
        const int64_t rec = (int64_t)v * n_out + g;
        // every term of a view's contribution is a multiple of its 2D
        // gradient: views without one (culled, or reaching no pixel's
        // compositing) are skipped before their projection record is read
        const float4 ga = g2d[rec * 3], gb = g2d[rec * 3 + 1], gc = g2d[rec * 3 + 2];
        if (ga.x == 0.f && ga.y == 0.f && ga.z == 0.f && ga.w == 0.f && gb.x == 0.f && gb.y == 0.f &&
            gb.z == 0.f && gb.w == 0.f && gc.x == 0.f)
            continue;
        // culled in this view (a 48-byte record comes from a fused call, whose
        // 2D gradient is zero for culled records: they are in no tile list)
        if (rec4 == kRecF4 && __float_as_uint(proj[rec * 4 + 3].z) == 0u) continue;
        const uint32_t mask = __float_as_uint(proj[rec * rec4 + 2].w);
        const Cam C = load_cam(cams + v);
        ViewGeom Vg;
        if (!view_geom(G, C, Vg)) continue;
        const float gu = ga.x, gv = ga.y, gA = ga.z, gB = ga.w, gC = gb.x, go = gb.y;
        const float grgb[3] = {gb.z, gb.w, gc.x};
        // opacity = sigmoid(logit)
        dlogit += go * G.opac * (1.f - G.opac);
        float gm[3];
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) gm[ch] = (mask & (1u << ch)) ? 0.f : grgb[ch];
        if (LIT) {
            // relit colour: the same in every view and linear in the
            // coefficients, so its gradient is summed first
            gsum[0] += gm[0]; gsum[1] += gm[1]; gsum[2] += gm[2];
        } else {
        // colour -> SH coefficients and view direction
        float Y[16];
        const float3 dsd = sh_dir(G, Vg.dir);
        sh_basis<D>(dsd.x, dsd.y, dsd.z, Y);
        float wsum[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) wsum[k] = 0.f;
#pragma unroll
        for (int pl = 0; pl < NPL; ++pl) {
            const float4 c4 = s_sh[LIT ? 0 : pl][threadIdx.x];
            const float cv[4] = {c4.x, c4.y, c4.z, c4.w};
            float4 d4 = s_dsh[LIT ? 0 : pl][threadIdx.x];
            float dv[4] = {d4.x, d4.y, d4.z, d4.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int j = 4 * pl + e;
                if (j >= 3 * NB) break;
                const int k = j / 3, ch = j % 3;
                dv[e] += gm[ch] * Y[k] * (k == 0 ? G.L : 1.f);
                wsum[k] += gm[ch] * cv[e];
            }
            s_dsh[LIT ? 0 : pl][threadIdx.x] = make_float4(dv[0], dv[1], dv[2], dv[3]);
        }
        float3 ddir = sh_basis_vjp<D>(dsd.x, dsd.y, dsd.z, wsum);
        if (G.moved) {  // the SH direction is R_g^T dir
            const float* R = G.Rg;
            ddir = make_float3(R[0] * ddir.x + R[1] * ddir.y + R[2] * ddir.z,
                               R[3] * ddir.x + R[4] * ddir.y + R[5] * ddir.z,
                               R[6] * ddir.x + R[7] * ddir.y + R[8] * ddir.z);
        }
        const float dd = Vg.dir.x * ddir.x + Vg.dir.y * ddir.y + Vg.dir.z * ddir.z;
        const float il = 1.f / Vg.len;
        dmx += (ddir.x - Vg.dir.x * dd) * il;
        dmy += (ddir.y - Vg.dir.y * dd) * il;
        dmz += (ddir.z - Vg.dir.z * dd) * il;
        }
        // conic (A, B, C) = (c, -b, a) / det
        const float a = Vg.a, b = Vg.b, c = Vg.c, id = 1.f / Vg.det, id2 = id * id;
        const float da = gA * (-c * c * id2) + gB * (b * c * id2) + gC * (id - a * c * id2);
        const float db = gA * (2.f * b * c * id2) + gB * (-id - 2.f * b * b * id2) + gC * (2.f * a * b * id2);
        const float dc = gA * (id - a * c * id2) + gB * (a * b * id2) + gC * (-a * a * id2);
        const float* S = G.S;
        const float* M0 = Vg.M0;
        const float* M1 = Vg.M1;
        const float SM0[3] = {S[0] * M0[0] + S[1] * M0[1] + S[2] * M0[2],
                              S[1] * M0[0] + S[3] * M0[1] + S[4] * M0[2],
                              S[2] * M0[0] + S[4] * M0[1] + S[5] * M0[2]};
        const float SM1[3] = {S[0] * M1[0] + S[1] * M1[1] + S[2] * M1[2],
                              S[1] * M1[0] + S[3] * M1[1] + S[4] * M1[2],
                              S[2] * M1[0] + S[4] * M1[1] + S[5] * M1[2]};
        float dM0[3], dM1[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            dM0[i] = 2.f * da * SM0[i] + db * SM1[i];
            dM1[i] = 2.f * dc * SM1[i] + db * SM0[i];
        }
        D00 += 2.f * (da * M0[0] * M0[0] + db * M0[0] * M1[0] + dc * M1[0] * M1[0]);
        D11 += 2.f * (da * M0[1] * M0[1] + db * M0[1] * M1[1] + dc * M1[1] * M1[1]);
        D22 += 2.f * (da * M0[2] * M0[2] + db * M0[2] * M1[2] + dc * M1[2] * M1[2]);
        D01 += 2.f * da * M0[0] * M0[1] + db * (M0[0] * M1[1] + M1[0] * M0[1]) + 2.f * dc * M1[0] * M1[1];
        D02 += 2.f * da * M0[0] * M0[2] + db * (M0[0] * M1[2] + M1[0] * M0[2]) + 2.f * dc * M1[0] * M1[2];
        D12 += 2.f * da * M0[1] * M0[2] + db * (M0[1] * M1[2] + M1[1] * M0[2]) + 2.f * dc * M1[1] * M1[2];
        // M0 = J00 W0 + J02 W2, M1 = J11 W1 + J12 W2
        const float* W = C.R;
        const float dJ00 = dM0[0] * W[0] + dM0[1] * W[1] + dM0[2] * W[2];
        const float dJ02 = dM0[0] * W[6] + dM0[1] * W[7] + dM0[2] * W[8];
        const float dJ11 = dM1[0] * W[3] + dM1[1] * W[4] + dM1[2] * W[5];
        const float dJ12 = dM1[0] * W[6] + dM1[1] * W[7] + dM1[2] * W[8];
        const float iz = Vg.iz, iz2 = iz * iz, iz3 = iz2 * iz;
        float dtx = 0.f, dty = 0.f, dtz = 0.f;
        dtz += -dJ00 * C.fx * iz2 - dJ11 * C.fy * iz2;
        dtz += dJ02 * 2.f * C.fx * Vg.xt * iz3 + dJ12 * 2.f * C.fy * Vg.yt * iz3;
        const float dxt = -dJ02 * C.fx * iz2, dyt = -dJ12 * C.fy * iz2;
        if (Vg.clx == 0) dtx += dxt; else dtz += dxt * (Vg.clx * Vg.limx);
        if (Vg.cly == 0) dty += dyt; else dtz += dyt * (Vg.cly * Vg.limy);
        // u = fx tx / tz + cx, v = fy ty / tz + cy
        dtx += gu * C.fx * iz;
        dty += gv * C.fy * iz;
        dtz += -(gu * C.fx * Vg.tx + gv * C.fy * Vg.ty) * iz2;
        // t = W mu + t_cam
        dmx += W[0] * dtx + W[3] * dty + W[6] * dtz;
        dmy += W[1] * dtx + W[4] * dty + W[7] * dtz;
        dmz += W[2] * dtx + W[5] * dty + W[8] * dtz;
    }
    if (G.moved) {  // back to the object frame: mean_w = R_g mean + t_g, Sigma_w = R_g Sigma R_g^T
        const float* Rg = G.Rg;
        const float m0 = dmx, m1 = dmy, m2 = dmz;
        dmx = Rg[0] * m0 + Rg[3] * m1 + Rg[6] * m2;
        dmy = Rg[1] * m0 + Rg[4] * m1 + Rg[7] * m2;
        dmz = Rg[2] * m0 + Rg[5] * m1 + Rg[8] * m2;
        const float Dw[9] = {D00, D01, D02, D01, D11, D12, D02, D12, D22};
        float T1[9];  // Dw R_g
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) T1[i * 3 + j] = Dw[i * 3] * Rg[j] + Dw[i * 3 + 1] * Rg[3 + j] + Dw[i * 3 + 2] * Rg[6 + j];
        // R_g^T T1
        D00 = Rg[0] * T1[0] + Rg[3] * T1[3] + Rg[6] * T1[6];
        D01 = Rg[0] * T1[1] + Rg[3] * T1[4] + Rg[6] * T1[7];
        D02 = Rg[0] * T1[2] + Rg[3] * T1[5] + Rg[6] * T1[8];
        D11 = Rg[1] * T1[1] + Rg[4] * T1[4] + Rg[7] * T1[7];
        D12 = Rg[1] * T1[2] + Rg[4] * T1[5] + Rg[7] * T1[8];
        D22 = Rg[2] * T1[2] + Rg[5] * T1[5] + Rg[8] * T1[8];
    }
    // Sigma = R diag(s^2) R^T:  dR = (dS + dS^T) R diag(s^2),  ds_k = s_k (R^T (dS + dS^T) R)_kk
    const float* R = G.Rq;
    const float s2[3] = {G.s.x * G.s.x, G.s.y * G.s.y, G.s.z * G.s.z};
    const float Dm[9] = {D00, D01, D02, D01, D11, D12, D02, D12, D22};
    float DR[9];  // Dm R
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            DR[i * 3 + j] = Dm[i * 3] * R[j] + Dm[i * 3 + 1] * R[3 + j] + Dm[i * 3 + 2] * R[6 + j];
    float dR[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) dR[i * 3 + j] = DR[i * 3 + j] * s2[j];
    float ds[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) ds[k] = R[k] * DR[k] + R[3 + k] * DR[3 + k] + R[6 + k] * DR[6 + k];
    // ds above is (R^T Dm R)_kk; d(log s_k) = s_k^2 (R^T Dm R)_kk
    const float w = G.q[0], x = G.q[1], y = G.q[2], z = G.q[3];
    float dq[4];
    dq[0] = dR[1] * (-2.f * z) + dR[2] * (2.f * y) + dR[3] * (2.f * z) + dR[5] * (-2.f * x) + dR[6] * (-2.f * y) + dR[7] * (2.f * x);
    dq[1] = dR[1] * (2.f * y) + dR[2] * (2.f * z) + dR[3] * (2.f * y) + dR[4] * (-4.f * x) + dR[5] * (-2.f * w) + dR[6] * (2.f * z) + dR[7] * (2.f * w) + dR[8] * (-4.f * x);
    dq[2] = dR[0] * (-4.f * y) + dR[1] * (2.f * x) + dR[2] * (2.f * w) + dR[3] * (2.f * x) + dR[5] * (2.f * z) + dR[6] * (-2.f * w) + dR[7] * (2.f * z) + dR[8] * (-4.f * y);
    dq[3] = dR[0] * (-4.f * z) + dR[1] * (-2.f * w) + dR[2] * (2.f * x) + dR[3] * (2.f * w) + dR[4] * (-4.f * z) + dR[5] * (2.f * y) + dR[6] * (2.f * x) + dR[7] * (2.f * y);
    const float qd = w * dq[0] + x * dq[1] + y * dq[2] + z * dq[3];
    const float iqn = 1.f / G.qn;
    float4 o0 = make_float4(dmx, dmy, dmz, dlogit);
    float4 o1 = make_float4(ds[0] * s2[0], ds[1] * s2[1], ds[2] * s2[2], 0.f);
    float4 o2 = make_float4((dq[0] - w * qd) * iqn, (dq[1] - x * qd) * iqn, (dq[2] - y * qd) * iqn,
                            (dq[3] - z * qd) * iqn);
    if (accumulate) {
        float4 p;
        p = dP[g]; o0.x += p.x; o0.y += p.y; o0.z += p.z; o0.w += p.w;
        p = dP[n + g]; o1.x += p.x; o1.y += p.y; o1.z += p.z; o1.w += p.w;
        p = dP[2 * n + g]; o2.x += p.x; o2.y += p.y; o2.z += p.z; o2.w += p.w;
    }
    dP[g] = o0;
    dP[n + g] = o1;
    dP[2 * n + g] = o2;
    // relit: coefficient j's gradient is the summed colour gradient times
    // its transfer weight (environment + visible direct light), formed here
    const float* lt = LIT ? lit_row(dyn, g) : nullptr;
    const float lv = LIT ? lit_vis(dyn, g) : 0.f;
#pragma unroll
    for (int pl = 0; pl < 12; ++pl) {
        float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
        if (pl < NPL) {
            if (LIT) {
                float ov[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int j = 4 * pl + e;
                    ov[e] = j < 3 * NB ? gsum[j % 3] * (__ldg(&lt[j]) + lv * __ldg(&lt[48 + j])) : 0.f;
                }
                o = make_float4(ov[0], ov[1], ov[2], ov[3]);
            } else {
                o = s_dsh[LIT ? 0 : pl][threadIdx.x];
            }
            // lanes beyond the 3*NB used coefficients carry no gradient
            if (4 * pl + 0 >= 3 * NB) o.x = 0.f;
            if (4 * pl + 1 >= 3 * NB) o.y = 0.f;
            if (4 * pl + 2 >= 3 * NB) o.z = 0.f;
            if (4 * pl + 3 >= 3 * NB) o.w = 0.f;
        }
        if (accumulate) {
            const float4 p = dP[(3 + pl) * n + g];
            o.x += p.x; o.y += p.y; o.z += p.z; o.w += p.w;
        }
        dP[(3 + pl) * n + g] = o;
    }
}

__global__ void k_view_table(const gs_camera* __restrict__ cams, int V, int tile, ViewInfo* vt,
                             long long expect_tiles, long long expect_super, DevStatus* status,
                             uint32_t* drange) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (drange) {
        drange[0] = 0xFFFFFFFFu;
        drange[1] = 0u;
    }
    int64_t toff = 0, poff = 0, soff = 0;
    for (int v = 0; v < V; ++v) {
        ViewInfo vi;
        vi.rect32 = vi.pad = 0;
        vi.width = cams[v].width;
        vi.height = cams[v].height;
        vi.tx = (vi.width + tile - 1) / tile;
        vi.ty = (vi.height + tile - 1) / tile;
        vi.tile_off = toff;
        vi.pix_off = poff;
        vi.stx = (vi.tx + kSuper - 1) >> kSuperShift;
        vi.sty = (vi.ty + kSuper - 1) >> kSuperShift;
        vi.stile_off = soff;
        vt[v] = vi;
        toff += (int64_t)vi.tx * vi.ty;
        poff += (int64_t)vi.width * vi.height;
        soff += (int64_t)vi.stx * vi.sty;
    }
    ViewInfo tot;
    tot.tx = tot.ty = tot.width = tot.height = tot.stx = tot.sty = 0;
    tot.tile_off = toff;
    tot.pix_off = poff;
    tot.stile_off = soff;
    tot.rect32 = 1;
    tot.pad = 0;
    for (int v = 0; v < V; ++v)
        if (vt[v].tx > 256 || vt[v].ty > 256) tot.rect32 = 0;
    vt[V] = tot;
    if (expect_tiles >= 0 && toff != expect_tiles) record_status(status, GS_ERR_ARG, toff);
    if (expect_super >= 0 && soff != expect_super) record_status(status, GS_ERR_ARG, soff);
}

}  // namespace

void launch_view_table(const gs_camera* d_cams, int V, int tile, ViewInfo* vt, long long expect_tiles,
                       DevStatus* status, cudaStream_t st, long long expect_super, uint32_t* drange) {
    k_view_table<<<1, 32, 0, st>>>(d_cams, V, tile, vt, expect_tiles, expect_super, status, drange);
}

void launch_project(const float* params, int64_t n, int sh_degree, const Dyn& dyn, const gs_camera* d_cams,
                    const ViewInfo* vt, int V, int tile, float* proj, uint64_t* depth_kv, cudaStream_t st,
                    int64_t g_off, int64_t n_out, uint2* rects, int rec4, uint32_t* drange) {
    if (n <= 0) return;
    if (n_out < 0) n_out = n;
    const int threads = 256;
    const unsigned blocks = (unsigned)((n + threads - 1) / threads);
    const float4* P = reinterpret_cast<const float4*>(params);
    float4* out = reinterpret_cast<float4*>(proj);
    const bool lit = dyn.lit_tab != nullptr;
    const size_t smem = lit && lit_groups(dyn) <= kStageGroups ? sizeof(float) * lit_groups(dyn) * kStageStride : 0;
#define GS_PROJ(DD)                                                                                              \
    (lit ? k_project<DD, true><<<blocks, threads, smem, st>>>(P, n, g_off, n_out, dyn, d_cams, vt, V, tile, out, depth_kv, rects, rec4, drange) \
         : k_project<DD, false><<<blocks, threads, sizeof(float4) * threads * ((3 * (DD + 1) * (DD + 1) + 3) / 4), st>>>( \
               P, n, g_off, n_out, dyn, d_cams, vt, V, tile, out, depth_kv, rects, rec4, drange))
    switch (sh_degree) {
        case 0: GS_PROJ(0); break;
        case 1: GS_PROJ(1); break;
        case 2: GS_PROJ(2); break;
        default: GS_PROJ(3); break;
    }
#undef GS_PROJ
}

void launch_project_bwd(const float* params, int64_t n, int sh_degree, const Dyn& dyn, const gs_camera* d_cams,
                        int V, const float* proj, const float* grad2d, float* dparams, int accumulate,
                        cudaStream_t st, int64_t n_out, int rec4) {
    if (n <= 0) return;
    if (n_out < 0) n_out = n;
    const int threads = 128;
    const unsigned blocks = (unsigned)((n + threads - 1) / threads);
    const float4* P = reinterpret_cast<const float4*>(params);
    const float4* pr = reinterpret_cast<const float4*>(proj);
    const float4* g2 = reinterpret_cast<const float4*>(grad2d);
    float4* dP = reinterpret_cast<float4*>(dparams);
    const bool lit = dyn.lit_tab != nullptr;
#define GS_PROJ_BWD(DD)                                                                                          \
    (lit ? k_project_bwd<DD, true><<<blocks, threads, 0, st>>>(P, n, n_out, dyn, d_cams, V, pr, g2, dP, accumulate, \
                                                               rec4)                                            \
         : k_project_bwd<DD, false><<<blocks, threads, 0, st>>>(P, n, n_out, dyn, d_cams, V, pr, g2, dP, accumulate, \
                                                                rec4))
    switch (sh_degree) {
        case 0: GS_PROJ_BWD(0); break;
        case 1: GS_PROJ_BWD(1); break;
        case 2: GS_PROJ_BWD(2); break;
        default: GS_PROJ_BWD(3); break;
    }
#undef GS_PROJ_BWD
}

}  // namespace gs

namespace gs {

void launch_light_table(const Dyn& dyn, const float* light, float* tab, cudaStream_t st) {
    const int G = dyn.group ? dyn.n_groups : 1;
    k_light_table<<<(G + 63) / 64, 64, 0, st>>>(dyn, light, tab, G);
}

}  // namespace gs
