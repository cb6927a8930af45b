// Device helpers shared by the projection and light-map kernels: the real SH
// basis of degree <= 3 and its vector-Jacobian product, the pinhole camera,
// one Gaussian's parameters decoded into mean / covariance / opacity, and the
// rigid object pose of Sec. 3.4.2.
#pragma once
#include "gs_internal.cuh"

namespace gs {
namespace {

// Real SH normalisation constants: sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!)
// times the polynomial factor, for the Condon-Shortley-phase real basis.
constexpr float kY0 = 0.28209479177387814f;   // sqrt(1/(4 pi))
constexpr float kY1 = 0.48860251190291992f;   // sqrt(3/(4 pi))
constexpr float kY2a = 1.0925484305920792f;   // sqrt(15/(4 pi))
constexpr float kY2b = 0.31539156525252005f;  // sqrt(5/(16 pi))
constexpr float kY2c = 0.54627421529603959f;  // sqrt(15/(16 pi))
constexpr float kY3a = 0.59004358992664352f;  // sqrt(35/(32 pi))
constexpr float kY3b = 2.8906114426405538f;   // sqrt(105/(4 pi))
constexpr float kY3c = 0.45704579946446572f;  // sqrt(21/(32 pi))
constexpr float kY3d = 0.3731763325901154f;   // sqrt(7/(16 pi))
constexpr float kY3e = 1.4453057213202769f;   // sqrt(105/(16 pi))

template <int D>
__device__ __forceinline__ void sh_basis(float x, float y, float z, float* Y) {
    Y[0] = kY0;
    if (D >= 1) {
        Y[1] = -kY1 * y;
        Y[2] = kY1 * z;
        Y[3] = -kY1 * x;
    }
    if (D >= 2) {
        const float xx = x * x, yy = y * y, zz = z * z;
        Y[4] = kY2a * x * y;
        Y[5] = -kY2a * y * z;
        Y[6] = kY2b * (2.f * zz - xx - yy);
        Y[7] = -kY2a * x * z;
        Y[8] = kY2c * (xx - yy);
        if (D >= 3) {
            Y[9] = -kY3a * y * (3.f * xx - yy);
            Y[10] = kY3b * x * y * z;
            Y[11] = -kY3c * y * (4.f * zz - xx - yy);
            Y[12] = kY3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
            Y[13] = -kY3c * x * (4.f * zz - xx - yy);
            Y[14] = kY3e * z * (xx - yy);
            Y[15] = -kY3a * x * (xx - 3.f * yy);
        }
    }
}

// sum_k w_k * grad Y_k at (x, y, z) (gradient of the polynomial forms above).
template <int D>
__device__ __forceinline__ float3 sh_basis_vjp(float x, float y, float z, const float* w) {
    float gx = 0.f, gy = 0.f, gz = 0.f;
    if (D >= 1) {
        gy += -kY1 * w[1];
        gz += kY1 * w[2];
        gx += -kY1 * w[3];
    }
    if (D >= 2) {
        const float xx = x * x, yy = y * y, zz = z * z;
        gx += kY2a * y * w[4];                 gy += kY2a * x * w[4];
        gy += -kY2a * z * w[5];                gz += -kY2a * y * w[5];
        gx += -2.f * kY2b * x * w[6];          gy += -2.f * kY2b * y * w[6];     gz += 4.f * kY2b * z * w[6];
        gx += -kY2a * z * w[7];                gz += -kY2a * x * w[7];
        gx += 2.f * kY2c * x * w[8];           gy += -2.f * kY2c * y * w[8];
        if (D >= 3) {
            gx += -kY3a * 6.f * x * y * w[9];
            gy += -kY3a * 3.f * (xx - yy) * w[9];
            gx += kY3b * y * z * w[10];  gy += kY3b * x * z * w[10];  gz += kY3b * x * y * w[10];
            gx += kY3c * 2.f * x * y * w[11];
            gy += -kY3c * (4.f * zz - xx - 3.f * yy) * w[11];
            gz += -kY3c * 8.f * y * z * w[11];
            gx += -kY3d * 6.f * x * z * w[12];
            gy += -kY3d * 6.f * y * z * w[12];
            gz += kY3d * (6.f * zz - 3.f * xx - 3.f * yy) * w[12];
            gx += -kY3c * (4.f * zz - 3.f * xx - yy) * w[13];
            gy += kY3c * 2.f * x * y * w[13];
            gz += -kY3c * 8.f * x * z * w[13];
            gx += 2.f * kY3e * x * z * w[14];  gy += -2.f * kY3e * y * z * w[14];  gz += kY3e * (xx - yy) * w[14];
            gx += -kY3a * 3.f * (xx - yy) * w[15];
            gy += kY3a * 6.f * x * y * w[15];
        }
    }
    return make_float3(gx, gy, gz);
}

struct Cam {
    float R[9], t[3], fx, fy, cx, cy, near;
    int W, H;
};

// The 80-byte camera record as five 16-byte loads when it is 16-byte aligned
// (any cudaMalloc'd array of them is), else field by field; the branch is
// uniform over the warp.
__device__ __forceinline__ Cam load_cam(const gs_camera* __restrict__ c) {
    Cam k;
    if ((reinterpret_cast<uintptr_t>(c) & 15u) == 0) {
        const float4* p = reinterpret_cast<const float4*>(c);
        const float4 a = __ldg(p), b = __ldg(p + 1), d = __ldg(p + 2), e = __ldg(p + 3), f = __ldg(p + 4);
        k.R[0] = a.x; k.R[1] = a.y; k.R[2] = a.z; k.R[3] = a.w;
        k.R[4] = b.x; k.R[5] = b.y; k.R[6] = b.z; k.R[7] = b.w;
        k.R[8] = d.x; k.t[0] = d.y; k.t[1] = d.z; k.t[2] = d.w;
        k.fx = e.x; k.fy = e.y; k.cx = e.z; k.cy = e.w;
        k.W = __float_as_int(f.x); k.H = __float_as_int(f.y); k.near = f.z;
        return k;
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) k.R[i] = __ldg(&c->R[i]);
#pragma unroll
    for (int i = 0; i < 3; ++i) k.t[i] = __ldg(&c->t[i]);
    k.fx = __ldg(&c->fx); k.fy = __ldg(&c->fy); k.cx = __ldg(&c->cx); k.cy = __ldg(&c->cy);
    k.near = __ldg(&c->near_plane);
    k.W = __ldg(&c->width); k.H = __ldg(&c->height);
    return k;
}

struct Gauss {
    float3 mu;       // world frame once apply_dyn has run
    float logit, opac;
    float3 s;        // exp(log-scale)
    float q[4];      // normalised quaternion (object frame)
    float qn;        // |q|
    float Rq[9];
    float S[6];      // Sigma: 00 01 02 11 12 22 (world frame once apply_dyn has run)
    bool moved;      // object pose applied
    float Rg[9];     // object rotation
    float L;         // relighting factor of the DC coefficient
};

__device__ __forceinline__ void quat_rot(float w, float x, float y, float z, float* R) {
    const float n = rsqrtf(w * w + x * x + y * y + z * z);
    w *= n; x *= n; y *= n; z *= n;
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z);       R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z);       R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y);       R[7] = 2.f * (y * z + w * x);       R[8] = 1.f - 2.f * (x * x + y * y);
}

// Object pose and relighting (Sec. 3.4): mean and covariance to the world
// frame, Lambertian factor of the DC coefficient.
__device__ __forceinline__ void apply_dyn(const Dyn& d, int64_t g, Gauss& G) {
    G.moved = d.group != nullptr;
    G.L = 1.f;
    if (!G.moved) return;
    const uint32_t grp = min((uint32_t)d.group[g], (uint32_t)(d.n_groups - 1));  // ids beyond the poses clamp
    const float4 q = d.poses[2 * grp], t = d.poses[2 * grp + 1];
    float* R = G.Rg;
    quat_rot(q.x, q.y, q.z, q.w, R);
    const float3 m = G.mu;
    G.mu = make_float3(R[0] * m.x + R[1] * m.y + R[2] * m.z + t.x, R[3] * m.x + R[4] * m.y + R[5] * m.z + t.y,
                       R[6] * m.x + R[7] * m.y + R[8] * m.z + t.z);
    // Sigma_w = R Sigma R^T
    const float* S = G.S;
    const float Sf[9] = {S[0], S[1], S[2], S[1], S[3], S[4], S[2], S[4], S[5]};
    float RS[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) RS[i * 3 + j] = R[i * 3] * Sf[j] + R[i * 3 + 1] * Sf[3 + j] + R[i * 3 + 2] * Sf[6 + j];
    float W[6];
    W[0] = RS[0] * R[0] + RS[1] * R[1] + RS[2] * R[2];
    W[1] = RS[0] * R[3] + RS[1] * R[4] + RS[2] * R[5];
    W[2] = RS[0] * R[6] + RS[1] * R[7] + RS[2] * R[8];
    W[3] = RS[3] * R[3] + RS[4] * R[4] + RS[5] * R[5];
    W[4] = RS[3] * R[6] + RS[4] * R[7] + RS[5] * R[8];
    W[5] = RS[6] * R[6] + RS[7] * R[7] + RS[8] * R[8];
#pragma unroll
    for (int i = 0; i < 6; ++i) G.S[i] = W[i];
    if (d.normals) {
        const float4 nl = d.normals[g];
        const float4 l = *d.light;
        const float nd = (R[0] * nl.x + R[1] * nl.y + R[2] * nl.z) * l.x +
                         (R[3] * nl.x + R[4] * nl.y + R[5] * nl.z) * l.y +
                         (R[6] * nl.x + R[7] * nl.y + R[8] * nl.z) * l.z;
        G.L = d.ambient + d.diffuse * fmaxf(0.f, nd);
    }
}

// View direction in the object frame (SH appearance turns with its object).
__device__ __forceinline__ float3 sh_dir(const Gauss& G, float3 dw) {
    if (!G.moved) return dw;
    const float* R = G.Rg;
    return make_float3(R[0] * dw.x + R[3] * dw.y + R[6] * dw.z, R[1] * dw.x + R[4] * dw.y + R[7] * dw.z,
                       R[2] * dw.x + R[5] * dw.y + R[8] * dw.z);
}

__device__ __forceinline__ void load_gauss(const float4* __restrict__ P, int64_t n, int64_t g, Gauss& G) {
    const float4 p0 = P[g], p1 = P[n + g], p2 = P[2 * n + g];
    G.mu = make_float3(p0.x, p0.y, p0.z);
    G.logit = p0.w;
    G.opac = 1.f / (1.f + expf(-p0.w));
    G.s = make_float3(expf(p1.x), expf(p1.y), expf(p1.z));
    G.qn = sqrtf(p2.x * p2.x + p2.y * p2.y + p2.z * p2.z + p2.w * p2.w);
    const float w = p2.x / G.qn, x = p2.y / G.qn, y = p2.z / G.qn, z = p2.w / G.qn;
    G.q[0] = w; G.q[1] = x; G.q[2] = y; G.q[3] = z;
    float* R = G.Rq;
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z);       R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z);       R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y);       R[7] = 2.f * (y * z + w * x);       R[8] = 1.f - 2.f * (x * x + y * y);
    const float s0 = G.s.x * G.s.x, s1 = G.s.y * G.s.y, s2 = G.s.z * G.s.z;
    // Sigma = R diag(s^2) R^T
    G.S[0] = R[0] * R[0] * s0 + R[1] * R[1] * s1 + R[2] * R[2] * s2;
    G.S[1] = R[0] * R[3] * s0 + R[1] * R[4] * s1 + R[2] * R[5] * s2;
    G.S[2] = R[0] * R[6] * s0 + R[1] * R[7] * s1 + R[2] * R[8] * s2;
    G.S[3] = R[3] * R[3] * s0 + R[4] * R[4] * s1 + R[5] * R[5] * s2;
    G.S[4] = R[3] * R[6] * s0 + R[4] * R[7] * s1 + R[5] * R[8] * s2;
    G.S[5] = R[6] * R[6] * s0 + R[7] * R[7] * s1 + R[8] * R[8] * s2;
}

}  // namespace
}  // namespace gs
