// gs_drive.cu -- the kernels around the renderer that the avatar module and the
// sensor composite need (sm_103a):
//   composite_kernel  nearest-fragment merge of two RGB-D layers (Sec. 3.2: the
//                     full-screen pass keeping, per pixel, the fragment with
//                     the smaller depth); streaming, 48 bytes per pixel
//   fk_kernel         skinning matrices of a joint tree by forward kinematics
//                     (Sec. 3.3.1), one CTA per avatar, one thread per joint,
//                     level by level down the tree
//   interp_kernel     joint matrices at a fractional frame position, linear
//                     between the two neighbouring frames (Sec. 3.3.1)
//   exp2_rate_kernel  throughput of the special-function unit's exp2, the one
//                     transcendental of every blend evaluation (for its roofline)
#include <cmath>

#include "gs_internal.cuh"
#include "gs_launch.h"

namespace gs {

// ---------------------------------------------------------------------------
// composite
// ---------------------------------------------------------------------------
__device__ __forceinline__ float layer_depth(float d) { return (d > 0.0f && d <= 3.402823466e38f) ? d : INFINITY; }

// Four pixels per thread (hw % 4 == 0, 16-byte aligned planes) or one.
template <int VEC>
__global__ void __launch_bounds__(256) composite_kernel(const float *__restrict__ rgb_a, const float *__restrict__ depth_a,
                                                        const float *__restrict__ rgb_b, const float *__restrict__ depth_b,
                                                        float *rgb_out, float *depth_out, int64_t n_views, int64_t hw)
{
    const int64_t per_view = hw / VEC;
    const int64_t total = n_views * per_view;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = i / per_view, p = (i - v * per_view) * VEC;
        const int64_t di = v * hw + p;
        if (VEC == 4) {
            const float4 da = *reinterpret_cast<const float4 *>(depth_a + di);
            const float4 db = *reinterpret_cast<const float4 *>(depth_b + di);
            const bool ta[4] = {layer_depth(da.x) < layer_depth(db.x), layer_depth(da.y) < layer_depth(db.y),
                                layer_depth(da.z) < layer_depth(db.z), layer_depth(da.w) < layer_depth(db.w)};
            *reinterpret_cast<float4 *>(depth_out + di) =
                make_float4(ta[0] ? da.x : db.x, ta[1] ? da.y : db.y, ta[2] ? da.z : db.z, ta[3] ? da.w : db.w);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int64_t k = (3 * v + c) * hw + p;
                const float4 ca = *reinterpret_cast<const float4 *>(rgb_a + k);
                const float4 cb = *reinterpret_cast<const float4 *>(rgb_b + k);
                *reinterpret_cast<float4 *>(rgb_out + k) =
                    make_float4(ta[0] ? ca.x : cb.x, ta[1] ? ca.y : cb.y, ta[2] ? ca.z : cb.z, ta[3] ? ca.w : cb.w);
            }
        } else {
            const float da = depth_a[di], db = depth_b[di];
            const bool ta = layer_depth(da) < layer_depth(db);
            depth_out[di] = ta ? da : db;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int64_t k = (3 * v + c) * hw + p;
                rgb_out[k] = ta ? rgb_a[k] : rgb_b[k];
            }
        }
    }
}

void launch_composite(const float *rgb_a, const float *depth_a, const float *rgb_b, const float *depth_b,
                      float *rgb_out, float *depth_out, int64_t n_views, int64_t hw, int n_sms, cudaStream_t s)
{
    const bool vec = hw % 4 == 0;
    const int64_t items = n_views * (vec ? hw / 4 : hw);
    int64_t grid = (items + 255) / 256;
    const int64_t cap = (int64_t)n_sms * 8;
    if (grid > cap) grid = cap;
    if (grid < 1) return;
    if (vec)
        composite_kernel<4><<<(unsigned)grid, 256, 0, s>>>(rgb_a, depth_a, rgb_b, depth_b, rgb_out, depth_out,
                                                           n_views, hw);
    else
        composite_kernel<1><<<(unsigned)grid, 256, 0, s>>>(rgb_a, depth_a, rgb_b, depth_b, rgb_out, depth_out,
                                                           n_views, hw);
}

// ---------------------------------------------------------------------------
// forward kinematics
// ---------------------------------------------------------------------------
// G_0 = [R_root R_0 | t_root], G_j = G_p [R_j | J_j - J_p], M_j = G_j [I | -J_j].
// Joints of one tree depth are independent: thread j computes G_j once its
// parent's level is done.
__global__ void __launch_bounds__(kMaxJoints) fk_kernel(const float *__restrict__ local_rot,
                                                        const float *__restrict__ root, const float *__restrict__ rest,
                                                        JointTree tree, float *__restrict__ out)
{
    __shared__ float G[kMaxJoints][12];
    const int a = blockIdx.x, j = threadIdx.x, J = tree.n;
    float Rl[9];
    if (j < J) {
#pragma unroll
        for (int i = 0; i < 9; ++i) Rl[i] = local_rot[((size_t)a * J + j) * 9 + i];
    }
    for (int level = 0; level <= tree.max_depth; ++level) {
        if (j < J && tree.depth[j] == level) {
            float P[12];
            float off[3];
            if (j == 0 || tree.parent[j] < 0) {
#pragma unroll
                for (int i = 0; i < 12; ++i) P[i] = root[(size_t)a * 12 + i];
                off[0] = off[1] = off[2] = 0.f;
            } else {
                const int p = tree.parent[j];
#pragma unroll
                for (int i = 0; i < 12; ++i) P[i] = G[p][i];
#pragma unroll
                for (int c = 0; c < 3; ++c) off[c] = rest[3 * j + c] - rest[3 * p + c];
            }
#pragma unroll
            for (int r = 0; r < 3; ++r) {
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    G[j][4 * r + c] = P[4 * r] * Rl[c] + P[4 * r + 1] * Rl[3 + c] + P[4 * r + 2] * Rl[6 + c];
                G[j][4 * r + 3] = P[4 * r] * off[0] + P[4 * r + 1] * off[1] + P[4 * r + 2] * off[2] + P[4 * r + 3];
            }
        }
        __syncthreads();
    }
    if (j < J) {
        float *M = out + ((size_t)a * J + j) * 12;
        const float jx = rest[3 * j], jy = rest[3 * j + 1], jz = rest[3 * j + 2];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            M[4 * r] = G[j][4 * r];
            M[4 * r + 1] = G[j][4 * r + 1];
            M[4 * r + 2] = G[j][4 * r + 2];
            M[4 * r + 3] = G[j][4 * r + 3] - (G[j][4 * r] * jx + G[j][4 * r + 1] * jy + G[j][4 * r + 2] * jz);
        }
    }
}

void launch_fk(const float *local_rot, const float *root, const float *rest, const JointTree &tree, int n_avatars,
               float *out, cudaStream_t s)
{
    fk_kernel<<<n_avatars, kMaxJoints, 0, s>>>(local_rot, root, rest, tree, out);
}

// ---------------------------------------------------------------------------
// interpolation of per-frame joint matrices
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) interp_kernel(const float *__restrict__ frames, const float *__restrict__ t,
                                                     int n_avatars, int n_frames, int per_frame, float *__restrict__ out)
{
    const int64_t total = (int64_t)n_avatars * per_frame;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)(i / per_frame), e = (int)(i - (int64_t)a * per_frame);
        const float tf = t[a];
        float f = floorf(tf);
        if (!(f >= 0.0f)) f = 0.0f;
        if (f > (float)(n_frames - 1)) f = (float)(n_frames - 1);
        float w = tf - f;
        if (!(w >= 0.0f)) w = 0.0f;
        if (w > 1.0f) w = 1.0f;
        const int f0 = (int)f, f1 = f0 + 1 < n_frames ? f0 + 1 : n_frames - 1;
        const float x0 = frames[((size_t)a * n_frames + f0) * per_frame + e];
        const float x1 = frames[((size_t)a * n_frames + f1) * per_frame + e];
        out[i] = (1.0f - w) * x0 + w * x1;
    }
}

void launch_interp(const float *frames, const float *t, int n_avatars, int n_frames, int n_joints, float *out,
                   int n_sms, cudaStream_t s)
{
    const int per_frame = n_joints * 12;
    int64_t grid = ((int64_t)n_avatars * per_frame + 255) / 256;
    if (grid > (int64_t)n_sms * 8) grid = (int64_t)n_sms * 8;
    if (grid < 1) return;
    interp_kernel<<<(unsigned)grid, 256, 0, s>>>(frames, t, n_avatars, n_frames, per_frame, out);
}

// ---------------------------------------------------------------------------
// Proxy capsules and the avatar queries (Sec. 3.3.2, Sec. 3.4)
// ---------------------------------------------------------------------------
// Capsule of joint j of avatar a: the segment from the posed parent joint to
// the posed joint j (the root: both ends at the root, a sphere), radius
// radius[j]; posed position = M_j [J_j; 1].  Rows (ax, ay, az, rho, bx, by, bz, 0).
__global__ void __launch_bounds__(256) capsules_kernel(const float *__restrict__ M, const float *__restrict__ rest,
                                                       const float *__restrict__ radius, const JointTree tree,
                                                       int n_avatars, float4 *__restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int J = tree.n;
    if (i >= (int64_t)n_avatars * J) return;
    const int a = (int)(i / J), j = (int)(i - (int64_t)a * J);
    const int par = j == 0 ? 0 : tree.parent[j];
    float pj[3], pp[3];
    const float *Mj = M + ((int64_t)a * J + j) * 12, *Mp = M + ((int64_t)a * J + par) * 12;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        pj[r] = __fmaf_rn(Mj[4 * r + 2], rest[3 * j + 2],
                          __fmaf_rn(Mj[4 * r + 1], rest[3 * j + 1], __fmaf_rn(Mj[4 * r], rest[3 * j], Mj[4 * r + 3])));
        pp[r] = __fmaf_rn(Mp[4 * r + 2], rest[3 * par + 2],
                          __fmaf_rn(Mp[4 * r + 1], rest[3 * par + 1], __fmaf_rn(Mp[4 * r], rest[3 * par], Mp[4 * r + 3])));
    }
    out[2 * i] = make_float4(pp[0], pp[1], pp[2], radius[j]);
    out[2 * i + 1] = make_float4(pj[0], pj[1], pj[2], 0.0f);
}

void launch_capsules(const float *M, const float *rest, const float *radius, const JointTree &tree, int n_avatars,
                     float *out, cudaStream_t s)
{
    const int64_t n = (int64_t)n_avatars * tree.n;
    if (n > 0) capsules_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(M, rest, radius, tree, n_avatars,
                                                                          reinterpret_cast<float4 *>(out));
}

// Distance from p to the segment a + s (b - a), s in [0, 1].
__device__ __forceinline__ float point_seg_dist(float3 p, float3 a, float3 b)
{
    const float3 ab = make_float3(b.x - a.x, b.y - a.y, b.z - a.z), ap = make_float3(p.x - a.x, p.y - a.y, p.z - a.z);
    const float ll = ab.x * ab.x + ab.y * ab.y + ab.z * ab.z;
    float s = ll > 0.0f ? (ap.x * ab.x + ap.y * ab.y + ap.z * ab.z) / ll : 0.0f;
    s = fminf(1.0f, fmaxf(0.0f, s));
    const float ex = ap.x - s * ab.x, ey = ap.y - s * ab.y, ez = ap.z - s * ab.z;
    return sqrtf(ex * ex + ey * ey + ez * ez);
}

// Step parameter u in [0, 1] of the point of the step p0 + u v closest to the
// segment a + s d (both clamped): the minimiser of the convex squared distance
// |r + u v - s d|^2, r = p0 - a, over the unit square, by the normal equations
// and their edges.
__device__ __forceinline__ float step_closest(float3 r, float3 v, float3 d)
{
    const float vv = v.x * v.x + v.y * v.y + v.z * v.z, dd = d.x * d.x + d.y * d.y + d.z * d.z;
    const float vd = v.x * d.x + v.y * d.y + v.z * d.z;
    const float rv = r.x * v.x + r.y * v.y + r.z * v.z, rd = r.x * d.x + r.y * d.y + r.z * d.z;
    if (vv <= 0.0f) return 0.0f; // no motion
    if (dd <= 0.0f) return fminf(1.0f, fmaxf(0.0f, -rv / vv)); // a sphere: closest to its centre
    const float den = vv * dd - vd * vd;
    float u = den > 1e-12f * vv * dd ? fminf(1.0f, fmaxf(0.0f, (vd * rd - rv * dd) / den)) : 0.0f;
    const float s = (rd + u * vd) / dd; // the segment's best s for this u
    if (s < 0.0f) u = fminf(1.0f, fmaxf(0.0f, -rv / vv));
    else if (s > 1.0f) u = fminf(1.0f, fmaxf(0.0f, (vd - rv) / vv));
    return u;
}

// One query per thread over the capsules of its env: signed distance from p0
// to the nearest capsule surface (the lowest index on ties), and for the step
// p0 -> p1 the first contact of the agent sphere (radius r): the convex
// distance to a capsule's axis falls until the step's closest point, so a
// capsule touches iff it is within rho + r there, and the first contact is
// found by bisection on [0, closest].
__global__ void __launch_bounds__(256) capsule_query_kernel(const float4 *__restrict__ caps,
                                                            const int64_t *__restrict__ cap_off, int n_envs,
                                                            const int32_t *__restrict__ query_env,
                                                            const float *__restrict__ p0, const float *__restrict__ p1,
                                                            float agent_r, int64_t n_q, float *__restrict__ out_dist,
                                                            int32_t *__restrict__ out_near, float *__restrict__ out_t,
                                                            uint8_t *__restrict__ out_blk)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n_q) return;
    const int e = query_env[q];
    const float3 P0 = make_float3(p0[3 * q], p0[3 * q + 1], p0[3 * q + 2]);
    const float3 P1 = p1 ? make_float3(p1[3 * q], p1[3 * q + 1], p1[3 * q + 2]) : P0;
    const float3 v = make_float3(P1.x - P0.x, P1.y - P0.y, P1.z - P0.z);
    float best = INFINITY, tmin = 1.0f;
    int32_t arg = -1;
    bool blocked = false;
    const int64_t c0 = (e >= 0 && e < n_envs) ? cap_off[e] : 0, c1 = (e >= 0 && e < n_envs) ? cap_off[e + 1] : 0;
    for (int64_t c = c0; c < c1; ++c) {
        const float4 ca = __ldg(caps + 2 * c), cb = __ldg(caps + 2 * c + 1);
        const float3 a = make_float3(ca.x, ca.y, ca.z), b = make_float3(cb.x, cb.y, cb.z);
        const float d = point_seg_dist(P0, a, b) - ca.w;
        if (d < best) {
            best = d;
            arg = (int32_t)(c - c0);
        }
        const float R = ca.w + agent_r;
        if (d + ca.w <= R) { // starts in contact
            blocked = true;
            tmin = 0.0f;
            continue;
        }
        const float3 r = make_float3(P0.x - a.x, P0.y - a.y, P0.z - a.z), dv = make_float3(b.x - a.x, b.y - a.y,
                                                                                              b.z - a.z);
        const float us = step_closest(r, v, dv);
        auto f = [&](float u) { return point_seg_dist(make_float3(P0.x + u * v.x, P0.y + u * v.y, P0.z + u * v.z), a, b); };
        if (f(us) > R) continue;
        float lo = 0.0f, hi = us;
#pragma unroll 1
        for (int it = 0; it < 30; ++it) {
            const float m = 0.5f * (lo + hi);
            if (f(m) <= R) hi = m;
            else lo = m;
        }
        blocked = true;
        tmin = fminf(tmin, hi);
    }
    out_dist[q] = best;
    out_near[q] = arg;
    if (out_t) out_t[q] = blocked ? tmin : 1.0f;
    if (out_blk) out_blk[q] = blocked ? 1u : 0u;
}

void launch_capsule_query(const float *caps, const int64_t *cap_off, int n_envs, const int32_t *query_env,
                          const float *p0, const float *p1, float agent_r, int64_t n_q, float *out_dist,
                          int32_t *out_near, float *out_t, uint8_t *out_blk, cudaStream_t s)
{
    if (n_q > 0)
        capsule_query_kernel<<<(unsigned)((n_q + 255) / 256), 256, 0, s>>>(
            reinterpret_cast<const float4 *>(caps), cap_off, n_envs, query_env, p0, p1, agent_r, n_q, out_dist,
            out_near, out_t, out_blk);
}

// ---------------------------------------------------------------------------
// exp2 throughput (a measurement, not part of the renderer)
// ---------------------------------------------------------------------------
// Eight independent chains per thread, x <- 2^(-x), which stays in (0.5, 1]:
// one ex2.approx per step and chain, nothing else on the dependent path.
__global__ void __launch_bounds__(256) exp2_rate_kernel(int iters, float *out)
{
    float x[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = 0.5f + 0.01f * (float)((threadIdx.x + c) & 15);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < 8; ++c) asm volatile("ex2.approx.ftz.f32 %0, %1;\n" : "=f"(x[c]) : "f"(-x[c]));
    }
    float acc = 0.f;
#pragma unroll
    for (int c = 0; c < 8; ++c) acc += x[c];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

void launch_exp2_rate(int n_blocks, int iters, float *out, cudaStream_t s)
{
    exp2_rate_kernel<<<n_blocks, 256, 0, s>>>(iters, out);
}

} // namespace gs
