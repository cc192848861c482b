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
