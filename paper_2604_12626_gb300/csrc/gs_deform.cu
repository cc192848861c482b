// gs_deform.cu -- linear blend skinning of canonical avatar Gaussians
// (Sec. 3.3: a CUDA LBS kernel deforms pre-baked canonical Gaussians to the
// current SMPL-X pose; Sec. 3.3.1: per-frame joint matrices).
//
// deform           one thread per avatar Gaussian: A = sum_k w_k G[avatar][j_k]
//                  (3x4, weights as given), mean' = A3 mean + a,
//                  cov' = A3 Sigma A3^T with Sigma = R(q) diag(exp(2 s)) R(q)^T;
//                  the joint matrices of the CTA's avatar are staged in shared
//                  memory.  100 bytes of HBM traffic per Gaussian.
// deform_backward  the adjoint; the joint gradients of the CTA's avatar are summed
//                  per warp by joint owners (lane l adds w dL/dA of the warp's
//                  32 Gaussians wherever joint l appears), then over the warps
//                  in shared memory, then one global atomic per (joint, entry).
#include "gs_internal.cuh"
#include "gs_launch.h"

namespace gs {


struct AvIn {
    const float *means, *log_scales, *quats, *weights;
    const uint16_t *joint_ids;
    const int32_t *avatar_of;
    const int64_t *dest;
    int64_t m;
    int32_t n_avatars, n_joints;
    // without dest: the rows of a batch's avatars, canonical row i of env e at
    // env_cov_begin[e] + (i - env_av_base[e]) (gs_render_avatars_backward)
    const Table *tb;
};

// Batch row of canonical avatar row i: e the last env whose first avatar row
// env_av_base[e] <= i (an env without avatars shares its successor's base and
// precedes it).
__device__ __forceinline__ int64_t avatar_row(const Table *tb, int64_t i)
{
    int lo = 0, hi = tb->n_envs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tb->env_av_base[mid] <= i) lo = mid;
        else hi = mid - 1;
    }
    return tb->env_cov_begin[lo] + (i - tb->env_av_base[lo]);
}

__global__ void __launch_bounds__(256) deform_kernel(AvIn in, const float *__restrict__ G, float *out_means,
                                                     float *out_cov)
{
    __shared__ __align__(16) float sG[kMaxJoints * 12];
    const int64_t base = (int64_t)blockIdx.x * blockDim.x;
    const int64_t i = base + threadIdx.x;
    // the Gaussian's inputs are loaded first, so that they are in flight while
    // the CTA stages its avatar's joint matrices
    const bool valid = i < in.m;
    const int64_t ic = valid ? i : base;
    const int av = clamp_avatar(in.avatar_of[ic], in.n_avatars);
    const ushort4 id = clamp_ids(reinterpret_cast<const ushort4 *>(in.joint_ids)[ic], in.n_joints);
    const float4 wt = reinterpret_cast<const float4 *>(in.weights)[ic];
    const float3 m = make_float3(in.means[3 * ic], in.means[3 * ic + 1], in.means[3 * ic + 2]);
    const float3 ls = make_float3(in.log_scales[3 * ic], in.log_scales[3 * ic + 1], in.log_scales[3 * ic + 2]);
    const float4 q = reinterpret_cast<const float4 *>(in.quats)[ic];
    const int a0 = clamp_avatar(in.avatar_of[base], in.n_avatars);
    const int nj12 = in.n_joints * 12;
    for (int k = threadIdx.x; k < nj12; k += blockDim.x) sG[k] = G[(size_t)a0 * nj12 + k];
    __syncthreads();
    if (!valid) return;
    const float *Gs = av == a0 ? sG : G + (size_t)av * nj12;
    float mu[3], cov[6];
    lbs_gaussian(Gs, id, wt, m, ls, q, mu, cov);
    const int64_t d = in.dest ? in.dest[i] : i;
    out_means[3 * d] = mu[0];
    out_means[3 * d + 1] = mu[1];
    out_means[3 * d + 2] = mu[2];
    float *oc = out_cov + 6 * d;
#pragma unroll
    for (int k = 0; k < 6; ++k) oc[k] = cov[k];
}

constexpr int kDeformWarps = 8; // 256 threads

// One Gaussian's share of the joint gradients, staged for its warp: dL/dA
// (3x4) and the four (joint, weight) pairs.  80 bytes (16-byte loads).
struct JointShare {
    float4 gA[3];
    float4 w;
    ushort4 ids;
    uint32_t pad[2];
};

__global__ void __launch_bounds__(256) deform_backward_kernel(AvIn in, const float *__restrict__ G,
                                                              const float *__restrict__ d_means,
                                                              const float *__restrict__ d_cov, float *d_cm,
                                                              float *d_cls, float *d_cq, float *d_G)
{
    __shared__ __align__(16) float sG[kMaxJoints * 12];
    __shared__ float sdG[kDeformWarps][kMaxJoints * 12]; // per-warp joint-gradient sums
    __shared__ JointShare sj[kDeformWarps][32];
    const int64_t base = (int64_t)blockIdx.x * blockDim.x;
    const int64_t i = base + threadIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int a0 = clamp_avatar(in.avatar_of[base], in.n_avatars);
    const int nj12 = in.n_joints * 12;
    for (int k = threadIdx.x; k < nj12; k += blockDim.x) sG[k] = G[(size_t)a0 * nj12 + k];
    JointShare mine;
    mine.gA[0] = mine.gA[1] = mine.gA[2] = mine.w = make_float4(0.f, 0.f, 0.f, 0.f); // no share
    mine.ids = make_ushort4(0, 0, 0, 0);
    __syncthreads();
    if (i < in.m) {
        const int av = clamp_avatar(in.avatar_of[i], in.n_avatars);
        const float *Gs = av == a0 ? sG : G + (size_t)av * nj12;
        const ushort4 id = clamp_ids(reinterpret_cast<const ushort4 *>(in.joint_ids)[i], in.n_joints);
        const float4 wt = reinterpret_cast<const float4 *>(in.weights)[i];
        float A[12];
        blend_matrix(Gs, id, wt, A);
        const float mu[3] = {in.means[3 * i], in.means[3 * i + 1], in.means[3 * i + 2]};
        const float3 ls = make_float3(in.log_scales[3 * i], in.log_scales[3 * i + 1], in.log_scales[3 * i + 2]);
        const float4 q = reinterpret_cast<const float4 *>(in.quats)[i];
        float S6[6];
        sigma_from_sq(ls, q, S6);
        const float S[9] = {S6[0], S6[1], S6[2], S6[1], S6[3], S6[4], S6[2], S6[4], S6[5]};
        const int64_t d = in.dest ? in.dest[i] : in.tb ? avatar_row(in.tb, i) : i;
        const float gm[3] = {d_means[3 * d], d_means[3 * d + 1], d_means[3 * d + 2]};
        const float *gc = d_cov + 6 * d;
        const float Gm[9] = {gc[0], 0.5f * gc[1], 0.5f * gc[2], 0.5f * gc[1], gc[3], 0.5f * gc[4],
                             0.5f * gc[2], 0.5f * gc[4], gc[5]};
        // dL/dA3 = gm mu^T + 2 Gm A3 S ; dL/da = gm
        float GA[9];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) GA[3 * r + c] = Gm[3 * r] * A[c] + Gm[3 * r + 1] * A[4 + c] + Gm[3 * r + 2] * A[8 + c];
        float gA[12];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
#pragma unroll
            for (int c = 0; c < 3; ++c)
                gA[4 * r + c] = gm[r] * mu[c] + 2.f * (GA[3 * r] * S[c] + GA[3 * r + 1] * S[3 + c] + GA[3 * r + 2] * S[6 + c]);
            gA[4 * r + 3] = gm[r];
        }
        // dL/dmu_c = A3^T gm
#pragma unroll
        for (int c = 0; c < 3; ++c) d_cm[3 * i + c] += A[c] * gm[0] + A[4 + c] * gm[1] + A[8 + c] * gm[2];
        // dL/dSigma_c = A3^T Gm A3 (symmetric)
        float gS[9];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c)
                gS[3 * r + c] = A[r] * GA[c] + A[4 + r] * GA[3 + c] + A[8 + r] * GA[6 + c];
        // Sigma = M M^T with M = R(q) diag(s)
        const float iq = 1.0f / sqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
        const float qw = q.x * iq, qx = q.y * iq, qy = q.z * iq, qz = q.w * iq;
        float R[9];
        quat_rot(qw, qx, qy, qz, R);
        const float sc[3] = {expf(ls.x), expf(ls.y), expf(ls.z)};
        float gR[9];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float gsc = 0.f;
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                const float gM = 2.f * (gS[3 * r] * R[c] + gS[3 * r + 1] * R[3 + c] + gS[3 * r + 2] * R[6 + c]) * sc[c];
                gsc += gM * R[3 * r + c];
                gR[3 * r + c] = gM * sc[c];
            }
            d_cls[3 * i + c] += gsc * sc[c];
        }
        const float gw = gR[1] * (-2 * qz) + gR[2] * (2 * qy) + gR[3] * (2 * qz) + gR[5] * (-2 * qx) +
                         gR[6] * (-2 * qy) + gR[7] * (2 * qx);
        const float gx = gR[1] * (2 * qy) + gR[2] * (2 * qz) + gR[3] * (2 * qy) + gR[4] * (-4 * qx) +
                         gR[5] * (-2 * qw) + gR[6] * (2 * qz) + gR[7] * (2 * qw) + gR[8] * (-4 * qx);
        const float gy = gR[0] * (-4 * qy) + gR[1] * (2 * qx) + gR[2] * (2 * qw) + gR[3] * (2 * qx) +
                         gR[5] * (2 * qz) + gR[6] * (-2 * qw) + gR[7] * (2 * qz) + gR[8] * (-4 * qy);
        const float gz = gR[0] * (-4 * qz) + gR[1] * (-2 * qw) + gR[2] * (2 * qx) + gR[3] * (2 * qw) +
                         gR[4] * (-4 * qz) + gR[5] * (2 * qy) + gR[6] * (2 * qx) + gR[7] * (2 * qy);
        const float dq = gw * qw + gx * qx + gy * qy + gz * qz;
        d_cq[4 * i] += (gw - qw * dq) * iq;
        d_cq[4 * i + 1] += (gx - qx * dq) * iq;
        d_cq[4 * i + 2] += (gy - qy * dq) * iq;
        d_cq[4 * i + 3] += (gz - qz * dq) * iq;
        // dL/dG[j_k] += w_k dL/dA: the CTA's avatar through the warp's owner
        // sums below, another avatar (a CTA that straddles two) directly
        if (av == a0) {
            mine.gA[0] = make_float4(gA[0], gA[1], gA[2], gA[3]);
            mine.gA[1] = make_float4(gA[4], gA[5], gA[6], gA[7]);
            mine.gA[2] = make_float4(gA[8], gA[9], gA[10], gA[11]);
            mine.w = wt;
            mine.ids = id;
        } else {
            const int ids[4] = {id.x, id.y, id.z, id.w};
            const float ws[4] = {wt.x, wt.y, wt.z, wt.w};
            float *dst = d_G + (size_t)av * nj12;
#pragma unroll
            for (int k = 0; k < 4; ++k)
#pragma unroll
                for (int e = 0; e < 12; ++e) atomicAdd(dst + 12 * ids[k] + e, ws[k] * gA[e]);
        }
    }
    // joint-owner sums over the warp's 32 Gaussians: lane l owns joints l and
    // l + 32 and adds w dL/dA wherever its joint appears (no atomics)
    sj[warp][lane] = mine;
    __syncwarp();
    for (int j = lane; j < in.n_joints; j += 32) {
        float acc[12];
#pragma unroll
        for (int e = 0; e < 12; ++e) acc[e] = 0.f;
#pragma unroll 4
        for (int q = 0; q < 32; ++q) {
            const JointShare &sh = sj[warp][q];
            const ushort4 id = sh.ids;
            const float4 w = sh.w;
            const float wj = (id.x == j ? w.x : 0.f) + (id.y == j ? w.y : 0.f) + (id.z == j ? w.z : 0.f) +
                             (id.w == j ? w.w : 0.f);
            const float4 g0 = sh.gA[0], g1 = sh.gA[1], g2 = sh.gA[2];
            acc[0] += wj * g0.x; acc[1] += wj * g0.y; acc[2] += wj * g0.z; acc[3] += wj * g0.w;
            acc[4] += wj * g1.x; acc[5] += wj * g1.y; acc[6] += wj * g1.z; acc[7] += wj * g1.w;
            acc[8] += wj * g2.x; acc[9] += wj * g2.y; acc[10] += wj * g2.z; acc[11] += wj * g2.w;
        }
#pragma unroll
        for (int e = 0; e < 12; ++e) sdG[warp][12 * j + e] = acc[e];
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nj12; k += blockDim.x) {
        float acc = 0.0f;
#pragma unroll
        for (int q = 0; q < kDeformWarps; ++q) acc += sdG[q][k];
        if (acc != 0.0f) atomicAdd(d_G + (size_t)a0 * nj12 + k, acc);
    }
}

static AvIn make_in(const gs_avatars *av, const Table *tb = nullptr)
{
    return AvIn{av->means, av->log_scales, av->quats, av->weights, av->joint_ids, av->avatar_of, av->dest,
                av->m, av->n_avatars, av->n_joints, tb};
}

void launch_deform(const gs_avatars *av, const float *G, float *out_means, float *out_cov, cudaStream_t s)
{
    const unsigned grid = (unsigned)((av->m + 255) / 256);
    if (grid) deform_kernel<<<grid, 256, 0, s>>>(make_in(av), G, out_means, out_cov);
}

void launch_deform_backward(const gs_avatars *av, const float *G, const float *d_means, const float *d_cov,
                            float *d_cm, float *d_cls, float *d_cq, float *d_G, cudaStream_t s, const Table *rows)
{
    const unsigned grid = (unsigned)((av->m + 255) / 256);
    if (grid)
        deform_backward_kernel<<<grid, 256, 0, s>>>(make_in(av, rows), G, d_means, d_cov, d_cm, d_cls, d_cq, d_G);
}

} // namespace gs
