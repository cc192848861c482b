// gs_forward.cu -- forward kernels of libgs (sm_103a).
//
// One gs_render call runs, on one stream and with no host synchronisation:
//   setup       batch table -> workspace, counters cleared
//   preprocess  one CTA per env-aligned chunk of Gaussians, each warp walking
//               32-Gaussian rounds over the views of the env: FP32 depth key +
//               near cull, covariance (or LBS of posed avatar rows, fused),
//               EWA projection with 0.3 px dilation, conic, radius, exact
//               per-pixel footprint range; visible entries queued per warp for
//               SH-3 colour on full warps; writes the 48-byte record, its
//               64-byte gradient row, the visibility bit, and the chunk's tile
//               counts (a shared 2D difference array, flushed per CTA)
//   scan        exclusive scan of the bin counts -> tile ranges [start, end),
//               heavy-bin list, large-bin chunk list
//   scatter     one (depth key << 32 | record) key per touched tile, placed in
//               its bin at the chunk's offset (order inside a bin is arbitrary)
//   sort        each bin sorted by key = (FP32 depth bits, record index), so the
//               result equals a stable sort of the keys emitted in record order
//               (gs_sort.cu)
//   blend       one CTA per (view, tile) -- or a persistent grid pulling tiles
//               from an atomic queue, heaviest first -- stages batches of
//               records in shared memory and blends front to back per pixel
//               with early exit once every pixel of the warp has stopped;
//               flags in its key every pair that some pixel blended.  At
//               2 x 1 pixels per thread (blendq_tile) each 4 x 4 quarter of a
//               warp's 8 x 8 block walks its own list of the batch entries
//               whose window reaches it, and the quarters that blended each
//               pair are kept for the backward.
// The rasterisation follows the 3DGS method the paper builds its renderer on
// (Sec. 2.2, Sec. 3.2); the exact definition is the one in include/gs.h.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "gs_internal.cuh"
#include "gs_launch.h"

namespace gs {

// ---------------------------------------------------------------------------
// setup
// ---------------------------------------------------------------------------
__global__ void setup_kernel(const Table tb, Ws w)
{
    const int32_t *src = reinterpret_cast<const int32_t *>(&tb);
    int32_t *dst = reinterpret_cast<int32_t *>(w.tb);
    const int n = (int)(sizeof(Table) / 4);
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
    uint32_t *h = reinterpret_cast<uint32_t *>(w.hdr);
    for (int i = threadIdx.x; i < (int)(sizeof(Header) / 4); i += blockDim.x) h[i] = 0;
}

// ---------------------------------------------------------------------------
// preprocess
// ---------------------------------------------------------------------------
struct GaussIn {
    const float *means, *log_scales, *quats, *ologits, *cov3d;
    const void *sh;
    // fused LBS (gs_render_avatars): the avatar rows of every env are posed
    // here from their canonical Gaussians instead of read from means / cov3d
    const float *av_means, *av_log_scales, *av_quats, *av_weights, *av_G;
    const uint16_t *av_ids;
    const int32_t *av_of;
    int32_t n_avatars, n_joints;
};

// The SH direction of a posed avatar Gaussian evaluated in its canonical
// frame: A3^-1 (mu' - C), A3 the linear part of its blended skinning matrix
// (inverse by the adjugate; the length does not matter, the colour normalises).
__device__ __forceinline__ void canonical_direction(const GaussIn &gin, int64_t i, float &d0, float &d1, float &d2)
{
    const int a = clamp_avatar(__ldg(gin.av_of + i), gin.n_avatars);
    const ushort4 id = clamp_ids(__ldg(reinterpret_cast<const ushort4 *>(gin.av_ids) + i), gin.n_joints);
    float A[12];
    blend_matrix(gin.av_G + (size_t)a * gin.n_joints * 12, id, __ldg(reinterpret_cast<const float4 *>(gin.av_weights) + i),
                 A);
    const float a00 = A[0], a01 = A[1], a02 = A[2], a10 = A[4], a11 = A[5], a12 = A[6], a20 = A[8], a21 = A[9],
                a22 = A[10];
    const float c00 = a11 * a22 - a12 * a21, c01 = a02 * a21 - a01 * a22, c02 = a01 * a12 - a02 * a11;
    const float c10 = a12 * a20 - a10 * a22, c11 = a00 * a22 - a02 * a20, c12 = a02 * a10 - a00 * a12;
    const float c20 = a10 * a21 - a11 * a20, c21 = a01 * a20 - a00 * a21, c22 = a00 * a11 - a01 * a10;
    const float det = a00 * c00 + a01 * c10 + a02 * c20;
    const float s = det < 0.0f ? -1.0f : 1.0f; // adj = det A^-1: keep the orientation of A^-1
    const float x = d0, y = d1, z = d2;
    d0 = s * (c00 * x + c01 * y + c02 * z);
    d1 = s * (c10 * x + c11 * y + c12 * z);
    d2 = s * (c20 * x + c21 * y + c22 * z);
}

// Every preprocess / scatter CTA owns a chunk of kChunk consecutive Gaussians.
// Per-(view, tile) counts and cursors of a chunk that lies inside one env are
// aggregated in shared memory, so that global atomics are one per (CTA, bin)
// rather than one per pair.

constexpr int kPreThreads = 256;

struct Chunk {
    int64_t g0, g1;
    int e0, e1, vb, nv, kmax;
    bool hist;
};

__device__ __forceinline__ void chunk_setup(const Table *tb, int cta, Chunk &c)
{
    int lo = 0, hi = tb->n_envs - 1; // env of the chunk: last e with chunk_off[e] <= cta
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tb->chunk_off[mid] <= cta) lo = mid;
        else hi = mid - 1;
    }
    c.e0 = c.e1 = lo;
    c.g0 = tb->env_off[lo] + (int64_t)(cta - tb->chunk_off[lo]) * tb->chunk;
    c.g1 = min(c.g0 + tb->chunk, tb->env_off[lo + 1]);
    c.vb = tb->env_view_begin[lo];
    c.nv = tb->env_view_begin[lo + 1] - c.vb;
    c.kmax = c.nv;
    c.hist = c.nv * tb->tiles_per_view <= kHistCap;
}

// One visible (view, Gaussian) waiting for its colour, record and bin counts.
struct QEntry {
    uint32_t rec, g;
    float uc, vc, zk, hx, hy, A, B, C, op, d0, d1, d2;
    uint16_t x0, x1, y0, y1;
    uint16_t v, k;
    uint32_t pad[3];
};
static_assert(sizeof(QEntry) % 16 == 0, "queue entries are copied as 16-byte vectors");

// Phase 2, one entry per lane of a warp: colour, record, visibility bit and
// bin counts of a queued visible (view, Gaussian).
template <int SHT>
__device__ __forceinline__ void finish_entry(const QEntry &en, bool active, uint32_t *hist, const Chunk &c,
                                             const GaussIn &gin, const Ws &w, const Table *tb)
{
    if (active) {
        const int tpv = tb->tiles_per_view, tx_n = tb->tiles_x, tw = tb->tile_w, th = tb->tile_h;
        float idn;
        const float3 dir = view_dir(en.d0, en.d1, en.d2, idn);
        const float3 col = sh_colour<SHT>(gin.sh, en.g, dir.x, dir.y, dir.z);
        const float op = en.op;
        const int bx0 = en.x0 / tw, bx1 = en.x1 / tw, by0 = en.y0 / th, by1 = en.y1 / th;
        float4 *dst = w.rec + 3 * (size_t)en.rec;
        dst[0] = make_float4(en.uc, en.vc, en.hx, en.hy);
        dst[1] = make_float4(en.A, en.B, en.C, op);
        dst[2] = make_float4(col.x, col.y, col.z, en.zk);
        // the record's gradient row starts at zero for the backward, which
        // accumulates into its first 10 floats; beside them the opacity (the
        // backward would otherwise gather the logit) and which colour channels
        // were clamped at 0 (they pass no gradient)
        float4 *dr = reinterpret_cast<float4 *>(w.d_rec + (size_t)en.rec * kGradStride);
        const uint32_t clamped = (col.x > 0.f ? 0u : 1u) | (col.y > 0.f ? 0u : 2u) | (col.z > 0.f ? 0u : 4u);
        dr[0] = dr[1] = make_float4(0.f, 0.f, 0.f, 0.f);
        dr[2] = make_float4(0.f, 0.f, op, 0.f);
        dr[3] = make_float4(__uint_as_float(clamped), 0.f, 0.f, 0.f);
        if (c.hist) {
            // the chunk's counts as a 2D difference array: +1 / -1 at the corners
            // of the tile rectangle (wrapping arithmetic), summed up once per CTA
            uint32_t *hk = hist + en.k * tpv;
            const bool xe = bx1 + 1 < tx_n, ye = by1 + 1 < tb->tiles_y;
            atomicAdd(hk + by0 * tx_n + bx0, 1u);
            if (xe) atomicAdd(hk + by0 * tx_n + bx1 + 1, 0xffffffffu);
            if (ye) atomicAdd(hk + (by1 + 1) * tx_n + bx0, 0xffffffffu);
            if (xe && ye) atomicAdd(hk + (by1 + 1) * tx_n + bx1 + 1, 1u);
        } else {
            uint32_t *hk = w.bin_fcount + (size_t)en.v * tpv;
            for (int by = by0; by <= by1; ++by)
                for (int bx = bx0; bx <= bx1; ++bx) atomicAdd(hk + by * tx_n + bx, 1u);
        }
    }
    // visibility bit, aggregated over the lanes that share a word
    const uint32_t word = active ? (en.rec >> 5) : 0xffffffffu;
    const unsigned grp = __match_any_sync(0xffffffffu, word);
    const uint32_t bits = __reduce_or_sync(grp, active ? (1u << (en.rec & 31)) : 0u);
    if (active && (threadIdx.x & 31) == __ffs(grp) - 1) atomicOr(w.vis + word, bits);
}

// One (view, Gaussian) that passed the near cull and the conservative image
// test, waiting for its projection.
struct AEntry {
    uint32_t g;
    uint16_t k;    // view slot of the chunk's env
    uint16_t kind; // covariance source: 0 (log-scales, rotation) in c, 1 posed covariance in c, 2 cov3d
    float mx, my, mz, zk, lo;
    float c[7];
    uint32_t pad[2];
};
static_assert(sizeof(AEntry) % 16 == 0, "queue entries are copied as 16-byte vectors");

// Conservative image test before the projection: false only if the Gaussian
// can touch no pixel.  Its radius is r = ceil(3 sqrt(lambda)) with lambda <=
// lambda_max(Sigma2) + sqrt(0.1) <= trace(J W Sigma W^T J^T) + 0.6 + 0.32 <=
// |J|_F^2 lambda_max(Sigma) + 0.92 (W a rotation), and a pixel i is covered
// only if |u - i| <= r; the bound carries 1% and 2 px of slack for FP32.
__device__ __forceinline__ bool may_touch_image(float mx, float my, float mz, float zk, float lam3,
                                                const gs_camera &cam, int W, int H)
{
    const float d0 = mx - cam.C[0], d1 = my - cam.C[1], d2 = mz - cam.C[2];
    const float px = cam.R[0] * d0 + cam.R[1] * d1 + cam.R[2] * d2;
    const float py = cam.R[3] * d0 + cam.R[4] * d1 + cam.R[5] * d2;
    const float iz = 1.0f / zk;
    const float limx = 1.3f * (0.5f * (float)W / cam.fx), limy = 1.3f * (0.5f * (float)H / cam.fy);
    const float tx = fminf(limx, fmaxf(-limx, px * iz)), ty = fminf(limy, fmaxf(-limy, py * iz));
    const float jx = cam.fx * iz, jy = cam.fy * iz;
    const float jf2 = jx * jx * (1.0f + tx * tx) + jy * jy * (1.0f + ty * ty);
    const float rb = 3.03f * sqrtf(jf2 * lam3 + 0.92f) + 2.0f;
    const float u = cam.fx * px * iz + cam.cx, v = cam.fy * py * iz + cam.cy;
    return u + rb >= 0.0f && u - rb <= (float)(W - 1) && v + rb >= 0.0f && v - rb <= (float)(H - 1);
}

// Each warp walks 32-Gaussian rounds of the chunk on its own (no CTA barrier in
// the loop), in three stages joined by ring queues in shared memory, so that
// the costly stages run on full warps:
//   A  every lane: FP32 depth key and near cull per view, then a conservative
//      image test from the largest scale (cheap, on all Gaussians);
//   B  32 queued survivors: covariance, EWA projection, conic, radius, pixel
//      window, exact pixel ranges;
//   C  32 queued visible entries: SH colour, record, gradient row, bin counts.
// Each round's means, logits, scales and rotations are copied into a per-warp
// shared-memory ring by cp.async two rounds ahead (one on the fused path), so
// that two rounds of loads are in flight while a round is processed.
constexpr int kWarpQ = 64; // each queue grows by at most 32 before it is drained below 32
constexpr int kFusedJointSlots = 96; // joint matrices a fused-LBS CTA stages (4 avatars of 24 joints)
constexpr int kMaxViewsPerChunk = 16; // cameras of a chunk's env staged in shared memory
// A round's inputs in shared memory: 32 rotations (float4), then 32 each of
// mean x, y, z, logit and log-scale x, y, z (floats): 1408 bytes per warp.
constexpr int kRingF4 = 32 + 7 * 32 / 4;
// rounds in the ring (a launch parameter): three, two rounds of loads in
// flight, where two CTAs per SM still fit; else two

// FUSED: the batch's avatar rows are posed by LBS here (gs_render_avatars); a
// separate instantiation so that the plain path carries none of its registers
template <int SHT, bool FUSED>
__global__ void __launch_bounds__(kPreThreads, 2) preprocess_kernel(const gs_camera *__restrict__ cams, GaussIn gin,
                                                                    Ws w, const __grid_constant__ Table tbp,
                                                                    int n_ring)
{
    extern __shared__ __align__(16) unsigned char smem_pre[];
    __shared__ gs_camera s_cam[kMaxViewsPerChunk];
    __shared__ int64_t s_roff[kMaxViewsPerChunk];
    // fused LBS: the joint matrices of the first avatars of the chunk's avatar rows
    __shared__ __align__(16) float s_G[FUSED ? kFusedJointSlots * 12 : 4];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int kNW = kPreThreads / 32;
    AEntry *qa = reinterpret_cast<AEntry *>(smem_pre) + warp * kWarpQ;
    QEntry *qb = reinterpret_cast<QEntry *>(smem_pre + kNW * kWarpQ * sizeof(AEntry)) + warp * kWarpQ;
    uint32_t *hist = reinterpret_cast<uint32_t *>(smem_pre + kNW * kWarpQ * (sizeof(AEntry) + sizeof(QEntry)) +
                                                  kNW * n_ring * kRingF4 * sizeof(float4));
    // the table as a kernel parameter: its fields are constant-bank operands,
    // never reloaded after the global stores of the stages
    const Table *tb = &tbp;
    Chunk c;
    chunk_setup(tb, blockIdx.x, c);
    const int tpv = tb->tiles_per_view;
    if (c.hist)
        for (int i = threadIdx.x; i < c.nv * tpv; i += blockDim.x) hist[i] = 0u;
    const bool cam_smem = c.nv <= kMaxViewsPerChunk;
    if (cam_smem)
        for (int k = threadIdx.x; k < c.nv; k += blockDim.x) {
            const int v = tb->env_views[c.vb + k];
            s_cam[k] = cams[v];
            s_roff[k] = tb->view_rec_off[v];
        }
    const int64_t cov_begin = tb->env_cov_begin[c.e0];
    // avatars a_lo .. a_lo + n_stage - 1 (from the chunk's first avatar row) are
    // staged in shared memory; rows of other avatars read their matrices from
    // global memory
    int a_lo = 0, n_stage = 0;
    if (FUSED && gin.n_joints > 0 && max(c.g0, cov_begin) < c.g1) {
        a_lo = clamp_avatar(__ldg(gin.av_of + tb->env_av_base[c.e0] + (max(c.g0, cov_begin) - cov_begin)),
                            gin.n_avatars);
        n_stage = min(kFusedJointSlots / gin.n_joints, gin.n_avatars - a_lo);
        const int nf = n_stage * gin.n_joints * 12;
        const float *src = gin.av_G + (size_t)a_lo * gin.n_joints * 12;
        for (int k = threadIdx.x; k < nf; k += blockDim.x) s_G[k] = __ldg(src + k);
    }
    __syncthreads();
    const int W = tb->W, H = tb->H;
    const float near_plane = tb->near_plane;
    const bool count_evals = (tb->flags & GS_FLAG_COUNT_EVALS) != 0;
    const int nwarps = blockDim.x >> 5;
    const int64_t env_base = tb->env_off[c.e0];
    const bool env_cov = gin.cov3d != nullptr;
    int ha = 0, ta = 0, hb = 0, tb_ = 0; // ring queues of this warp: A (to project), B (visible)

    // stage C on the 32 oldest visible entries (or the last few)
    auto stage_c = [&](int n) {
        const bool act = lane < n;
        QEntry mine;
        if (act) mine = qb[(hb + lane) & (kWarpQ - 1)];
        hb += n;
        __syncwarp();
        finish_entry<SHT>(mine, act, hist, c, gin, w, tb);
    };
    // stage B on the 32 oldest queued survivors (or the last few)
    auto stage_b = [&](int n) {
        const bool act = lane < n;
        bool vis = false;
        QEntry en;
        if (act) {
            const AEntry ea = qa[(ha + lane) & (kWarpQ - 1)];
            const int k = ea.k;
            const int v = cam_smem ? 0 : tb->env_views[c.vb + k];
            const gs_camera &cam = cam_smem ? s_cam[k] : cams[v];
            Proj pj;
            bool proj_ok;
            if (ea.kind == 0) {
                // scales and rotation: the factor form (a thin Gaussian's conic
                // without cancellation)
                float M[9];
                factor_from_sq(make_float3(ea.c[0], ea.c[1], ea.c[2]), make_float4(ea.c[3], ea.c[4], ea.c[5], ea.c[6]),
                               M);
                proj_ok = project_ewa_factor(ea.mx, ea.my, ea.mz, ea.zk, M, cam, W, H, pj);
            } else {
                float S[6];
                if (ea.kind == 1) {
#pragma unroll
                    for (int i = 0; i < 6; ++i) S[i] = ea.c[i];
                } else {
#pragma unroll
                    for (int i = 0; i < 6; ++i) S[i] = __ldg(gin.cov3d + 6 * (int64_t)ea.g + i);
                }
                proj_ok = project_ewa(ea.mx, ea.my, ea.mz, ea.zk, S, cam, W, H, pj);
            }
            if (proj_ok) {
                const float r = radius_px(pj);
                const float idet = 1.0f / pj.det;
                const float cA = pj.c * idet, cB = -pj.b * idet, cC = pj.a * idet;
                const float op = 1.0f / (1.0f + expf(-ea.lo));
                // the pixel window: the square footprint narrowed to where
                // alpha can reach 1/255 (the square alone when evaluations are
                // counted, so that the count follows the definition)
                float hx = r, hy = r;
                if (!count_evals) alpha_window(op, cA, cB, cC, r, hx, hy);
                int x0, x1, y0, y1;
                if (hx >= 0.0f && pixel_range(pj.uc, hx, cam.cx, W, x0, x1) &&
                    pixel_range(pj.vc, hy, cam.cy, H, y0, y1)) {
                    vis = true;
                    const int64_t g = ea.g;
                    en.rec = (uint32_t)((cam_smem ? s_roff[k] : tb->view_rec_off[v]) + (g - env_base));
                    en.g = ea.g;
                    en.uc = pj.uc; en.vc = pj.vc; en.zk = ea.zk; en.hx = hx; en.hy = hy; en.op = op;
                    en.A = cA; en.B = cB; en.C = cC;
                    en.d0 = pj.d0; en.d1 = pj.d1; en.d2 = pj.d2;
                    if (FUSED && (tb->flags & GS_FLAG_AVATAR_CANONICAL_SH) && g >= cov_begin)
                        canonical_direction(gin, tb->env_av_base[c.e0] + (g - cov_begin), en.d0, en.d1, en.d2);
                    en.x0 = (uint16_t)x0; en.x1 = (uint16_t)x1; en.y0 = (uint16_t)y0; en.y1 = (uint16_t)y1;
                    en.v = (uint16_t)(cam_smem ? tb->env_views[c.vb + k] : v); en.k = (uint16_t)k;
                    // its SH row, read by stage C once 32 entries are queued
                    prefetch_l2(sh_row<SHT>(gin.sh, g), sh_row_bytes<SHT>());
                }
            }
        }
        ha += n;
        const unsigned bal = __ballot_sync(0xffffffffu, vis);
        if (vis) qb[(tb_ + __popc(bal & ((1u << lane) - 1u))) & (kWarpQ - 1)] = en;
        tb_ += __popc(bal);
        __syncwarp();
        if (tb_ - hb >= 32) stage_c(32);
    };

    // the round ring: round r's inputs land in buffer r % n_ring, issued
    // n_ring - 1 rounds ahead by cp.async, one commit group per round and lane
    float4 *ring = reinterpret_cast<float4 *>(smem_pre + kNW * kWarpQ * (sizeof(AEntry) + sizeof(QEntry))) +
                   warp * n_ring * kRingF4;
    auto issue_round = [&](int64_t gg, int slot) {
        float4 *q4 = ring + slot * kRingF4;
        float *f = reinterpret_cast<float *>(q4 + 32);
        if (gg < c.g1) {
            cp_async4(f + lane, gin.means + 3 * gg);
            cp_async4(f + 32 + lane, gin.means + 3 * gg + 1);
            cp_async4(f + 64 + lane, gin.means + 3 * gg + 2);
            cp_async4(f + 96 + lane, gin.ologits + gg);
            if (!((env_cov || FUSED) && gg >= cov_begin)) { // posed rows take their covariance elsewhere
                cp_async4(f + 128 + lane, gin.log_scales + 3 * gg);
                cp_async4(f + 160 + lane, gin.log_scales + 3 * gg + 1);
                cp_async4(f + 192 + lane, gin.log_scales + 3 * gg + 2);
                cp_async16(q4 + lane, reinterpret_cast<const float4 *>(gin.quats) + gg);
            }
        }
        cp_async_commit();
    };
    int64_t g = c.g0 + warp * 32 + lane;
    const int64_t gstep = 32 * nwarps;
    for (int r = 0; r < n_ring - 1; ++r) issue_round(g + r * gstep, r);
    int slot = 0, slot_next = n_ring - 1; // buffers of this round and of the round issued next
    for (int64_t base = c.g0 + warp * 32; base < c.g1; base += gstep, g += gstep) {
        const bool valid = g < c.g1;
        if (n_ring == 3) cp_async_wait<1>(); // this round's group has landed
        else cp_async_wait<0>();
        float mx = 0.f, my = 0.f, mz = 0.f, lo = 0.f;
        float3 cls = make_float3(0.f, 0.f, 0.f);
        float4 cq = make_float4(1.f, 0.f, 0.f, 0.f);
        {
            const float4 *q4 = ring + slot * kRingF4;
            const float *f = reinterpret_cast<const float *>(q4 + 32);
            if (valid) {
                mx = f[lane];
                my = f[32 + lane];
                mz = f[64 + lane];
                lo = f[96 + lane];
                if (!((env_cov || FUSED) && g >= cov_begin)) {
                    cls = make_float3(f[128 + lane], f[160 + lane], f[192 + lane]);
                    cq = q4[lane];
                }
            }
        }
        // the buffer of the previous round is free again (its values were used there)
        issue_round(g + (n_ring - 1) * gstep, slot_next);
        slot = slot + 1 == n_ring ? 0 : slot + 1;
        slot_next = slot_next + 1 == n_ring ? 0 : slot_next + 1;
        const int nv = valid ? c.nv : 0;
        // covariance source of this lane's Gaussian and the largest variance
        // of its 3D covariance for the image test
        uint16_t kind = 0;
        float cc[7] = {cls.x, cls.y, cls.z, cq.x, cq.y, cq.z, cq.w};
        float lam3 = __expf(2.0f * fmaxf(cls.x, fmaxf(cls.y, cls.z))) * 1.001f;
        if (FUSED && valid && g >= cov_begin) {
            // posed mean and covariance by LBS, never written to memory
            const int64_t i = tb->env_av_base[c.e0] + (g - cov_begin);
            const int a = clamp_avatar(__ldg(gin.av_of + i), gin.n_avatars);
            const ushort4 id = clamp_ids(__ldg(reinterpret_cast<const ushort4 *>(gin.av_ids) + i), gin.n_joints);
            const float4 wt = __ldg(reinterpret_cast<const float4 *>(gin.av_weights) + i);
            const float *Gs = a - a_lo >= 0 && a - a_lo < n_stage ? s_G + (a - a_lo) * gin.n_joints * 12
                                                                 : gin.av_G + (size_t)a * gin.n_joints * 12;
            float mu[3], S[6];
            lbs_gaussian(Gs, id, wt,
                         make_float3(__ldg(gin.av_means + 3 * i), __ldg(gin.av_means + 3 * i + 1),
                                     __ldg(gin.av_means + 3 * i + 2)),
                         make_float3(__ldg(gin.av_log_scales + 3 * i), __ldg(gin.av_log_scales + 3 * i + 1),
                                     __ldg(gin.av_log_scales + 3 * i + 2)),
                         __ldg(reinterpret_cast<const float4 *>(gin.av_quats) + i), mu, S);
            mx = mu[0];
            my = mu[1];
            mz = mu[2];
            kind = 1;
#pragma unroll
            for (int j = 0; j < 6; ++j) cc[j] = S[j];
            lam3 = fmaxf(S[0] + S[3] + S[5], 0.0f) * 1.001f; // >= lambda_max of a PSD matrix
        } else if (env_cov && valid && g >= cov_begin) {
            kind = 2;
            lam3 = INFINITY; // read in stage B; no image test
        }
        for (int k = 0; k < c.kmax; ++k) {
            bool push = false;
            float zk = 0.0f;
            if (k < nv) {
                const int v = cam_smem ? 0 : tb->env_views[c.vb + k];
                const gs_camera &cam = cam_smem ? s_cam[k] : cams[v];
                zk = depth_key(mx, my, mz, cam);
                push = zk > near_plane && (kind == 2 || may_touch_image(mx, my, mz, zk, lam3, cam, W, H));
            }
            const unsigned bal = __ballot_sync(0xffffffffu, push);
            if (push) {
                AEntry ea;
                ea.g = (uint32_t)g;
                ea.k = (uint16_t)k;
                ea.kind = kind;
                ea.mx = mx; ea.my = my; ea.mz = mz; ea.zk = zk; ea.lo = lo;
#pragma unroll
                for (int j = 0; j < 7; ++j) ea.c[j] = cc[j];
                qa[(ta + __popc(bal & ((1u << lane) - 1u))) & (kWarpQ - 1)] = ea;
            }
            ta += __popc(bal);
            __syncwarp();
            if (ta - ha >= 32) stage_b(32);
        }
    }
    cp_async_wait<0>();
    if (ta > ha) stage_b(ta - ha);
    if (tb_ > hb) stage_c(tb_ - hb);
    __syncthreads();
    if (c.hist) {
        // 2D inclusive prefix sums of the difference array: rows (one warp per
        // row, shuffle scan in 32-tile pieces), then columns (one thread each)
        const int tx_n = tb->tiles_x, ty_n = tb->tiles_y;
        for (int r = warp; r < c.nv * ty_n; r += nwarps) {
            uint32_t *row = hist + (r / ty_n) * tpv + (r % ty_n) * tx_n;
            uint32_t carry = 0;
            for (int x0 = 0; x0 < tx_n; x0 += 32) {
                uint32_t v = x0 + lane < tx_n ? row[x0 + lane] : 0u;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t u = __shfl_up_sync(0xffffffffu, v, o);
                    if (lane >= o) v += u;
                }
                if (x0 + lane < tx_n) row[x0 + lane] = v + carry;
                carry += __shfl_sync(0xffffffffu, v, 31);
            }
        }
        __syncthreads();
        for (int col = threadIdx.x; col < c.nv * tx_n; col += blockDim.x) {
            uint32_t *cp = hist + (col / tx_n) * tpv + (col % tx_n);
            uint32_t acc = 0;
            for (int y = 0; y < ty_n; ++y) {
                acc += cp[y * tx_n];
                cp[y * tx_n] = acc;
            }
        }
        __syncthreads();
        // the returned old count is this chunk's offset inside the bin
        uint32_t *rel = w.rel + (size_t)blockIdx.x * kHistCap;
        for (int i = threadIdx.x; i < c.nv * tpv; i += blockDim.x) {
            const uint32_t cnt = hist[i];
            if (cnt) {
                const int v = tb->env_views[c.vb + i / tpv];
                rel[i] = atomicAdd(w.bin_count + (size_t)v * tpv + (i % tpv), cnt);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// scan of the bin counts (single CTA, any number of bins)
// ---------------------------------------------------------------------------
constexpr int kScanPer = 4; // consecutive bins per thread and tile

// Bins with at least heavy_min pairs go to the heavy-first list, bucketed by
// floor(log2(count)) from the largest bucket down (order inside a bucket is
// arbitrary: it only steers scheduling); heavy_min is the smallest power of two
// >= kHeavyMin that keeps the list within kHeavyCap entries.
__global__ void __launch_bounds__(1024) scan_bins_kernel(Ws w)
{
    const int nb = w.tb->n_bins;
    const int T = blockDim.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned long long cap = (unsigned long long)w.tb->pair_capacity;
    __shared__ unsigned long long wsum[32];
    __shared__ unsigned long long carry;
    __shared__ uint32_t lg[33], bucket_at[33];
    __shared__ uint32_t n_big, max_pass, smax, hmin, nh;
    __shared__ uint32_t hcnt[kHeavyCap];
    __shared__ uint32_t hscan[32];
    if (threadIdx.x < 33) lg[threadIdx.x] = 0;
    if (threadIdx.x == 0) {
        n_big = max_pass = smax = 0;
        carry = 0;
    }
    __syncthreads();
    uint32_t mx = 0;
    const int tile = T * kScanPer;
    for (int t0 = 0; t0 < nb; t0 += tile) {
        const int b0 = t0 + threadIdx.x * kScanPer;
        uint32_t c[kScanPer];
        unsigned long long s = 0;
#pragma unroll
        for (int k = 0; k < kScanPer; ++k) {
            c[k] = b0 + k < nb ? w.bin_count[b0 + k] + w.bin_fcount[b0 + k] : 0u;
            s += c[k];
        }
        unsigned long long incl = s;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned long long v = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += v;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            unsigned long long x = lane < (T >> 5) ? wsum[lane] : 0ull;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const unsigned long long v = __shfl_up_sync(0xffffffffu, x, off);
                if (lane >= off) x += v;
            }
            wsum[lane] = x;
        }
        __syncthreads();
        // pair counts beyond the capacity (or 32 bits) are clamped: every bin
        // range stays inside [0, capacity) and the status word records it
        unsigned long long run = carry + (warp ? wsum[warp - 1] : 0ull) + incl - s;
#pragma unroll
        for (int k = 0; k < kScanPer; ++k) {
            const int i = b0 + k;
            if (i >= nb) break;
            const unsigned long long lo = min(run, cap);
            w.bin_start[i] = (uint32_t)lo;
            run += c[k];
            mx = max(mx, c[k]);
            if (c[k] >= (uint32_t)kHeavyMin) atomicAdd(&lg[32 - __clz(c[k])], 1u);
            // bins of more than kSortChunk pairs (after the clamp) are sorted in
            // kSortChunk-long chunks and merged: one list entry per chunk
            const uint32_t n = (uint32_t)(min(run, cap) - lo);
            if (n > (uint32_t)kSortChunk) {
                const uint32_t nch = (n + kSortChunk - 1) / kSortChunk;
                const uint32_t at = atomicAdd(&n_big, nch);
                for (uint32_t t = 0; t < nch; ++t) w.big_list[at + t] = ((unsigned long long)i << 32) | t;
                atomicMax(&max_pass, (uint32_t)(32 - __clz(nch - 1u)));
            }
        }
        __syncthreads();
        if (threadIdx.x == T - 1) carry += wsum[(T >> 5) - 1];
        __syncthreads();
    }
    mx = __reduce_max_sync(0xffffffffu, mx);
    if (lane == 0) atomicMax(&smax, mx);
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned long long total = carry;
        w.bin_start[nb] = (uint32_t)min(total, cap);
        w.hdr->n_pairs = (uint32_t)min(total, 0xffffffffull);
        if (total > cap) set_status(w.hdr, GS_ERR_CAPACITY);
        w.hdr->max_bin = smax;
        w.hdr->n_big = n_big;
        w.hdr->max_pass = max_pass;
        // heavy threshold, then the start of every included bucket, largest first
        uint32_t acc = 0, bth = 33;
        for (int b = 32; b >= 0; --b) {
            if (acc + lg[b] > (uint32_t)kHeavyCap) break;
            acc += lg[b];
            if (lg[b]) bth = b;
        }
        uint32_t th = bth == 33 ? 0xffffffffu : (bth == 0 ? 0u : (1u << (bth - 1)));
        th = max(th, (uint32_t)kHeavyMin);
        hmin = th;
        uint32_t at = 0;
        for (int b = 32; b >= 0; --b) {
            bucket_at[b] = at;
            const bool in = b > 0 && (1u << (b - 1)) >= th;
            if (in) at += lg[b];
        }
        nh = at;
    }
    __syncthreads();
    const uint32_t th = hmin;
    // heavy list and heavy_of, one more coalesced pass over the counts
    for (int t0 = 0; t0 < nb; t0 += tile) {
        const int b0 = t0 + threadIdx.x * kScanPer;
#pragma unroll
        for (int k = 0; k < kScanPer; ++k) {
            const int i = b0 + k;
            if (i >= nb) break;
            const uint32_t c = w.bin_count[i] + w.bin_fcount[i];
            int32_t h = -1;
            if (c >= th) {
                h = (int32_t)atomicAdd(&bucket_at[32 - __clz(c)], 1u);
                w.heavy[h] = (uint32_t)i;
                hcnt[h] = c;
            }
            w.heavy_of[i] = h;
        }
    }
    __syncthreads();
    // backward segments of the heavy bins: ceil(count / kSeg) each, scanned
    const uint32_t n_h = nh;
    uint32_t seg[kHeavyCap / 1024];
    uint32_t ssum = 0;
#pragma unroll
    for (int k = 0; k < kHeavyCap / 1024; ++k) {
        const uint32_t i = threadIdx.x * (kHeavyCap / 1024) + k;
        seg[k] = i < n_h ? (hcnt[i] + kSeg - 1) / kSeg : 0u;
        ssum += seg[k];
    }
    uint32_t sincl = ssum;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, sincl, off);
        if (lane >= off) sincl += v;
    }
    if (lane == 31) hscan[warp] = sincl;
    __syncthreads();
    if (warp == 0) {
        uint32_t x = lane < (T >> 5) ? hscan[lane] : 0u;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, x, off);
            if (lane >= off) x += v;
        }
        hscan[lane] = x;
    }
    __syncthreads();
    uint32_t srun = (warp ? hscan[warp - 1] : 0u) + sincl - ssum;
#pragma unroll
    for (int k = 0; k < kHeavyCap / 1024; ++k) {
        const uint32_t i = threadIdx.x * (kHeavyCap / 1024) + k;
        if (i < n_h) w.heavy_seg[i] = srun;
        srun += seg[k];
    }
    if (threadIdx.x == T - 1) {
        w.heavy_seg[n_h] = srun;
        w.hdr->n_heavy_items = srun;
        w.hdr->n_heavy = n_h;
        w.hdr->heavy_min = n_h > 0 ? th : 0xffffffffu;
    }
}

// ---------------------------------------------------------------------------
// scatter: one key per (visible record, touched tile)
// ---------------------------------------------------------------------------
// hist_words: the preprocess's (view, tile) counter count; the shared memory
// holds that many slots and one chunk of record indices (the registers allow
// 3 CTAs per SM)
__global__ void __launch_bounds__(256, 3) scatter_kernel(const gs_camera *__restrict__ cams, Ws w, int hist_words)
{
    extern __shared__ uint32_t smem_sc[];
    uint32_t *base = smem_sc;              // [hist_words] next free slot per (view slot, tile)
    uint32_t *list = smem_sc + hist_words; // visible records of one view slot, compacted
    __shared__ int list_n;
    const Table *tb = w.tb;
    Chunk c;
    chunk_setup(tb, blockIdx.x, c);
    const int W = tb->W, H = tb->H, tw = tb->tile_w, th = tb->tile_h, tx_n = tb->tiles_x, tpv = tb->tiles_per_view;
    const uint64_t cap = (uint64_t)tb->pair_capacity;
    // first slot of each of this chunk's bins: bin start + the chunk's offset
    // (chunks with more bins than shared memory holds place their pairs after
    // the aggregated ones of each bin, one global cursor atomic per pair)
    const uint32_t *rel = w.rel + (size_t)blockIdx.x * kHistCap;
    if (c.hist)
        for (int i = threadIdx.x; i < c.nv * tpv; i += blockDim.x) {
            const size_t bin = (size_t)tb->env_views[c.vb + i / tpv] * tpv + (i % tpv);
            base[i] = w.bin_start[bin] + rel[i]; // unused where the chunk has no pair
        }
    const bool overflow = (uint64_t)w.hdr->n_pairs > cap;
    const int64_t loc0 = c.g0 - tb->env_off[c.e0], loc1 = c.g1 - tb->env_off[c.e0];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    for (int k = 0; k < c.nv; ++k) {
        // visible records of view slot k, compacted
        if (threadIdx.x == 0) list_n = 0;
        __syncthreads();
        const int v = tb->env_views[c.vb + k];
        const int64_t roff = tb->view_rec_off[v];
        const int64_t r0 = roff + loc0, r1 = roff + loc1;
        const int64_t wlo = r0 >> 5, whi = (r1 - 1) >> 5;
        for (int64_t wd = wlo + threadIdx.x; wd <= whi; wd += blockDim.x) {
            uint32_t bits = __ldg(w.vis + wd);
            const int64_t b0 = wd << 5;
            if (b0 < r0) bits &= ~((1u << (uint32_t)(r0 - b0)) - 1u);
            if (b0 + 32 > r1) bits &= (uint32_t)((1ull << (uint32_t)(r1 - b0)) - 1ull);
            if (!bits) continue;
            int at = atomicAdd(&list_n, __popc(bits));
            while (bits) {
                const int bb = __ffs(bits) - 1;
                bits &= bits - 1u;
                list[at++] = (uint32_t)(b0 + bb);
            }
        }
        __syncthreads();
        const gs_camera &cam = cams[v];
        uint32_t *bk = base + (c.hist ? k * tpv : 0);
        const size_t bbase = (size_t)v * tpv;
        const int n = list_n;
        // each warp expands 32 records into their (record, tile) pairs, 32
        // pairs at a time, so that the per-record tile loops do not diverge
        // the record rows of the next 32 are loaded while these are expanded
        uint32_t nrec = 0;
        float4 nra = make_float4(0.f, 0.f, -1.f, -1.f);
        uint32_t nzb = 0;
        if (warp * 32 + lane < n) {
            nrec = list[warp * 32 + lane];
            nra = w.rec[3 * (size_t)nrec];
            nzb = __float_as_uint(w.rec[3 * (size_t)nrec + 2].w);
        }
        for (int i0 = warp * 32; i0 < n; i0 += nwarps * 32) {
            const int i = i0 + lane;
            uint32_t rec = 0, zb = 0, tx0 = 0, ty0 = 0, ntx = 0, cnt = 0;
            const float4 ra = nra;
            if (i < n) {
                rec = nrec;
                zb = nzb;
            }
            if (i + nwarps * 32 < n) {
                nrec = list[i + nwarps * 32];
                nra = w.rec[3 * (size_t)nrec];
                nzb = __float_as_uint(w.rec[3 * (size_t)nrec + 2].w);
            }
            if (i < n) {
                // the tiles of the record's pixel window, from the same FP32 values
                // the preprocess counted them with
                int x0, x1, y0, y1;
                if (pixel_range(ra.x, ra.z, cam.cx, W, x0, x1) && pixel_range(ra.y, ra.w, cam.cy, H, y0, y1)) {
                    tx0 = x0 / tw;
                    ty0 = y0 / th;
                    ntx = x1 / tw - tx0 + 1;
                    cnt = ntx * (y1 / th - ty0 + 1);
                }
            }
            uint32_t incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
            for (uint32_t t0 = 0; t0 < total; t0 += 32) {
                const uint32_t t = t0 + lane;
                // owner: the first lane whose inclusive count exceeds t
                int lo = 0;
#pragma unroll
                for (int step = 16; step > 0; step >>= 1) {
                    const uint32_t pv = __shfl_sync(0xffffffffu, incl, lo + step - 1);
                    if (pv <= t) lo += step;
                }
                const uint32_t o_incl = __shfl_sync(0xffffffffu, incl, lo);
                const uint32_t o_cnt = __shfl_sync(0xffffffffu, cnt, lo);
                const uint32_t o_rec = __shfl_sync(0xffffffffu, rec, lo);
                const uint32_t o_zb = __shfl_sync(0xffffffffu, zb, lo);
                const uint32_t o_tx0 = __shfl_sync(0xffffffffu, tx0, lo);
                const uint32_t o_ty0 = __shfl_sync(0xffffffffu, ty0, lo);
                const uint32_t o_ntx = __shfl_sync(0xffffffffu, ntx, lo);
                if (t < total) {
                    const uint32_t jj = t - (o_incl - o_cnt);
                    const uint32_t ty = o_ty0 + jj / o_ntx, tx = o_tx0 + jj % o_ntx;
                    const int tl = (int)(ty * tx_n + tx);
                    uint32_t slot;
                    if (c.hist) {
                        slot = atomicAdd(bk + tl, 1u);
                    } else {
                        const size_t bin = bbase + tl;
                        slot = w.bin_start[bin] + w.bin_count[bin] + atomicAdd(w.bin_cursor + bin, 1u);
                    }
                    if (!overflow || (slot < w.bin_start[bbase + tl + 1] && (uint64_t)slot < cap))
                        w.keys[slot] = ((unsigned long long)o_zb << 32) | o_rec;
                }
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// blend
// ---------------------------------------------------------------------------
struct OutPtrs {
    float *rgb, *depth, *T;
    int32_t *ncontrib;
};

// Blends one (view, tile) bin.  Each thread owns PX x PY neighbouring pixels,
// so every Gaussian fetched from shared memory serves several pixels.  Batches
// of B records are gathered into shared memory with cp.async, double-buffered:
// batch b+1 is in flight while batch b is blended (keys of batch b+2 are
// prefetched into registers).
constexpr int kMaxPer = 4; // records per thread and batch (B <= 4 x threads)
constexpr int kUnroll = 8; // Gaussians evaluated together in the blend loop

// COUNT (GS_FLAG_COUNT_EVALS): also count per pixel the covered Gaussians
// examined (the evaluations) and those up to the last blended one.
template <int PX, int PY, bool COUNT>
__device__ __forceinline__ void blend_tile(const Ws &w, const gs_camera *cams, const OutPtrs &o, int bin, int heavy,
                                          float4 *sm)
{
    constexpr int NP = PX * PY;
    const Table *tb = w.tb;
    const int v = bin / tb->tiles_per_view;
    const int t = bin - v * tb->tiles_per_view;
    const int tyi = t / tb->tiles_x, txi = t - tyi * tb->tiles_x;
    const int tcols = tb->tile_w / PX;
    const int i0 = txi * tb->tile_w + (threadIdx.x % tcols) * PX, j0 = tyi * tb->tile_h + (threadIdx.x / tcols) * PY;
    const int W = tb->W, H = tb->H;
    const gs_camera &cam = cams[v];
    float pxc[PX], pyc[PY];
#pragma unroll
    for (int a = 0; a < PX; ++a) pxc[a] = pix_c(i0 + a, cam.cx);
#pragma unroll
    for (int b = 0; b < PY; ++b) pyc[b] = pix_c(j0 + b, cam.cy);
    const float2 npx2 = make_float2(-pxc[0], -pxc[PX - 1]);
    uint32_t start, n;
    bin_range(w, bin, start, n);
    unsigned long long *keys = w.keys + start;
    const int B = tb->batch_depth;
    const int nthr = blockDim.x;
    const uint32_t R = (uint32_t)tb->n_records;
    const int nb = (int)((n + B - 1) / B);
    // one bit per entry of the current 32-entry window, set where some pixel of
    // this thread blended its Gaussian (appended from the right: the window's
    // first entry ends highest); OR-ed over the warp and flagged in the key (bit
    // 31 of the record word) so that the backward walks the blended pairs only
    uint32_t mk = 0;
    const int lane = threadIdx.x & 31;
    auto flag_window = [&](uint32_t base, int n_app) { // n_app in 1..32 entries appended
        const uint32_t wm = __brev(__reduce_or_sync(0xffffffffu, mk << (32 - n_app)));
        mk = 0;
        if ((wm >> lane) & 1u) atomicOr(reinterpret_cast<unsigned int *>(keys + base + lane), kKeyBlended);
    };
    unsigned long long kr[kMaxPer];
    auto load_keys = [&](int b) {
#pragma unroll
        for (int q = 0; q < kMaxPer; ++q) {
            const int e = threadIdx.x + q * nthr;
            const uint32_t idx = (uint32_t)b * B + e;
            kr[q] = (b < nb && e < B && idx < n) ? keys[idx] : 0ull;
        }
    };
    auto issue = [&](int b) {
        float4 *buf = sm + (b & 1) * 3 * B;
#pragma unroll
        for (int q = 0; q < kMaxPer; ++q) {
            const int e = threadIdx.x + q * nthr;
            const uint32_t idx = (uint32_t)b * B + e;
            if (e < B && idx < n) {
                uint32_t rec = (uint32_t)kr[q] & kKeyRecord;
                if (rec >= R) rec = 0; // only after a capacity overflow
                const float4 *src = w.rec + 3 * (size_t)rec;
                cp_async16(buf + e, src);
                cp_async16(buf + B + e, src + 1);
                cp_async16(buf + 2 * B + e, src + 2);
            }
        }
    };
    float T[NP], C0[NP], C1[NP], C2[NP], D[NP];
    int32_t ncov[NP], ncovl[NP], ncon[NP]; // ncov, ncovl: only with COUNT
    uint32_t last[NP];
    bool dn[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        T[p] = 1.0f; C0[p] = C1[p] = C2[p] = D[p] = 0.0f;
        ncov[p] = ncovl[p] = ncon[p] = 0;
        last[p] = 0;
        dn[p] = !(i0 + p % PX < W && j0 + p / PX < H);
    }
    bool tdone = true;
#pragma unroll
    for (int p = 0; p < NP; ++p) tdone = tdone && dn[p];
    if (nb > 0) {
        load_keys(0);
        issue(0);
        cp_async_commit();
        load_keys(1);
    }
    const int tpx = tb->tile_w * tb->tile_h;
    const uint32_t ck_base = heavy >= 0 ? w.heavy_seg[heavy] : 0u;
    for (int b = 0; b < nb; ++b) {
        if (heavy >= 0 && b > 0 && ((uint32_t)b * B) % kSeg == 0) {
            // checkpoint before list position b B, for the backward's segments
            const size_t slot = (size_t)(ck_base + ((uint32_t)b * B) / kSeg - 1) * tpx;
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                const int lpx = ((threadIdx.x / tcols) * PY + p / PX) * tb->tile_w + (threadIdx.x % tcols) * PX + p % PX;
                w.ck_C[slot + lpx] = make_float4(T[p], C0[p], C1[p], C2[p]);
                w.ck_D[slot + lpx] = D[p];
            }
        }
        if (b + 1 < nb) issue(b + 1);
        cp_async_commit();
        if (b + 2 < nb) load_keys(b + 2);
        cp_async_wait<1>();
        if (__syncthreads_count(tdone) == nthr) break;
        const float4 *s0 = sm + (b & 1) * 3 * B, *s1 = s0 + B, *s2 = s0 + 2 * B;
        const int cnt = (int)min((uint32_t)B, n - (uint32_t)b * B);
        // warp-synchronous: every lane runs the same iterations (predicated),
        // the warp leaves once all its lanes have stopped.  kUnroll Gaussians at a
        // time: their falloff and alpha (independent of T) first, for ILP, then
        // the front-to-back updates in order.
#pragma unroll 1
        for (int k0 = 0; k0 < cnt; k0 += kUnroll) {
            if (__all_sync(0xffffffffu, tdone)) {
                if (k0 & 31) flag_window((uint32_t)b * B + (uint32_t)(k0 & ~31), k0 & 31);
                break;
            }
            uint32_t m4 = 0; // this thread's blended bits of the kUnroll entries
            if (!tdone) {
                float al[kUnroll][NP];
                bool ok[kUnroll][NP], cv[kUnroll][NP];
#pragma unroll
                for (int u = 0; u < kUnroll; ++u) {
                    const float4 a = s0[k0 + u]; // < B + kUnroll: inside the buffers and their padding
                    const float4 q = s1[k0 + u];
                    if constexpr (PX == 2) {
                        // the two pixels of a row as packed FP32 pairs
#pragma unroll
                        for (int b = 0; b < PY; ++b) {
                            const float dy = __fsub_rn(a.y, pyc[b]);
                            const float2 dx2 = __fadd2_rn(make_float2(a.x, a.x), npx2); // = a.x - pxc
                            const float2 pw = gauss_power2(q.x, q.y, q.z, dx2, dy);
                            const float2 ar = __fmul2_rn(make_float2(q.w, q.w), make_float2(__expf(pw.x), __expf(pw.y)));
                            const float dxs[2] = {dx2.x, dx2.y}, pws[2] = {pw.x, pw.y}, ars[2] = {ar.x, ar.y};
#pragma unroll
                            for (int h = 0; h < 2; ++h) {
                                const int p = 2 * b + h;
                                cv[u][p] = (k0 + u < cnt) && fabsf(dxs[h]) <= a.z && fabsf(dy) <= a.w;
                                al[u][p] = fminf(kAlphaMax, ars[h]);
                                ok[u][p] = cv[u][p] && pws[h] <= 0.0f && al[u][p] >= kAlphaMin;
                            }
                        }
                    } else {
#pragma unroll
                        for (int p = 0; p < NP; ++p) {
                            const float dx = __fsub_rn(a.x, pxc[p % PX]), dy = __fsub_rn(a.y, pyc[p / PX]);
                            cv[u][p] = (k0 + u < cnt) && fabsf(dx) <= a.z && fabsf(dy) <= a.w;
                            const float power = gauss_power(q.x, q.y, q.z, dx, dy);
                            al[u][p] = fminf(kAlphaMax, raw_alpha(q.w, power));
                            ok[u][p] = cv[u][p] && power <= 0.0f && al[u][p] >= kAlphaMin;
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < kUnroll; ++u) {
                    const float4 c = s2[k0 + u];
                    const float z = c.w;
                    bool blu = false;
                    if constexpr (PX == 2) {
                        // the two pixels of a row updated as packed pairs, branch-free: a
                        // pixel that does not blend this Gaussian gets weight 0 (C + c 0 = C,
                        // T (1 - 0) = T exactly), so the arithmetic is the scalar path's
                        const uint32_t pos = (uint32_t)b * B + k0 + u + 1;
#pragma unroll
                        for (int r = 0; r < PY; ++r) {
                            const int p0 = 2 * r, p1 = 2 * r + 1;
                            const bool a0 = !dn[p0] && cv[u][p0], a1 = !dn[p1] && cv[u][p1];
                            if constexpr (COUNT) {
                                ncov[p0] += a0;
                                ncov[p1] += a1;
                            }
                            const bool k0k = a0 && ok[u][p0], k1k = a1 && ok[u][p1];
                            const float2 T2 = make_float2(T[p0], T[p1]);
                            const float2 om = __fadd2_rn(make_float2(1.0f, 1.0f), make_float2(-al[u][p0], -al[u][p1]));
                            const float2 Tn = __fmul2_rn(T2, om);
                            const bool s0b = k0k && Tn.x < kTStop, s1b = k1k && Tn.y < kTStop;
                            const bool bl0 = k0k && !s0b, bl1 = k1k && !s1b;
                            blu = blu || bl0 || bl1;
                            dn[p0] = dn[p0] || s0b;
                            dn[p1] = dn[p1] || s1b;
                            const float2 wgt =
                                __fmul2_rn(make_float2(bl0 ? al[u][p0] : 0.0f, bl1 ? al[u][p1] : 0.0f), T2);
                            const float2 c0 = __ffma2_rn(make_float2(c.x, c.x), wgt, make_float2(C0[p0], C0[p1]));
                            const float2 c1 = __ffma2_rn(make_float2(c.y, c.y), wgt, make_float2(C1[p0], C1[p1]));
                            const float2 c2 = __ffma2_rn(make_float2(c.z, c.z), wgt, make_float2(C2[p0], C2[p1]));
                            const float2 dd = __ffma2_rn(make_float2(z, z), wgt, make_float2(D[p0], D[p1]));
                            C0[p0] = c0.x; C0[p1] = c0.y;
                            C1[p0] = c1.x; C1[p1] = c1.y;
                            C2[p0] = c2.x; C2[p1] = c2.y;
                            D[p0] = dd.x; D[p1] = dd.y;
                            T[p0] = bl0 ? Tn.x : T[p0];
                            T[p1] = bl1 ? Tn.y : T[p1];
                            ncon[p0] += bl0;
                            ncon[p1] += bl1;
                            if constexpr (COUNT) {
                                ncovl[p0] = bl0 ? ncov[p0] : ncovl[p0];
                                ncovl[p1] = bl1 ? ncov[p1] : ncovl[p1];
                            }
                            last[p0] = bl0 ? pos : last[p0];
                            last[p1] = bl1 ? pos : last[p1];
                        }
                    } else {
#pragma unroll
                        for (int p = 0; p < NP; ++p) {
                            if (!dn[p] && cv[u][p]) {
                                if constexpr (COUNT) ++ncov[p];
                                if (ok[u][p]) {
                                    // explicit roundings: the packed pair path above does the same
                                    const float alpha = al[u][p];
                                    const float Tn = __fmul_rn(T[p], __fsub_rn(1.0f, alpha));
                                    if (Tn < kTStop) {
                                        dn[p] = true;
                                    } else {
                                        const float wgt = __fmul_rn(alpha, T[p]);
                                        C0[p] = __fmaf_rn(c.x, wgt, C0[p]);
                                        C1[p] = __fmaf_rn(c.y, wgt, C1[p]);
                                        C2[p] = __fmaf_rn(c.z, wgt, C2[p]);
                                        D[p] = __fmaf_rn(z, wgt, D[p]);
                                        T[p] = Tn;
                                        ++ncon[p];
                                        if constexpr (COUNT) ncovl[p] = ncov[p];
                                        last[p] = (uint32_t)b * B + k0 + u + 1;
                                        blu = true;
                                    }
                                }
                            }
                        }
                    }
                    m4 = (m4 << 1) | (uint32_t)blu;
                }
                tdone = true;
#pragma unroll
                for (int p = 0; p < NP; ++p) tdone = tdone && dn[p];
            }
            mk = (mk << kUnroll) | m4;
            if (((k0 + kUnroll) & 31) == 0 || k0 + kUnroll >= cnt)
                flag_window((uint32_t)b * B + (uint32_t)(k0 & ~31), (k0 & 31) + kUnroll);
            __syncwarp();
        }
        __syncthreads();
    }
    cp_async_wait<0>();
    if constexpr (COUNT) {
        unsigned long long ev = 0, el = 0;
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            ev += (uint32_t)ncov[p];
            el += (uint32_t)ncovl[p];
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            ev += __shfl_xor_sync(0xffffffffu, ev, off);
            el += __shfl_xor_sync(0xffffffffu, el, off);
        }
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(&w.hdr->n_evals, ev);
            atomicAdd(&w.hdr->n_cov, el);
        }
    }
    const size_t HW = (size_t)W * H;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        const int i = i0 + p % PX, j = j0 + p / PX;
        if (i < W && j < H) {
            const size_t px = (size_t)j * W + i;
            o.rgb[(3 * (size_t)v + 0) * HW + px] = C0[p] + T[p] * tb->bg[0];
            o.rgb[(3 * (size_t)v + 1) * HW + px] = C1[p] + T[p] * tb->bg[1];
            o.rgb[(3 * (size_t)v + 2) * HW + px] = C2[p] + T[p] * tb->bg[2];
            float dd = D[p];
            if (tb->flags & GS_FLAG_NORMALIZE_DEPTH) dd = (1.0f - T[p]) < 1e-4f ? 0.0f : D[p] / (1.0f - T[p]);
            o.depth[(size_t)v * HW + px] = dd;
            o.T[(size_t)v * HW + px] = T[p];
            o.ncontrib[(size_t)v * HW + px] = ncon[p];
            w.pix_T[(size_t)v * HW + px] = T[p];
            w.pix_last[(size_t)v * HW + px] = last[p];
            w.pix_C[(size_t)v * HW + px] = make_float4(C0[p] + T[p] * tb->bg[0], C1[p] + T[p] * tb->bg[1],
                                                       C2[p] + T[p] * tb->bg[2], D[p]);
        }
    }
}

// ---------------------------------------------------------------------------
// blend at 2 x 1 pixels per lane, with a Gaussian list per 4 x 4 quarter
// ---------------------------------------------------------------------------
// The tile is cut into 8 x 8 blocks, one per warp (tile_w and tile_h are
// multiples of 8), and every block into four 4 x 4 quarters of 8 lanes: lane
// 8q + m owns the pixel pair at (2 (m & 1), m >> 1) of quarter q, whose origin
// in the block is (4 (q & 1), 4 (q >> 1)).  The CTA stages each batch of the
// tile's list in shared memory as before; then every warp lists, for each of
// its quarters and in list order, the batch entries whose pixel window meets
// the quarter, and the four quarters walk their own lists in lockstep -- a
// Gaussian costs a quarter's lanes a step only where it can reach them, and
// each pixel still sees every Gaussian that covers it, in depth order.  Per
// pair, the quarters that blended it are kept (4 bits per warp) for the
// backward, and bit 31 of the key marks a pair some pixel of the tile blended.
// The quarter test carries 0.01 px + 1e-6 |uc| of slack for FP32 rounding.

// Lists, per quarter of this warp's block, the entries [0, cnt) of the staged
// batch whose pixel window [uc - hx, uc + hx] x [vc - hy, vc + hy] meets the
// quarter's pixel centres; returns the four lengths.
__device__ __forceinline__ void build_quarter_lists(const float4 *s0, int cnt, const float (&qx0)[4],
                                                    const float (&qy0)[4], uint8_t *ql, int qs, int (&len)[4])
{
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int q = 0; q < 4; ++q) len[q] = 0;
    for (int e0 = 0; e0 < cnt; e0 += 32) {
        const int e = e0 + lane;
        const float4 a = s0[e < cnt ? e : 0];
        const float sx = 0.01f + 1e-6f * fabsf(a.x), sy = 0.01f + 1e-6f * fabsf(a.y);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            // quarter q covers pixel centres [qx0, qx0 + 3] x [qy0, qy0 + 3]
            const bool hit = e < cnt && a.x - a.z <= qx0[q] + 3.0f + sx && a.x + a.z >= qx0[q] - sx &&
                             a.y - a.w <= qy0[q] + 3.0f + sy && a.y + a.w >= qy0[q] - sy;
            const unsigned bal = __ballot_sync(0xffffffffu, hit);
            if (hit) ql[q * qs + len[q] + __popc(bal & lt)] = (uint8_t)e;
            len[q] += __popc(bal);
        }
    }
    __syncwarp();
}

template <bool COUNT>
__device__ __forceinline__ void blendq_tile(const Ws &w, const gs_camera *cams, const OutPtrs &o, int bin, int heavy,
                                           float4 *sm, uint8_t *qls, uint32_t *wbs)
{
    const Table *tb = w.tb;
    const int v = bin / tb->tiles_per_view;
    const int t = bin - v * tb->tiles_per_view;
    const int tyi = t / tb->tiles_x, txi = t - tyi * tb->tiles_x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    const int q = lane >> 3, m = lane & 7;
    const int wx = tb->tile_w >> 3;
    const int tx0 = txi * tb->tile_w, ty0 = tyi * tb->tile_h;
    const int bx = tx0 + (warp % wx) * 8, by = ty0 + (warp / wx) * 8; // this warp's block
    const int i0 = bx + (q & 1) * 4 + (m & 1) * 2, j0 = by + (q >> 1) * 4 + (m >> 1);
    const int W = tb->W, H = tb->H;
    const gs_camera &cam = cams[v];
    const float pyc = pix_c(j0, cam.cy);
    const float2 npx2 = make_float2(-pix_c(i0, cam.cx), -pix_c(i0 + 1, cam.cx));
    float qx0[4], qy0[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        qx0[k] = pix_c(bx + (k & 1) * 4, cam.cx);
        qy0[k] = pix_c(by + (k >> 1) * 4, cam.cy);
    }
    const int B = tb->batch_depth;
    const int qs = qlist_stride(B);
    uint8_t *ql = qls + warp * 4 * qs;
    uint32_t *wb = wbs + warp * B; // quarters of this warp that blended each batch entry
    uint32_t start, n;
    bin_range(w, bin, start, n);
    unsigned long long *keys = w.keys + start;
    const int nthr = blockDim.x;
    const uint32_t R = (uint32_t)tb->n_records;
    const int nb = (int)((n + B - 1) / B);
    unsigned long long kr[kMaxPer];
    auto load_keys = [&](int b) {
#pragma unroll
        for (int qq = 0; qq < kMaxPer; ++qq) {
            const int e = threadIdx.x + qq * nthr;
            const uint32_t idx = (uint32_t)b * B + e;
            kr[qq] = (b < nb && e < B && idx < n) ? keys[idx] : 0ull;
        }
    };
    auto issue = [&](int b) {
        float4 *buf = sm + (b & 1) * 3 * B;
#pragma unroll
        for (int qq = 0; qq < kMaxPer; ++qq) {
            const int e = threadIdx.x + qq * nthr;
            const uint32_t idx = (uint32_t)b * B + e;
            if (e < B && idx < n) {
                uint32_t rec = (uint32_t)kr[qq] & kKeyRecord;
                if (rec >= R) rec = 0; // only after a capacity overflow
                const float4 *src = w.rec + 3 * (size_t)rec;
                cp_async16(buf + e, src);
                cp_async16(buf + B + e, src + 1);
                cp_async16(buf + 2 * B + e, src + 2);
            }
        }
    };
    float T[2], C0[2], C1[2], C2[2], D[2];
    int32_t ncov[2], ncovl[2], ncon[2]; // ncov, ncovl: only with COUNT
    uint32_t last[2];
    bool dn[2];
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        T[p] = 1.0f; C0[p] = C1[p] = C2[p] = D[p] = 0.0f;
        ncov[p] = ncovl[p] = ncon[p] = 0;
        last[p] = 0;
        dn[p] = !(i0 + p < W && j0 < H);
    }
    bool tdone = dn[0] && dn[1];
    for (int e = lane; e < B; e += 32) wb[e] = 0u;
    if (nb > 0) {
        load_keys(0);
        issue(0);
        cp_async_commit();
        load_keys(1);
    }
    const int tpx = tb->tile_w * tb->tile_h;
    const int lpx = (j0 - ty0) * tb->tile_w + (i0 - tx0); // tile-local index of the first pixel
    const uint32_t ck_base = heavy >= 0 ? w.heavy_seg[heavy] : 0u;
    for (int b = 0; b < nb; ++b) {
        if (heavy >= 0 && b > 0 && ((uint32_t)b * B) % kSeg == 0) {
            // checkpoint before list position b B, for the backward's segments
            const size_t slot = (size_t)(ck_base + ((uint32_t)b * B) / kSeg - 1) * tpx;
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                w.ck_C[slot + lpx + p] = make_float4(T[p], C0[p], C1[p], C2[p]);
                w.ck_D[slot + lpx + p] = D[p];
            }
        }
        if (b + 1 < nb) issue(b + 1);
        cp_async_commit();
        if (b + 2 < nb) load_keys(b + 2);
        cp_async_wait<1>();
        if (__syncthreads_count(tdone) == nthr) break;
        const float4 *s0 = sm + (b & 1) * 3 * B, *s1 = s0 + B, *s2 = s0 + 2 * B;
        const int cnt = (int)min((uint32_t)B, n - (uint32_t)b * B);
        int len[4];
        build_quarter_lists(s0, cnt, qx0, qy0, ql, qs, len);
        const int mylen = q == 0 ? len[0] : q == 1 ? len[1] : q == 2 ? len[2] : len[3];
        const int maxlen = max(max(len[0], len[1]), max(len[2], len[3]));
        const uint8_t *myl = ql + q * qs;
#pragma unroll 1
        for (int k0 = 0; k0 < maxlen; k0 += kUnroll) {
            if (__all_sync(0xffffffffu, tdone || k0 >= mylen)) break;
            // this quarter's next kUnroll entries (past its list's end: entry 0, not covered)
            const uint2 id8 = *reinterpret_cast<const uint2 *>(myl + k0);
            int idx[kUnroll];
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
                const uint32_t word = u < 4 ? id8.x : id8.y;
                idx[u] = k0 + u < mylen ? (int)((word >> (8 * (u & 3))) & 0xffu) : 0;
            }
            uint32_t m8 = 0; // bit u: this lane blended its quarter's entry k0 + u
            if (!tdone && k0 < mylen) {
                float al[kUnroll][2];
                bool ok[kUnroll][2], cv[kUnroll][2];
#pragma unroll
                for (int u = 0; u < kUnroll; ++u) {
                    const float4 a = s0[idx[u]];
                    const float4 qv = s1[idx[u]];
                    const float dy = __fsub_rn(a.y, pyc);
                    const float2 dx2 = __fadd2_rn(make_float2(a.x, a.x), npx2); // = a.x - pxc
                    const float2 pw = gauss_power2(qv.x, qv.y, qv.z, dx2, dy);
                    const float2 ar = __fmul2_rn(make_float2(qv.w, qv.w), make_float2(__expf(pw.x), __expf(pw.y)));
                    const bool inl = k0 + u < mylen && fabsf(dy) <= a.w;
                    cv[u][0] = inl && fabsf(dx2.x) <= a.z;
                    cv[u][1] = inl && fabsf(dx2.y) <= a.z;
                    al[u][0] = fminf(kAlphaMax, ar.x);
                    al[u][1] = fminf(kAlphaMax, ar.y);
                    ok[u][0] = cv[u][0] && pw.x <= 0.0f && al[u][0] >= kAlphaMin;
                    ok[u][1] = cv[u][1] && pw.y <= 0.0f && al[u][1] >= kAlphaMin;
                }
#pragma unroll
                for (int u = 0; u < kUnroll; ++u) {
                    const float4 c = s2[idx[u]];
                    const float z = c.w;
                    // both pixels as packed pairs, branch-free: a pixel that does not
                    // blend this Gaussian gets weight 0 (C + c 0 = C, T (1 - 0) = T)
                    const uint32_t pos = (uint32_t)b * B + idx[u] + 1;
                    const bool a0 = !dn[0] && cv[u][0], a1 = !dn[1] && cv[u][1];
                    if constexpr (COUNT) {
                        ncov[0] += a0;
                        ncov[1] += a1;
                    }
                    const bool k0k = a0 && ok[u][0], k1k = a1 && ok[u][1];
                    const float2 T2 = make_float2(T[0], T[1]);
                    const float2 om = __fadd2_rn(make_float2(1.0f, 1.0f), make_float2(-al[u][0], -al[u][1]));
                    const float2 Tn = __fmul2_rn(T2, om);
                    const bool s0b = k0k && Tn.x < kTStop, s1b = k1k && Tn.y < kTStop;
                    const bool bl0 = k0k && !s0b, bl1 = k1k && !s1b;
                    m8 |= (uint32_t)(bl0 || bl1) << u;
                    dn[0] = dn[0] || s0b;
                    dn[1] = dn[1] || s1b;
                    const float2 wgt = __fmul2_rn(make_float2(bl0 ? al[u][0] : 0.0f, bl1 ? al[u][1] : 0.0f), T2);
                    const float2 c0 = __ffma2_rn(make_float2(c.x, c.x), wgt, make_float2(C0[0], C0[1]));
                    const float2 c1 = __ffma2_rn(make_float2(c.y, c.y), wgt, make_float2(C1[0], C1[1]));
                    const float2 c2 = __ffma2_rn(make_float2(c.z, c.z), wgt, make_float2(C2[0], C2[1]));
                    const float2 dd = __ffma2_rn(make_float2(z, z), wgt, make_float2(D[0], D[1]));
                    C0[0] = c0.x; C0[1] = c0.y;
                    C1[0] = c1.x; C1[1] = c1.y;
                    C2[0] = c2.x; C2[1] = c2.y;
                    D[0] = dd.x; D[1] = dd.y;
                    T[0] = bl0 ? Tn.x : T[0];
                    T[1] = bl1 ? Tn.y : T[1];
                    ncon[0] += bl0;
                    ncon[1] += bl1;
                    if constexpr (COUNT) {
                        ncovl[0] = bl0 ? ncov[0] : ncovl[0];
                        ncovl[1] = bl1 ? ncov[1] : ncovl[1];
                    }
                    last[0] = bl0 ? pos : last[0];
                    last[1] = bl1 ? pos : last[1];
                }
                tdone = dn[0] && dn[1];
            }
            // the quarter's blended entries (OR over its 8 lanes): its first lane records them
            uint32_t qm = m8;
            qm |= __shfl_xor_sync(0xffffffffu, qm, 1);
            qm |= __shfl_xor_sync(0xffffffffu, qm, 2);
            qm |= __shfl_xor_sync(0xffffffffu, qm, 4);
            // lane m of the quarter records entry m (the quarter's 8 lanes hold the same idx[])
            int my_idx = idx[0];
#pragma unroll
            for (int u = 1; u < kUnroll; ++u) my_idx = m == u ? idx[u] : my_idx;
            if ((qm >> m) & 1u) atomicOr(wb + my_idx, 1u << q);
        }
        __syncthreads();
        // per batch entry: the quarters of every warp that blended it, and the
        // key's blended bit when any did (this CTA alone touches the bin)
        uint32_t *pq = w.pq + start + (uint32_t)b * B;
        for (int e = threadIdx.x; e < cnt; e += nthr) {
            uint32_t word = 0;
            for (int ww = 0; ww < nwarps; ++ww) word |= wbs[ww * B + e] << (8 * ww);
            if (word) {
                pq[e] = word;
                reinterpret_cast<uint32_t *>(keys + (uint32_t)b * B + e)[0] |= kKeyBlended;
            }
        }
        __syncthreads();
        for (int e = lane; e < cnt; e += 32) wb[e] = 0u;
    }
    cp_async_wait<0>();
    if constexpr (COUNT) {
        unsigned long long ev = (uint32_t)ncov[0] + (uint32_t)ncov[1], el = (uint32_t)ncovl[0] + (uint32_t)ncovl[1];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            ev += __shfl_xor_sync(0xffffffffu, ev, off);
            el += __shfl_xor_sync(0xffffffffu, el, off);
        }
        if (lane == 0) {
            atomicAdd(&w.hdr->n_evals, ev);
            atomicAdd(&w.hdr->n_cov, el);
        }
    }
    const size_t HW = (size_t)W * H;
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const int i = i0 + p, j = j0;
        if (i < W && j < H) {
            const size_t px = (size_t)j * W + i;
            o.rgb[(3 * (size_t)v + 0) * HW + px] = C0[p] + T[p] * tb->bg[0];
            o.rgb[(3 * (size_t)v + 1) * HW + px] = C1[p] + T[p] * tb->bg[1];
            o.rgb[(3 * (size_t)v + 2) * HW + px] = C2[p] + T[p] * tb->bg[2];
            float dd = D[p];
            if (tb->flags & GS_FLAG_NORMALIZE_DEPTH) dd = (1.0f - T[p]) < 1e-4f ? 0.0f : D[p] / (1.0f - T[p]);
            o.depth[(size_t)v * HW + px] = dd;
            o.T[(size_t)v * HW + px] = T[p];
            o.ncontrib[(size_t)v * HW + px] = ncon[p];
            w.pix_T[(size_t)v * HW + px] = T[p];
            w.pix_last[(size_t)v * HW + px] = last[p];
            w.pix_C[(size_t)v * HW + px] = make_float4(C0[p] + T[p] * tb->bg[0], C1[p] + T[p] * tb->bg[1],
                                                       C2[p] + T[p] * tb->bg[2], D[p]);
        }
    }
}

// The blend loop reads kUnroll slots at a time, up to kUnroll - 1 past a
// batch's end (batch depths need not be multiples of kUnroll): the two batch
// buffers are followed by kUnroll padding slots, and all slots must hold finite
// values (the packed pixel-pair update multiplies them by weight 0), so they
// start at zero (later they hold earlier, valid records).
__device__ __forceinline__ void clear_batch_buffers(float4 *sm, int B)
{
    for (int k = threadIdx.x; k < 2 * 3 * B + kUnroll; k += blockDim.x) sm[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();
}

template <int PX, int PY, bool COUNT>
__device__ __forceinline__ void blend_one(const gs_camera *cams, const Ws &w, const OutPtrs &o)
{
    extern __shared__ float4 smem_f4[];
    clear_batch_buffers(smem_f4, w.tb->batch_depth);
    blend_tile<PX, PY, COUNT>(w, cams, o, blockIdx.x, w.heavy_of[blockIdx.x], smem_f4);
}

template <int PX, int PY, bool COUNT>
__device__ __forceinline__ void blend_persistent(const gs_camera *cams, const Ws &w, const OutPtrs &o)
{
    extern __shared__ float4 smem_f4[];
    __shared__ uint32_t item;
    clear_batch_buffers(smem_f4, w.tb->batch_depth);
    const uint32_t n_items = (uint32_t)w.tb->n_bins + w.hdr->n_heavy;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) item = atomicAdd(&w.hdr->queue, 1u);
        __syncthreads();
        if (item >= n_items) break;
        const int bin = bin_of_item(w, item);
        if (bin >= 0) blend_tile<PX, PY, COUNT>(w, cams, o, bin, item < w.hdr->n_heavy ? (int)item : -1, smem_f4);
    }
}

template <int PX, int PY, bool COUNT>
__global__ void blend_kernel(const gs_camera *__restrict__ cams, Ws w, OutPtrs o, const __grid_constant__ Table tbp)
{
    w.tb = const_cast<Table *>(&tbp); // the table from the constant bank (see the preprocess)
    blend_one<PX, PY, COUNT>(cams, w, o);
}

template <int PX, int PY, bool COUNT>
__global__ void blend_persistent_kernel(const gs_camera *__restrict__ cams, Ws w, OutPtrs o,
                                        const __grid_constant__ Table tbp)
{
    w.tb = const_cast<Table *>(&tbp); // the table from the constant bank (see the preprocess)
    blend_persistent<PX, PY, COUNT>(cams, w, o);
}

// 2 x 1 pixels per lane: the quarter-list kernels.  Shared memory: the two
// batch buffers, then per warp four quarter lists (qlist_stride(B) bytes each)
// and B words of blended-quarter bits.
__device__ __forceinline__ void blendq_smem(float4 *smem, int B, int nwarps, uint8_t *&qls, uint32_t *&wbs)
{
    qls = reinterpret_cast<uint8_t *>(smem + 2 * 3 * B + kUnroll);
    wbs = reinterpret_cast<uint32_t *>(qls + nwarps * 4 * qlist_stride(B));
}

template <bool COUNT>
__global__ void __launch_bounds__(256) blendq_kernel(const gs_camera *__restrict__ cams, Ws w, OutPtrs o,
                                                     const __grid_constant__ Table tbp)
{
    w.tb = const_cast<Table *>(&tbp); // the table from the constant bank (see the preprocess)
    extern __shared__ float4 smem_f4[];
    const int B = w.tb->batch_depth;
    uint8_t *qls;
    uint32_t *wbs;
    blendq_smem(smem_f4, B, blockDim.x >> 5, qls, wbs);
    clear_batch_buffers(smem_f4, B);
    blendq_tile<COUNT>(w, cams, o, blockIdx.x, w.heavy_of[blockIdx.x], smem_f4, qls, wbs);
}

template <bool COUNT>
__global__ void __launch_bounds__(256) blendq_persistent_kernel(const gs_camera *__restrict__ cams, Ws w, OutPtrs o,
                                                                const __grid_constant__ Table tbp)
{
    w.tb = const_cast<Table *>(&tbp); // the table from the constant bank (see the preprocess)
    extern __shared__ float4 smem_f4[];
    __shared__ uint32_t item;
    const int B = w.tb->batch_depth;
    uint8_t *qls;
    uint32_t *wbs;
    blendq_smem(smem_f4, B, blockDim.x >> 5, qls, wbs);
    clear_batch_buffers(smem_f4, B);
    const uint32_t n_items = (uint32_t)w.tb->n_bins + w.hdr->n_heavy;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) item = atomicAdd(&w.hdr->queue, 1u);
        __syncthreads();
        if (item >= n_items) break;
        const int bin = bin_of_item(w, item);
        if (bin >= 0) blendq_tile<COUNT>(w, cams, o, bin, item < w.hdr->n_heavy ? (int)item : -1, smem_f4, qls, wbs);
    }
}

// the kernels of one (PX, PY, COUNT) variant
template <int PX, int PY, bool COUNT> struct BlendKernels {
    static constexpr auto one = blend_kernel<PX, PY, COUNT>;
    static constexpr auto persistent = blend_persistent_kernel<PX, PY, COUNT>;
};
template <bool COUNT> struct BlendKernels<2, 1, COUNT> {
    static constexpr auto one = blendq_kernel<COUNT>;
    static constexpr auto persistent = blendq_persistent_kernel<COUNT>;
};

// ---------------------------------------------------------------------------
// host-side launchers
// ---------------------------------------------------------------------------
void launch_setup(const Table &tb, const Ws &w, cudaStream_t s) { setup_kernel<<<1, 256, 0, s>>>(tb, w); }

// dynamic shared memory of the preprocess: the two queues of every warp, its
// round ring and the chunk's (view, tile) counters
static int pre_smem(int n_ring, int hist_words)
{
    return (kPreThreads / 32) * (kWarpQ * (int)(sizeof(AEntry) + sizeof(QEntry)) + n_ring * kRingF4 * 16) +
           hist_words * 4;
}
constexpr int kPreSmemMax = (kPreThreads / 32) * (kWarpQ * (int)(sizeof(AEntry) + sizeof(QEntry)) + 3 * kRingF4 * 16) +
                            kHistCap * 4;

template <int SHT, bool FUSED>
static void launch_pre_t(unsigned grid, int hist_words, cudaStream_t s, const gs_camera *cams, const GaussIn &gin,
                         const Ws &w, const Table &tb)
{
    int n_ring = 3, nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, preprocess_kernel<SHT, FUSED>, kPreThreads,
                                                      pre_smem(3, hist_words)) != cudaSuccess ||
        nb < 2)
        n_ring = 2;
    preprocess_kernel<SHT, FUSED><<<grid, kPreThreads, pre_smem(n_ring, hist_words), s>>>(cams, gin, w, tb, n_ring);
}

void launch_preprocess(const Table &tb, const gs_gaussians *g, const gs_camera *cams, const Ws &w, int n_chunks,
                       int hist_words, cudaStream_t s, const gs_avatars *av, const float *joint_G)
{
    GaussIn gin{g->means, g->log_scales, g->quats, g->opacity_logits, g->cov3d, g->sh,
                nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 0, 0};
    if (av && joint_G) {
        gin.av_means = av->means; gin.av_log_scales = av->log_scales; gin.av_quats = av->quats;
        gin.av_weights = av->weights; gin.av_G = joint_G; gin.av_ids = av->joint_ids; gin.av_of = av->avatar_of;
        gin.n_avatars = av->n_avatars; gin.n_joints = av->n_joints;
    }
    const unsigned grid = (unsigned)n_chunks;
    if (grid == 0) return;
    const bool fused = gin.av_G != nullptr;
    const int hw = std::min(std::max(hist_words, 0), kHistCap);
    switch (g->sh_dtype * 2 + (fused ? 1 : 0)) {
    case GS_SH_F16 * 2: launch_pre_t<GS_SH_F16, false>(grid, hw, s, cams, gin, w, tb); break;
    case GS_SH_F16 * 2 + 1: launch_pre_t<GS_SH_F16, true>(grid, hw, s, cams, gin, w, tb); break;
    case GS_SH_BF16 * 2: launch_pre_t<GS_SH_BF16, false>(grid, hw, s, cams, gin, w, tb); break;
    case GS_SH_BF16 * 2 + 1: launch_pre_t<GS_SH_BF16, true>(grid, hw, s, cams, gin, w, tb); break;
    case GS_SH_F32 * 2 + 1: launch_pre_t<GS_SH_F32, true>(grid, hw, s, cams, gin, w, tb); break;
    default: launch_pre_t<GS_SH_F32, false>(grid, hw, s, cams, gin, w, tb); break;
    }
}

void launch_scan(const Ws &w, cudaStream_t s) { scan_bins_kernel<<<1, 1024, 0, s>>>(w); }

constexpr int kScatterSmem = kHistCap * 4 + kChunkMax * 4;

void launch_scatter(const gs_camera *cams, const Ws &w, int n_chunks, int hist_words, int chunk, cudaStream_t s)
{
    hist_words = std::min(std::max(hist_words, 0), kHistCap);
    chunk = std::min(std::max(chunk, 1), kChunkMax);
    if (n_chunks) scatter_kernel<<<n_chunks, 256, (hist_words + chunk) * 4, s>>>(cams, w, hist_words);
}

// q_warps: warps of a quarter-list CTA (2 x 1 pixels per lane), else 0
int blend_smem_bytes(int batch_depth, int q_warps)
{
    return (2 * 3 * batch_depth + kUnroll) * (int)sizeof(float4) +
           q_warps * (4 * qlist_stride(batch_depth) + 4 * batch_depth);
}

template <int PX, int PY, bool COUNT>
static void launch_blend_c(const Table &tb, const gs_camera *cams, const Ws &w, const OutPtrs &o, int n_bins,
                           int threads, int batch_depth, bool persistent, int n_sms, cudaStream_t s)
{
    const int smem = blend_smem_bytes(batch_depth, PX == 2 && PY == 1 ? threads / 32 : 0);
    using K = BlendKernels<PX, PY, COUNT>;
    if (persistent) {
        int nb = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, K::persistent, threads, smem);
        int grid = n_sms * (nb > 0 ? nb : 1);
        if (grid > n_bins) grid = n_bins;
        K::persistent<<<grid, threads, smem, s>>>(cams, w, o, tb);
    } else {
        K::one<<<n_bins, threads, smem, s>>>(cams, w, o, tb);
    }
}

template <int PX, int PY>
static void launch_blend_t(const Table &tb, const gs_camera *cams, const Ws &w, const OutPtrs &o, int n_bins,
                           int threads, int batch_depth, bool persistent, bool count, int n_sms, cudaStream_t s)
{
    if (count) launch_blend_c<PX, PY, true>(tb, cams, w, o, n_bins, threads, batch_depth, persistent, n_sms, s);
    else launch_blend_c<PX, PY, false>(tb, cams, w, o, n_bins, threads, batch_depth, persistent, n_sms, s);
}

template <int PX, int PY>
static int blend_limit_t()
{
    const void *ks[] = {reinterpret_cast<const void *>(BlendKernels<PX, PY, false>::one),
                        reinterpret_cast<const void *>(BlendKernels<PX, PY, false>::persistent),
                        reinterpret_cast<const void *>(BlendKernels<PX, PY, true>::one),
                        reinterpret_cast<const void *>(BlendKernels<PX, PY, true>::persistent)};
    int lim = 1 << 30;
    for (const void *k : ks) {
        cudaFuncAttributes a;
        if (cudaFuncGetAttributes(&a, k) != cudaSuccess) return 0;
        lim = a.maxThreadsPerBlock < lim ? a.maxThreadsPerBlock : lim;
    }
    return lim;
}

int blend_thread_limit(int px, int py)
{
    if (px == 2 && py == 2) return blend_limit_t<2, 2>();
    if (px == 2) return blend_limit_t<2, 1>();
    if (py == 2) return blend_limit_t<1, 2>();
    return blend_limit_t<1, 1>();
}

void launch_blend(const Table &tb, const gs_camera *cams, const Ws &w, float *rgb, float *depth, float *T,
                  int32_t *ncontrib, int n_bins, int px, int py, int threads, int batch_depth, bool persistent,
                  bool count, int n_sms, cudaStream_t s)
{
    OutPtrs o{rgb, depth, T, ncontrib};
    if (px == 2 && py == 2) launch_blend_t<2, 2>(tb, cams, w, o, n_bins, threads, batch_depth, persistent, count, n_sms, s);
    else if (px == 2) launch_blend_t<2, 1>(tb, cams, w, o, n_bins, threads, batch_depth, persistent, count, n_sms, s);
    else if (py == 2) launch_blend_t<1, 2>(tb, cams, w, o, n_bins, threads, batch_depth, persistent, count, n_sms, s);
    else launch_blend_t<1, 1>(tb, cams, w, o, n_bins, threads, batch_depth, persistent, count, n_sms, s);
}

cudaError_t configure_forward_kernels()
{
    cudaError_t e = cudaSuccess;
    const void *pre[] = {reinterpret_cast<const void *>(preprocess_kernel<GS_SH_F32, false>),
                         reinterpret_cast<const void *>(preprocess_kernel<GS_SH_F32, true>),
                         reinterpret_cast<const void *>(preprocess_kernel<GS_SH_F16, false>),
                         reinterpret_cast<const void *>(preprocess_kernel<GS_SH_F16, true>),
                         reinterpret_cast<const void *>(preprocess_kernel<GS_SH_BF16, false>),
                         reinterpret_cast<const void *>(preprocess_kernel<GS_SH_BF16, true>)};
    for (const void *k : pre)
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kPreSmemMax);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kScatterSmem);
    return e;
}



} // namespace gs
