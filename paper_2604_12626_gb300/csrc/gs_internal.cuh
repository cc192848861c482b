// gs_internal.cuh -- device-side data layout and the helpers every kernel of
// libgs shares.  Not part of the C ABI.
//
// Workspace layout (all sections 256-byte aligned, sizes from the batch):
//   Header      device counters and the sticky status word
//   Table       the batch structure (env/view offsets), written by setup
//   rec         [R] Record (48 B): (uc, vc, hx, hy) (A, B, C, opacity) (r, g, b, z)
//               R = sum over views of the Gaussians of the view's env; (hx, hy)
//               the half widths of the pixel window (alpha_window), z the FP32
//               depth key
//   vis         [R/32] visibility bitmask of the records
//   bin_count   [B] pairs per (view, tile) bin, B = V * tiles
//   bin_start   [B+1] exclusive scan of bin_count (tile ranges)
//   bin_cursor  [B] scatter cursors
//   big_list    [2 P_cap/4096 + 2] (bin << 32 | chunk) of the bins of > 4096 pairs
//   keys        [P_cap] uint64 (FP32 depth bits << 32 | record index)
//   scratch     [P_cap] uint64, ping-pong buffer of the large-bin merges
//   pix_T       [V*H*W] final transmittance (saved for the backward)
//   pix_last    [V*H*W] 1 + tile-list position of the last blended pair
//   pq          [P_cap] uint32 (2 x 1 pixels per lane only): per sorted pair,
//               byte w holds the 4 x 4 quarters of warp w that blended it
//   d_rec       [R] 16 floats (64 B, one DRAM burst): dL/d(uc, vc), the 2D
//               covariance gradient dL/dSigma2 (xx, xy, yy; xy = half of the
//               off-diagonal entry's derivative), dL/d(opacity, r, g, b, z),
//               the opacity, 1 unused, then at [12] the bits of the colour
//               channels that were clamped at 0 (written by the forward)
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "gs.h"

namespace gs {

constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaMax = 0.99f;
// sorted pair keys: depth bits << 32 | record; the blend sets bit 31 of the
// record word once some pixel of the tile has blended the pair
constexpr uint32_t kKeyBlended = 0x80000000u;
constexpr uint32_t kKeyRecord = 0x7fffffffu;
constexpr float kTStop = 1e-4f;
constexpr float kDilation = 0.3f;
constexpr int kSortChunk = 4096; // keys one CTA sorts; larger bins are merged
// floats per record row of d_rec: dL/d(u, v), dL/dSigma2 (xx, xy, yy),
// dL/d(opacity, r, g, b, z), the opacity, 0, the colour-clamp mask, 0, 0, 0
constexpr int kGradStride = 16;
constexpr int kAccStride = 12;    // floats per record in the backward's shared-memory accumulator
constexpr int kMaxJoints = 64;    // joints of one avatar tree

// Triangle-mesh layer: the mesh, and the view/env structure passed by value.
struct MeshIn {
    const float *verts, *colors;
    const int32_t *tris;
    int64_t n_verts, n_tris;
};
struct MeshTable {
    int32_t n_views, W, H;
    float near_plane;
    float bg[3];
    int32_t view_env[GS_MAX_VIEWS];
    int64_t view_rec_off[GS_MAX_VIEWS + 1]; // (view, triangle) records of view v start here
    int64_t env_off[GS_MAX_ENVS + 1];       // triangles of env e: [env_off[e], env_off[e+1])
};

// A joint tree passed by value: parent and depth of every joint (parent < child).
struct JointTree {
    int32_t n, max_depth;
    int8_t parent[kMaxJoints];
    int8_t depth[kMaxJoints];
};

struct Header {
    int32_t status;     // sticky GS_ERR_* (0 = ok)
    uint32_t n_visible; // visible records
    uint32_t n_pairs;   // total pairs (before capacity clamp)
    uint32_t max_bin;   // largest bin
    uint32_t n_big;     // 4096-key chunks of the bins of more than 4096 pairs
    uint32_t queue;     // persistent blend work counter
    uint32_t queue_bwd; // persistent backward work counter
    uint32_t big_queue; // chunk-sort work counter
    uint32_t n_heavy;   // bins in the heavy-first list
    uint32_t heavy_min; // pair count from which a bin is in that list
    uint32_t n_heavy_items; // backward work items of the heavy bins (one per kSeg-long segment)
    uint32_t max_pass;  // merge passes the largest bin needs
    unsigned long long n_evals; // blend evaluations, counted under GS_FLAG_COUNT_EVALS
    unsigned long long n_cov;   // covered Gaussians up to each pixel's last blended one (same flag)
    uint32_t n_backward;  // gs_render_backward calls since the forward (d_rec is clean while 0)
    uint32_t queue_zero;  // gradient-clearing items taken by the blend backward
    uint32_t small_queue; // bins taken by the warp-per-bin sort
    uint32_t pad[45];
};

struct Table {
    int32_t n_envs, n_views;
    int32_t W, H, tile_w, tile_h, tiles_x, tiles_y, tiles_per_view, n_bins;
    int32_t pix_x, pix_y; // pixels per blend thread
    int32_t batch_depth, flags;
    int32_t chunk, n_chunks; // Gaussians per preprocess / scatter CTA, and how many CTAs
    int64_t n_records, pair_capacity, n_gauss;
    float bg[3];
    float near_plane;
    int64_t env_off[GS_MAX_ENVS + 1];
    int64_t env_cov_begin[GS_MAX_ENVS];
    int64_t env_av_base[GS_MAX_ENVS]; // fused LBS: canonical-avatar row of the env's first avatar Gaussian
    int64_t view_rec_off[GS_MAX_VIEWS + 1];
    int32_t view_env[GS_MAX_VIEWS];
    int32_t env_view_begin[GS_MAX_ENVS + 1];
    int32_t env_views[GS_MAX_VIEWS];
    int32_t chunk_off[GS_MAX_ENVS + 1]; // first chunk of each env (chunks never straddle envs)
};

struct Ws {
    Header *hdr;
    Table *tb;
    float4 *rec;  // 3 float4 per record
    uint32_t *vis;
    uint32_t *bin_count, *bin_start, *bin_cursor, *heavy;
    unsigned long long *big_list;
    uint32_t *bin_fcount; // pairs of chunks counted without shared-memory aggregation
    uint32_t *rel;        // [n_chunks][kHistCap] offset of a chunk's pairs inside each bin
    uint32_t *heavy_seg;  // [kHeavyCap + 1] first backward segment of each heavy bin
    int32_t *heavy_of;    // [n_bins] position in the heavy list, -1 if not heavy
    float4 *pix_C;        // [V*H*W] final (r, g, b, depth), background included
    float4 *ck_C;         // [slots][tile pixels] (T, r, g, b) before each segment boundary
    float *ck_D;          // [slots][tile pixels] depth before each segment boundary
    unsigned long long *keys, *scratch;
    float *pix_T;
    uint32_t *pix_last;
    float *d_rec; // kGradStride floats per record
    uint32_t *pq; // [P_cap] at 2 x 1 pixels per lane: per pair, byte w = the quarters of warp w that blended it
};

// Bytes of one quarter list in shared memory (2 x 1 pixels per lane): batch
// entries as uint8, read 8 at a time.
__host__ __device__ __forceinline__ int qlist_stride(int B) { return (B + 15) & ~15; }

constexpr int kSeg = 2048;       // backward segment of a heavy bin (a multiple of every batch depth)
constexpr int kHeavyMin = 1024;  // pairs from which a bin may be scheduled first
constexpr int kHeavyCap = 4096;  // entries of the heavy-first list
constexpr int kChunkMax = 8192; // Gaussians per preprocess / scatter CTA, at most
constexpr int kChunkMin = 1024;
constexpr int kHistCap = 8192;   // (view, tile) counters a chunk keeps in shared memory

// Chunk size from the Gaussian count alone: about 2048 chunks, 1024..8192.
inline int chunk_of(int64_t n)
{
    int c = kChunkMin;
    while (c < kChunkMax && (int64_t)c * 2048 < n) c *= 2;
    return c;
}

// ---------------------------------------------------------------------------
// Decisions both the forward and the backward take; written with explicit
// round-to-nearest intrinsics so that every kernel gets the same bits.
// ---------------------------------------------------------------------------

// FP32 view depth: fl(fl(fl(R20 d0) + fl(R21 d1)) + fl(R22 d2)), d = fl(mu - C).
__device__ __forceinline__ float depth_key(float mx, float my, float mz, const gs_camera &c)
{
    float d0 = __fsub_rn(mx, c.C[0]);
    float d1 = __fsub_rn(my, c.C[1]);
    float d2 = __fsub_rn(mz, c.C[2]);
    float s = __fadd_rn(__fmul_rn(c.R[6], d0), __fmul_rn(c.R[7], d1));
    return __fadd_rn(s, __fmul_rn(c.R[8], d2));
}

// Pixel coordinate relative to the principal point.
__device__ __forceinline__ float pix_c(int i, float c) { return __fsub_rn((float)i, c); }

// Pixel window test in one axis: |uc - pxc| <= h.  With h = r this is the
// square footprint (pixel covered iff |uc - pxc| <= r and the same in y).
__device__ __forceinline__ bool covers1(float uc, float r, float pxc) { return fabsf(__fsub_rn(uc, pxc)) <= r; }

// Half widths (hx, hy) of the pixel window of a Gaussian: the square footprint
// r, narrowed to where the skip rule (alpha = o e^power < 1/255, Sec. 3.2) can
// still let a pixel blend.  With Q the conic, o e^power >= 1/255 needs
// d^T Q d <= t = 2 ln(255 o), and on that ellipse |dx| <= sqrt(t (Q^-1)_xx),
// (Q^-1)_xx = C / (A C - B^2).  The margins cover the FP32 rounding of the
// blend's power (relative 1e-5 per unit of A C / (A C - B^2)), of the fast exp
// and of the window itself, so every pixel the blend finds with alpha >= 1/255
// lies inside; a pixel outside has alpha < 1/255 and would be skipped anyway,
// so the window changes no output.  Where the square is the tighter bound
// (hx = r exactly) the window test is the footprint test itself.  hx < 0: no
// pixel can blend (o < 1/255).  Nearly degenerate conics keep the square.
__device__ __forceinline__ void alpha_window(float o, float A, float B, float C, float r, float &hx, float &hy)
{
    hx = hy = r;
    const float ac = A * C, dq = ac - B * B;
    const float L = __logf(255.0f * o) + 1e-4f; // fast log: absolute error far below the margin
    if (!(L > 0.0f)) {
        hx = hy = -1.0f;
        return;
    }
    if (!(dq > 1e-3f * ac)) return;
    const float t = 2.0f * L * (1.0f + 1e-5f * (ac / dq)) + 1e-4f;
    hx = fminf(r, sqrtf(t * C / dq) * 1.001f + 0.01f);
    hy = fminf(r, sqrtf(t * A / dq) * 1.001f + 0.01f);
}

// Smallest and largest i in [0, n) covered in one axis; false when none.
__device__ __forceinline__ bool pixel_range(float uc, float r, float c, int n, int &lo, int &hi)
{
    float g = fminf(fmaxf(uc + c - r, -1.0f), (float)n + 1.0f);
    int a = (int)ceilf(g);
    a = a < 0 ? 0 : (a > n ? n : a);
#pragma unroll 1
    for (int k = 0; k < 4 && a > 0 && covers1(uc, r, pix_c(a - 1, c)); ++k) --a;
#pragma unroll 1
    for (int k = 0; k < 4 && a < n && !covers1(uc, r, pix_c(a, c)); ++k) ++a;
    if (a >= n || !covers1(uc, r, pix_c(a, c))) return false;
    float h = fminf(fmaxf(uc + c + r, -1.0f), (float)n + 1.0f);
    int b = (int)floorf(h);
    b = b < a ? a : (b > n - 1 ? n - 1 : b);
#pragma unroll 1
    for (int k = 0; k < 4 && b < n - 1 && covers1(uc, r, pix_c(b + 1, c)); ++k) ++b;
#pragma unroll 1
    for (int k = 0; k < 4 && b > a && !covers1(uc, r, pix_c(b, c)); ++k) --b;
    lo = a;
    hi = b;
    return true;
}

// Gaussian falloff exponent at offset (dx, dy) = centre - pixel.
__device__ __forceinline__ float gauss_power(float A, float B, float C, float dx, float dy)
{
    float q = __fmaf_rn(A, __fmul_rn(dx, dx), __fmul_rn(C, __fmul_rn(dy, dy)));
    return __fmaf_rn(-0.5f, q, -__fmul_rn(B, __fmul_rn(dx, dy)));
}

// gauss_power for two pixels of one row at once, with packed FP32 pairs
// (sm_100+): the same operations in the same order, so each element is
// bit-identical to gauss_power(A, B, C, dx2.{x,y}, dy).
__device__ __forceinline__ float2 gauss_power2(float A, float B, float C, float2 dx2, float dy)
{
    const float cdy = __fmul_rn(C, __fmul_rn(dy, dy));
    const float2 q = __ffma2_rn(make_float2(A, A), __fmul2_rn(dx2, dx2), make_float2(cdy, cdy));
    const float2 nb = __fmul2_rn(make_float2(-B, -B), __fmul2_rn(dx2, make_float2(dy, dy))); // = -(B (dx dy))
    return __ffma2_rn(make_float2(-0.5f, -0.5f), q, nb);
}

// Prefetch into L2 of the lines holding bytes [p, p + n) (n <= 256): a
// scattered row that a later stage reads arrives from L2 instead of HBM.
__device__ __forceinline__ void prefetch_l2(const void *p, int n)
{
    const uintptr_t a = reinterpret_cast<uintptr_t>(p);
    for (uintptr_t l = a & ~(uintptr_t)127; l < a + (uintptr_t)n; l += 128)
        asm volatile("prefetch.global.L2 [%0];\n" ::"l"(l));
}

// SH row of Gaussian g for the storage type (48 coefficients)
template <int SHT> __device__ __forceinline__ const void *sh_row(const void *sh, int64_t g)
{
    return static_cast<const char *>(sh) + g * 48 * (SHT == GS_SH_F32 ? 4 : 2);
}
template <int SHT> __host__ __device__ constexpr int sh_row_bytes() { return 48 * (SHT == GS_SH_F32 ? 4 : 2); }

// cp.async gathers (16 bytes each) into shared memory
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Persistent blend order: heavy bins (sorted by pair count, largest first), then
// every other bin in index order.  Returns -1 for a slot that is skipped.
__device__ __forceinline__ int bin_of_item(const Ws &w, uint32_t item)
{
    const uint32_t nh = w.hdr->n_heavy;
    if (item < nh) return (int)w.heavy[item];
    const uint32_t b = item - nh;
    return w.bin_count[b] + w.bin_fcount[b] >= w.hdr->heavy_min ? -1 : (int)b;
}

// alpha before the clamp; the clamp is min(0.99, .)
__device__ __forceinline__ float raw_alpha(float opacity, float power) { return __fmul_rn(opacity, __expf(power)); }

__device__ __forceinline__ void set_status(Header *h, int32_t code) { atomicCAS(&h->status, 0, code); }

// Pair range [start, start + n) of a bin, clamped to the pair capacity.
__device__ __forceinline__ void bin_range(const Ws &w, int bin, uint32_t &start, uint32_t &n)
{
    const uint64_t cap = (uint64_t)w.tb->pair_capacity;
    uint64_t s = w.bin_start[bin], e = w.bin_start[bin + 1];
    if (e > cap) e = cap;
    if (s > e) s = e;
    start = (uint32_t)s;
    n = (uint32_t)(e - s);
}

// ---------------------------------------------------------------------------
// Projection of one Gaussian into one view (forward and backward share it).
// ---------------------------------------------------------------------------

// Rotation of the normalised quaternion (w, x, y, z), row-major.
__device__ __forceinline__ void quat_rot(float w, float x, float y, float z, float (&R)[9])
{
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z); R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z); R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y); R[7] = 2.f * (y * z + w * x); R[8] = 1.f - 2.f * (x * x + y * y);
}

// M = R(q) diag(exp(s)), the factor of Sigma = M M^T (row-major 3 x 3).
__device__ __forceinline__ void factor_from_sq(float3 ls, float4 q, float (&M)[9])
{
    const float inv = 1.0f / sqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
    float R[9];
    quat_rot(q.x * inv, q.y * inv, q.z * inv, q.w * inv, R);
    const float s0 = expf(ls.x), s1 = expf(ls.y), s2 = expf(ls.z);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        M[3 * r] = R[3 * r] * s0;
        M[3 * r + 1] = R[3 * r + 1] * s1;
        M[3 * r + 2] = R[3 * r + 2] * s2;
    }
}

// Sigma = R(q) diag(exp(2 s)) R(q)^T as (xx, xy, xz, yy, yz, zz).
__device__ __forceinline__ void sigma_from_sq(float3 ls, float4 q, float (&S)[6])
{
    float M[9];
    factor_from_sq(ls, q, M);
    S[0] = M[0] * M[0] + M[1] * M[1] + M[2] * M[2];
    S[1] = M[0] * M[3] + M[1] * M[4] + M[2] * M[5];
    S[2] = M[0] * M[6] + M[1] * M[7] + M[2] * M[8];
    S[3] = M[3] * M[3] + M[4] * M[4] + M[5] * M[5];
    S[4] = M[3] * M[6] + M[4] * M[7] + M[5] * M[8];
    S[5] = M[6] * M[6] + M[7] * M[7] + M[8] * M[8];
}

struct Proj {
    float d0, d1, d2;         // mu - C
    float px, py, pz;         // view space (pz is the FP32 depth key)
    float uc, vc;             // fx px/pz, fy py/pz (pixel offset from the principal point)
    float tx, ty;             // px/pz, py/pz clamped for the Jacobian
    bool clampx, clampy;
    float t[6];               // T = J W (2x3)
    float a, b, c, det;       // dilated 2D covariance, determinant
};

// EWA projection with the lateral clamp at 1.3 x the half field and the
// 0.3 px^2 dilation.  Returns false when the conic is singular.
// View, screen position and T = J W of the EWA projection (everything but
// the 2D covariance).
__device__ __forceinline__ void project_view(float mx, float my, float mz, float zk, const gs_camera &cam, int W, int H,
                                             Proj &p)
{
    p.d0 = __fsub_rn(mx, cam.C[0]);
    p.d1 = __fsub_rn(my, cam.C[1]);
    p.d2 = __fsub_rn(mz, cam.C[2]);
    p.px = cam.R[0] * p.d0 + cam.R[1] * p.d1 + cam.R[2] * p.d2;
    p.py = cam.R[3] * p.d0 + cam.R[4] * p.d1 + cam.R[5] * p.d2;
    p.pz = zk;
    const float izx = p.px / p.pz, izy = p.py / p.pz;
    p.uc = cam.fx * izx;
    p.vc = cam.fy * izy;
    const float limx = 1.3f * (0.5f * (float)W / cam.fx), limy = 1.3f * (0.5f * (float)H / cam.fy);
    p.clampx = izx < -limx || izx > limx;
    p.clampy = izy < -limy || izy > limy;
    p.tx = fminf(limx, fmaxf(-limx, izx));
    p.ty = fminf(limy, fmaxf(-limy, izy));
    const float j00 = cam.fx / p.pz, j02 = -cam.fx * p.tx / p.pz, j11 = cam.fy / p.pz, j12 = -cam.fy * p.ty / p.pz;
    float *t = p.t;
    t[0] = j00 * cam.R[0] + j02 * cam.R[6];
    t[1] = j00 * cam.R[1] + j02 * cam.R[7];
    t[2] = j00 * cam.R[2] + j02 * cam.R[8];
    t[3] = j11 * cam.R[3] + j12 * cam.R[6];
    t[4] = j11 * cam.R[4] + j12 * cam.R[7];
    t[5] = j11 * cam.R[5] + j12 * cam.R[8];
}

// EWA projection of a Gaussian given by its 3D covariance S (xx, xy, xz, yy,
// yz, zz): Sigma2 = T S T^T + 0.3 I, det = a c - b^2.
__device__ __forceinline__ bool project_ewa(float mx, float my, float mz, float zk, const float (&S)[6],
                                            const gs_camera &cam, int W, int H, Proj &p)
{
    project_view(mx, my, mz, zk, cam, W, H, p);
    const float *t = p.t;
    const float u0 = S[0] * t[0] + S[1] * t[1] + S[2] * t[2], u1 = S[1] * t[0] + S[3] * t[1] + S[4] * t[2],
                u2 = S[2] * t[0] + S[4] * t[1] + S[5] * t[2];
    const float w0 = S[0] * t[3] + S[1] * t[4] + S[2] * t[5], w1 = S[1] * t[3] + S[3] * t[4] + S[4] * t[5],
                w2 = S[2] * t[3] + S[4] * t[4] + S[5] * t[5];
    p.a = t[0] * u0 + t[1] * u1 + t[2] * u2 + kDilation;
    p.b = t[0] * w0 + t[1] * w1 + t[2] * w2;
    p.c = t[3] * w0 + t[4] * w1 + t[5] * w2 + kDilation;
    p.det = p.a * p.c - p.b * p.b;
    return p.det > 0.0f;
}

// The same projection from the factor M (S = M M^T) of a scale-rotation
// Gaussian: with G = T M (2 x 3), Sigma2 = G G^T + 0.3 I and det(Sigma2) =
// det(G G^T) + 0.3 tr(G G^T) + 0.09, det(G G^T) the sum of the squared 2 x 2
// minors of G (Cauchy-Binet).  Every term is non-negative, so a thin
// Gaussian's nearly singular G G^T costs no cancellation: its conic keeps FP32
// accuracy where a c - b^2 loses digits in proportion to a c / det.
__device__ __forceinline__ bool project_ewa_factor(float mx, float my, float mz, float zk, const float (&M)[9],
                                                   const gs_camera &cam, int W, int H, Proj &p)
{
    project_view(mx, my, mz, zk, cam, W, H, p);
    const float *t = p.t;
    float G0[3], G1[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        G0[j] = t[0] * M[j] + t[1] * M[3 + j] + t[2] * M[6 + j];
        G1[j] = t[3] * M[j] + t[4] * M[3 + j] + t[5] * M[6 + j];
    }
    const float a1 = G0[0] * G0[0] + G0[1] * G0[1] + G0[2] * G0[2];
    const float c1 = G1[0] * G1[0] + G1[1] * G1[1] + G1[2] * G1[2];
    p.b = G0[0] * G1[0] + G0[1] * G1[1] + G0[2] * G1[2];
    const float m01 = G0[0] * G1[1] - G0[1] * G1[0], m02 = G0[0] * G1[2] - G0[2] * G1[0],
                m12 = G0[1] * G1[2] - G0[2] * G1[1];
    const float dg = m01 * m01 + m02 * m02 + m12 * m12;
    p.a = a1 + kDilation;
    p.c = c1 + kDilation;
    p.det = __fmaf_rn(kDilation, a1 + c1, dg) + kDilation * kDilation;
    return p.det > 0.0f;
}

// 3-sigma radius of the dilated 2D covariance, an integer number of pixels:
// lambda_max = mid + sqrt(((a - c) / 2)^2 + b^2), the discriminant (mid^2 -
// det) as a sum of squares, floored at 0.1.
__device__ __forceinline__ float radius_px(const Proj &p)
{
    const float mid = 0.5f * (p.a + p.c);
    const float hd = 0.5f * (p.a - p.c);
    const float lam = mid + sqrtf(fmaxf(0.1f, hd * hd + p.b * p.b));
    return ceilf(3.0f * sqrtf(lam));
}

// Real SH basis of degree 3 (3DGS ordering and signs) at unit direction (x, y, z).
constexpr float kSH0 = 0.28209479177387814f;
constexpr float kSH1 = 0.48860251190291987f;
constexpr float kSH2a = 1.0925484305920792f, kSH2b = 0.31539156525252005f, kSH2c = 0.54627421529603959f;
constexpr float kSH3a = 0.59004358992664352f, kSH3b = 2.8906114426405538f, kSH3c = 0.45704579946446572f,
                kSH3d = 0.3731763325901154f, kSH3e = 1.4453057213202769f;

__device__ __forceinline__ void sh_basis(float x, float y, float z, float (&Y)[16])
{
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[0] = kSH0;
    Y[1] = -kSH1 * y;
    Y[2] = kSH1 * z;
    Y[3] = -kSH1 * x;
    Y[4] = kSH2a * x * y;
    Y[5] = -kSH2a * y * z;
    Y[6] = kSH2b * (2.0f * zz - xx - yy);
    Y[7] = -kSH2a * x * z;
    Y[8] = kSH2c * (xx - yy);
    Y[9] = -kSH3a * y * (3.0f * xx - yy);
    Y[10] = kSH3b * x * y * z;
    Y[11] = -kSH3c * y * (4.0f * zz - xx - yy);
    Y[12] = kSH3d * z * (2.0f * zz - 3.0f * xx - 3.0f * yy);
    Y[13] = -kSH3c * x * (4.0f * zz - xx - yy);
    Y[14] = kSH3e * z * (xx - yy);
    Y[15] = -kSH3a * x * (xx - 3.0f * yy);
}

// Unit view direction d / |d| (d = mu - C) with every rounding explicit, so
// that the forward and the backward evaluate the colour -- and take its clamp
// decision -- on identical values.  inv receives 1 / |d|.
__device__ __forceinline__ float3 view_dir(float d0, float d1, float d2, float &inv)
{
    const float n2 = __fmaf_rn(d0, d0, __fmaf_rn(d1, d1, __fmul_rn(d2, d2)));
    inv = __fdiv_rn(1.0f, __fsqrt_rn(n2));
    return make_float3(__fmul_rn(d0, inv), __fmul_rn(d1, inv), __fmul_rn(d2, inv));
}


// SH-3 colour at a unit direction: 0.5 + sum_i Y_i k_i per channel, clamped
// below at 0.  The coefficients are streamed in memory order (no 48-value
// array held in registers); each channel is one chain of fused multiply-adds
// in index order, the same sequence wherever it is called.
template <int SHT>
__device__ __forceinline__ float3 sh_colour_basis(const void *sh, int64_t g, const float (&Y)[16])
{
    float acc[3] = {0.5f, 0.5f, 0.5f};
    if (SHT == GS_SH_F32) {
        const float4 *p = reinterpret_cast<const float4 *>(sh) + g * 12;
#pragma unroll
        for (int i = 0; i < 12; ++i) {
            const float4 v = __ldg(p + i);
            const float c[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[(4 * i + j) % 3] = __fmaf_rn(Y[(4 * i + j) / 3], c[j], acc[(4 * i + j) % 3]);
        }
    } else {
        const uint4 *p = reinterpret_cast<const uint4 *>(sh) + g * 6;
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            const uint4 v = __ldg(p + i);
            const uint32_t u[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float lo, hi;
                if (SHT == GS_SH_F16) {
                    const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&u[j]));
                    lo = f.x;
                    hi = f.y;
                } else {
                    lo = __uint_as_float(u[j] << 16);
                    hi = __uint_as_float(u[j] & 0xffff0000u);
                }
                const int e = 8 * i + 2 * j;
                acc[e % 3] = __fmaf_rn(Y[e / 3], lo, acc[e % 3]);
                acc[(e + 1) % 3] = __fmaf_rn(Y[(e + 1) / 3], hi, acc[(e + 1) % 3]);
            }
        }
    }
    return make_float3(fmaxf(acc[0], 0.0f), fmaxf(acc[1], 0.0f), fmaxf(acc[2], 0.0f));
}

template <int SHT>
__device__ __forceinline__ float3 sh_colour(const void *sh, int64_t g, float x, float y, float z)
{
    float Y[16];
    sh_basis(x, y, z, Y);
    return sh_colour_basis<SHT>(sh, g, Y);
}

// joint ids >= n_joints (a caller error) are clamped so that reads stay in bounds
__device__ __forceinline__ ushort4 clamp_ids(ushort4 id, int nj)
{
    const unsigned short m = (unsigned short)(nj - 1);
    return make_ushort4(min(id.x, m), min(id.y, m), min(id.z, m), min(id.w, m));
}

__device__ __forceinline__ int clamp_avatar(int a, int na) { return a < 0 ? 0 : (a >= na ? na - 1 : a); }

__device__ __forceinline__ void blend_matrix(const float *Gs, const ushort4 id, const float4 wt, float (&A)[12])
{
    const float *g0 = Gs + 12 * id.x, *g1 = Gs + 12 * id.y, *g2 = Gs + 12 * id.z, *g3 = Gs + 12 * id.w;
    if ((reinterpret_cast<uintptr_t>(Gs) & 15u) == 0) {
        // 16-byte rows: three vector loads per joint instead of twelve (the
        // joints of a warp's lanes differ, so shared-memory wavefronts count)
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const float4 a0 = reinterpret_cast<const float4 *>(g0)[r], a1 = reinterpret_cast<const float4 *>(g1)[r],
                         a2 = reinterpret_cast<const float4 *>(g2)[r], a3 = reinterpret_cast<const float4 *>(g3)[r];
            A[4 * r + 0] = __fmaf_rn(wt.w, a3.x, __fmaf_rn(wt.z, a2.x, __fmaf_rn(wt.y, a1.x, __fmul_rn(wt.x, a0.x))));
            A[4 * r + 1] = __fmaf_rn(wt.w, a3.y, __fmaf_rn(wt.z, a2.y, __fmaf_rn(wt.y, a1.y, __fmul_rn(wt.x, a0.y))));
            A[4 * r + 2] = __fmaf_rn(wt.w, a3.z, __fmaf_rn(wt.z, a2.z, __fmaf_rn(wt.y, a1.z, __fmul_rn(wt.x, a0.z))));
            A[4 * r + 3] = __fmaf_rn(wt.w, a3.w, __fmaf_rn(wt.z, a2.w, __fmaf_rn(wt.y, a1.w, __fmul_rn(wt.x, a0.w))));
        }
        return;
    }
#pragma unroll
    for (int e = 0; e < 12; ++e)
        A[e] = __fmaf_rn(wt.w, g3[e], __fmaf_rn(wt.z, g2[e], __fmaf_rn(wt.y, g1[e], __fmul_rn(wt.x, g0[e]))));
}

// LBS of one canonical Gaussian (Sec. 3.3): A = sum_k w_k G[j_k] (3x4),
// mean' = A3 mean + a, cov' = A3 Sigma A3^T (upper triangle xx, xy, xz, yy,
// yz, zz), every rounding explicit so that the deform kernel and the fused
// preprocess produce identical bits.
__device__ __forceinline__ void lbs_gaussian(const float *Gs, ushort4 id, float4 wt, float3 m, float3 ls, float4 q,
                                             float (&mu)[3], float (&cov)[6])
{
    float A[12];
    blend_matrix(Gs, id, wt, A);
    float S[6];
    sigma_from_sq(ls, q, S);
    const float Sf[9] = {S[0], S[1], S[2], S[1], S[3], S[4], S[2], S[4], S[5]};
    float AS[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            AS[3 * r + c] = __fmaf_rn(A[4 * r + 2], Sf[6 + c], __fmaf_rn(A[4 * r + 1], Sf[3 + c], __fmul_rn(A[4 * r], Sf[c])));
#pragma unroll
    for (int r = 0; r < 3; ++r)
        mu[r] = __fmaf_rn(A[4 * r + 2], m.z, __fmaf_rn(A[4 * r + 1], m.y, __fmaf_rn(A[4 * r], m.x, A[4 * r + 3])));
    const int ri[6] = {0, 0, 0, 1, 1, 2}, ci[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const int r = ri[k], c = ci[k];
        cov[k] = __fmaf_rn(AS[3 * r + 2], A[4 * c + 2], __fmaf_rn(AS[3 * r + 1], A[4 * c + 1], __fmul_rn(AS[3 * r], A[4 * c])));
    }
}

} // namespace gs
