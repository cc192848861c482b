// gs_backward.cu -- adjoint kernels of libgs (sm_103a).
//
// blend_backward   persistent CTAs over (view, tile) bins -- heavy bins split
//                  into 2048-pair segments that start from the forward's
//                  checkpoints.  Each pixel walks the pairs back to front from
//                  the last one it blended, rebuilding the transmittance by
//                  division (T_i = T_{i+1} / (1 - alpha_i)), so only T_final and
//                  the last index per pixel were saved; only the pairs the
//                  forward flagged as blended are walked.  The per-pair
//                  gradients of (uc, vc, 2D covariance, opacity, colour, z) --
//                  the covariance one summed as (Q d)(Q d)^T / 2 per pixel, Q
//                  the conic and d the offset, so no conic-to-covariance
//                  conversion follows the sum -- are reduced
//                  by shuffle transposes (across the warp; or per 4 x 4
//                  quarter of the tile, over its 8 or 4 lanes, where the
//                  forward kept per-quarter lists at 2 x 1 pixels per
//                  thread), then across the CTA in shared memory, and flushed
//                  with float4 atomics per (tile, record) into the record's
//                  gradient row.  In overwrite
//                  mode the same kernel clears the dense parameter gradients
//                  (TMA bulk copies).
// preprocess_backward  env-aligned chunks; the Gaussians some view sees go
//                  through per-warp queues: the chain rule through the
//                  dilation, J W Sigma W^T J^T, the quaternion
//                  normalisation and scales, the SH direction and coefficients,
//                  and the opacity sigmoid.
// Discrete decisions (cull, radius, footprint, skips, stop) are the forward's,
// recomputed bit for bit from the same helpers; the 0.99 clamp and the colour
// clamp at 0 pass zero gradient where active.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "gs_internal.cuh"
#include "gs_launch.h"

namespace gs {


// Sums v[0..31] over the warp with 31 shuffles (butterfly transpose): on
// return, lane l holds the warp total of v[l].
__device__ __forceinline__ float warp_transpose_sum32(float (&v)[32])
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 16, m = 32; o > 0; o >>= 1, m >>= 1) {
        const bool up = lane & o;
#pragma unroll
        for (int i = 0; i < m / 2; ++i) {
            const float keep = up ? v[i + m / 2] : v[i], send = up ? v[i] : v[i + m / 2];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    return v[0];
}

constexpr int kMaxPerB = 4;
constexpr int kGroup = 3; // Gaussians whose gradients share one warp reduction

// One (view, tile) bin, back to front, batches gathered with cp.async and
// double-buffered like the forward.  A thread owns PX x PY pixels and sums
// their contributions before the warp reduction, so there is one reduction per
// (warp, Gaussian) for PX x PY x 32 pixels.
// Segment [seg_lo, seg_hi) of the bin's list (the whole list for light bins).
// A segment that ends before the tile's last blended position starts from the
// forward's checkpoint at seg_hi: T there, and behind it the final colour and
// depth minus what was accumulated in front of seg_hi.
template <int PX, int PY>
__device__ __forceinline__ void blend_backward_tile(const Ws &w, const gs_camera *cams, const float *d_rgb,
                                                   const float *d_depth, int bin, uint32_t seg_lo, uint32_t seg_hi,
                                                   int64_t ck_slot, float4 *sm, float *acc, uint32_t *sidx,
                                                   uint32_t *clist, uint32_t *smax_last)
{
    constexpr int NP = PX * PY;
    const Table *tb = w.tb;
    const int B = tb->batch_depth;
    const int nthr = blockDim.x;
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
    const size_t HW = (size_t)W * H;
    uint32_t start, n;
    bin_range(w, bin, start, n);
    const unsigned long long *keys = w.keys + start;
    const uint32_t R = (uint32_t)tb->n_records;

    float T[NP], dC0[NP], dC1[NP], dC2[NP], dD[NP], S0[NP], S1[NP], S2[NP], SD[NP];
    uint32_t last[NP];
    uint32_t tlast = 0;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        const int i = i0 + p % PX, j = j0 + p / PX;
        T[p] = 1.0f; dC0[p] = dC1[p] = dC2[p] = dD[p] = 0.f; S0[p] = S1[p] = S2[p] = SD[p] = 0.f;
        last[p] = 0;
        if (i < W && j < H) {
            const size_t px = (size_t)j * W + i;
            T[p] = w.pix_T[(size_t)v * HW + px];
            last[p] = w.pix_last[(size_t)v * HW + px];
            dC0[p] = d_rgb[(3 * (size_t)v + 0) * HW + px];
            dC1[p] = d_rgb[(3 * (size_t)v + 1) * HW + px];
            dC2[p] = d_rgb[(3 * (size_t)v + 2) * HW + px];
            dD[p] = d_depth[(size_t)v * HW + px];
            S0[p] = T[p] * tb->bg[0];
            S1[p] = T[p] * tb->bg[1];
            S2[p] = T[p] * tb->bg[2];
        }
        tlast = max(tlast, last[p]);
    }
    if (threadIdx.x == 0) *smax_last = 0;
    __syncthreads();
    const uint32_t wl = __reduce_max_sync(0xffffffffu, tlast);
    if ((threadIdx.x & 31) == 0) atomicMax(smax_last, wl);
    __syncthreads();
    const uint32_t tile_last = min(*smax_last, n);
    if (seg_lo >= tile_last) return; // nothing blended in this segment
    const uint32_t n_proc = min(tile_last, seg_hi);
    if (n_proc < tile_last) {
        // start from the checkpoint before position seg_hi
        const int tpx = tb->tile_w * tb->tile_h;
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            const int i = i0 + p % PX, j = j0 + p / PX;
            if (i < W && j < H) {
                const int lpx = ((threadIdx.x / tcols) * PY + p / PX) * tb->tile_w + (threadIdx.x % tcols) * PX + p % PX;
                const float4 ck = w.ck_C[(size_t)ck_slot * tpx + lpx];
                const float ckd = w.ck_D[(size_t)ck_slot * tpx + lpx];
                const float4 fin = w.pix_C[(size_t)v * HW + (size_t)j * W + i];
                T[p] = ck.x;
                S0[p] = fin.x - ck.y;
                S1[p] = fin.y - ck.z;
                S2[p] = fin.z - ck.w;
                SD[p] = fin.w - ckd;
            }
        }
    }
    // PX == 2: the two pixels of a row as packed FP32 pairs.  The colour and
    // depth terms of dL/dalpha enter through one running dot product per
    // pixel, ndcs = -(dC . S), S the colour and depth accumulated behind the
    // current pair: S grows by c wgt, so ndcs falls by wgt (dC . c).
    float2 T2[PY], ndcs[PY], dc0[PY], dc1[PY], dc2[PY], dd[PY];
    if constexpr (PX == 2) {
#pragma unroll
        for (int b = 0; b < PY; ++b) {
            T2[b] = make_float2(T[2 * b], T[2 * b + 1]);
            dc0[b] = make_float2(dC0[2 * b], dC0[2 * b + 1]);
            dc1[b] = make_float2(dC1[2 * b], dC1[2 * b + 1]);
            dc2[b] = make_float2(dC2[2 * b], dC2[2 * b + 1]);
            dd[b] = make_float2(dD[2 * b], dD[2 * b + 1]);
            float x[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int q = 2 * b + e;
                x[e] = -(dC0[q] * S0[q] + dC1[q] * S1[q] + dC2[q] * S2[q] + dD[q] * SD[q]);
            }
            ndcs[b] = make_float2(x[0], x[1]);
        }
    }
    const int lane = threadIdx.x & 31;
    const int nb = (int)((n_proc - seg_lo + B - 1) / B);
    // batch b covers [lo_b, hi_b), hi_b = n_proc - b B, lo_b >= seg_lo
    auto lo_of = [&](int b) {
        const int32_t x = (int32_t)n_proc - (b + 1) * B;
        return x < (int32_t)seg_lo ? (int32_t)seg_lo : x;
    };
    auto hi_of = [&](int b) { return (int32_t)n_proc - b * B; };
    unsigned long long kr[kMaxPerB];
    auto load_keys = [&](int b) {
        const int32_t lo = lo_of(b), cnt = hi_of(b) - lo;
#pragma unroll
        for (int q = 0; q < kMaxPerB; ++q) {
            const int e = threadIdx.x + q * nthr;
            kr[q] = (b < nb && e < cnt) ? keys[lo + e] : 0ull;
        }
    };
    auto issue = [&](int b) {
        float4 *buf = sm + (b & 1) * 3 * B;
        uint32_t *ib = sidx + (b & 1) * B;
        const int32_t cnt = hi_of(b) - lo_of(b);
#pragma unroll
        for (int q = 0; q < kMaxPerB; ++q) {
            const int e = threadIdx.x + q * nthr;
            if (e < cnt) {
                const uint32_t word = (uint32_t)kr[q], fl = word & kKeyBlended;
                uint32_t rec = word & kKeyRecord;
                if (rec >= R) rec = 0; // only after a capacity overflow
                if (fl) { // pairs that no pixel blended are never read
                    const float4 *src = w.rec + 3 * (size_t)rec;
                    cp_async16(buf + e, src);
                    cp_async16(buf + B + e, src + 1);
                    cp_async16(buf + 2 * B + e, src + 2);
                }
                ib[e] = rec | fl;
            }
        }
    };
    if (nb > 0) {
        load_keys(0);
        issue(0);
        cp_async_commit();
        load_keys(1);
    }
    for (int b = 0; b < nb; ++b) {
        if (b + 1 < nb) issue(b + 1);
        cp_async_commit();
        if (b + 2 < nb) load_keys(b + 2);
        const int32_t lo = lo_of(b), cnt = hi_of(b) - lo;
        for (int k = threadIdx.x; k < cnt * kAccStride; k += nthr) acc[k] = 0.0f;
        cp_async_wait<1>();
        __syncthreads();
        const uint32_t *ibc = sidx + (b & 1) * B;
        if (threadIdx.x < 32) { // the batch's blended entries, in list order
            uint32_t base = 0;
            for (int c0 = 0; c0 < cnt; c0 += 32) {
                const int k = c0 + lane;
                const bool f = k < cnt && (ibc[k] & kKeyBlended);
                const unsigned bal = __ballot_sync(0xffffffffu, f);
                if (f) clist[base + __popc(bal & ((1u << lane) - 1u))] = (uint32_t)k;
                base += __popc(bal);
            }
            if (lane == 0) clist[B] = base;
        }
        __syncthreads();
        const int ncl = (int)clist[B];
        const float4 *s0 = sm + (b & 1) * 3 * B, *s1 = s0 + B, *s2 = s0 + 2 * B;
        // groups of kGroup blended Gaussians, back to front: falloff and alpha
        // first (independent of T), then the sequential transmittance rebuild
        // and gradients, then one warp reduction of the group's 10 x kGroup sums
        for (int i1 = ncl - 1; i1 >= 0; i1 -= kGroup) {
            int kk[kGroup]; // entries of the group (-1: past the list's front)
#pragma unroll
            for (int u = 0; u < kGroup; ++u) kk[u] = i1 - u >= 0 ? (int)clist[i1 - u] : -1;
            float g[32];
#pragma unroll
            for (int x = 0; x < 32; ++x) g[x] = 0.f;
            bool contrib = false;
            if (__any_sync(0xffffffffu, i1 < kGroup - 1 || (uint32_t)(lo + kk[kGroup - 1]) < tlast)) {
                float ar[kGroup][NP], ex[kGroup][NP], dxs[kGroup][NP], dys[kGroup][NP];
                bool ok[kGroup][NP];
#pragma unroll
                for (int u = 0; u < kGroup; ++u) {
                    const int k = kk[u], ks = k < 0 ? kk[0] : k;
                    const float4 a = s0[ks];
                    const float4 q = s1[ks];
                    float pw[NP];
                    if constexpr (PX == 2) {
                        // the two pixels of a row as packed FP32 pairs
#pragma unroll
                        for (int b = 0; b < PY; ++b) {
                            const float dy = __fsub_rn(a.y, pyc[b]);
                            const float2 dx2 = __fadd2_rn(make_float2(a.x, a.x), npx2); // = a.x - pxc
                            const float2 p2 = gauss_power2(q.x, q.y, q.z, dx2, dy);
                            dxs[u][2 * b] = dx2.x;
                            dxs[u][2 * b + 1] = dx2.y;
                            dys[u][2 * b] = dys[u][2 * b + 1] = dy;
                            pw[2 * b] = p2.x;
                            pw[2 * b + 1] = p2.y;
                        }
                    } else {
#pragma unroll
                        for (int p = 0; p < NP; ++p) {
                            dxs[u][p] = __fsub_rn(a.x, pxc[p % PX]);
                            dys[u][p] = __fsub_rn(a.y, pyc[p / PX]);
                            pw[p] = gauss_power(q.x, q.y, q.z, dxs[u][p], dys[u][p]);
                        }
                    }
#pragma unroll
                    for (int p = 0; p < NP; ++p) {
                        ex[u][p] = __expf(pw[p]);
                        ar[u][p] = __fmul_rn(q.w, ex[u][p]); // = raw_alpha(q.w, power)
                        ok[u][p] = k >= 0 && (uint32_t)(lo + k) < last[p] && fabsf(dxs[u][p]) <= a.z &&
                                   fabsf(dys[u][p]) <= a.w && pw[p] <= 0.0f &&
                                   fminf(kAlphaMax, ar[u][p]) >= kAlphaMin;
                        if (!ok[u][p]) ex[u][p] = 0.f; // finite where a zero weight multiplies it
                    }
                }
                if constexpr (PX == 2) {
                    // every pixel of the group: a pixel that the pair does not
                    // reach gets alpha = 0 and adds exact zeros
                    float2 G[kGroup][10];
#pragma unroll
                    for (int u = 0; u < kGroup; ++u)
#pragma unroll
                        for (int x = 0; x < 10; ++x) G[u][x] = make_float2(0.f, 0.f);
#pragma unroll
                    for (int u = 0; u < kGroup; ++u) {
                        const int ks = kk[u] < 0 ? kk[0] : kk[u];
                        const float4 q = s1[ks];
                        const float4 c = s2[ks];
                        const float2 cx = make_float2(c.x, c.x), cy = make_float2(c.y, c.y),
                                     cz = make_float2(c.z, c.z), az = make_float2(c.w, c.w);
                        const float2 qx = make_float2(q.x, q.x), qy = make_float2(q.y, q.y);
#pragma unroll
                        for (int b = 0; b < PY; ++b) {
                            const int p0 = 2 * b, p1 = 2 * b + 1;
                            if (!(ok[u][p0] || ok[u][p1])) continue;
                            contrib = true;
                            const float2 nal = make_float2(ok[u][p0] ? -fminf(kAlphaMax, ar[u][p0]) : 0.f,
                                                           ok[u][p1] ? -fminf(kAlphaMax, ar[u][p1]) : 0.f);
                            const float2 om = __fadd2_rn(make_float2(1.f, 1.f), nal);
                            const float2 iom = make_float2(__fdividef(1.0f, om.x), __fdividef(1.0f, om.y));
                            const float2 Ti = __fmul2_rn(T2[b], iom);
                            const float2 nwgt = __fmul2_rn(nal, Ti);
                            G[u][6] = __ffma2_rn(nwgt, dc0[b], G[u][6]);
                            G[u][7] = __ffma2_rn(nwgt, dc1[b], G[u][7]);
                            G[u][8] = __ffma2_rn(nwgt, dc2[b], G[u][8]);
                            G[u][9] = __ffma2_rn(nwgt, dd[b], G[u][9]);
                            const float2 dcc = __ffma2_rn(
                                dd[b], az, __ffma2_rn(dc2[b], cz, __ffma2_rn(dc1[b], cy, __fmul2_rn(dc0[b], cx))));
                            const float2 dal = __ffma2_rn(ndcs[b], iom, __fmul2_rn(dcc, Ti));
                            ndcs[b] = __ffma2_rn(nwgt, dcc, ndcs[b]);
                            T2[b] = Ti;
                            // the 0.99 clamp passes no gradient to opacity and footprint
                            const float2 dalm = make_float2(ar[u][p0] < kAlphaMax ? dal.x : 0.f,
                                                            ar[u][p1] < kAlphaMax ? dal.y : 0.f);
                            const float2 dx = make_float2(dxs[u][p0], dxs[u][p1]);
                            const float dy1 = dys[u][p0];
                            const float2 dy = make_float2(dy1, dy1);
                            G[u][5] = __ffma2_rn(dalm, make_float2(ex[u][p0], ex[u][p1]), G[u][5]);
                            const float2 ngp = __fmul2_rn(dalm, nal); // -dL/dalpha * alpha
                            // w = Q d (Q the conic): dpower/dd = -w and dpower/dSigma2 =
                            // w w^T / 2, so the covariance gradient is summed in that
                            // form directly (no conic-to-covariance conversion, whose
                            // cancellation on thin ellipses would amplify rounding)
                            const float qyd = q.y * dy1, qzd = q.z * dy1;
                            const float2 wx = __ffma2_rn(qx, dx, make_float2(qyd, qyd));
                            const float2 wy = __ffma2_rn(qy, dx, make_float2(qzd, qzd));
                            G[u][0] = __ffma2_rn(ngp, wx, G[u][0]);
                            G[u][1] = __ffma2_rn(ngp, wy, G[u][1]);
                            const float2 nhw = __fmul2_rn(__fmul2_rn(ngp, make_float2(-0.5f, -0.5f)), wx);
                            G[u][2] = __ffma2_rn(nhw, wx, G[u][2]);
                            G[u][3] = __ffma2_rn(nhw, wy, G[u][3]);
                            G[u][4] = __ffma2_rn(__fmul2_rn(__fmul2_rn(ngp, make_float2(-0.5f, -0.5f)), wy), wy,
                                                 G[u][4]);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < kGroup; ++u) {
#pragma unroll
                        for (int x = 0; x < 6; ++x) g[10 * u + x] = G[u][x].x + G[u][x].y;
#pragma unroll
                        for (int x = 6; x < 10; ++x) g[10 * u + x] = -(G[u][x].x + G[u][x].y);
                    }
                } else {
#pragma unroll
                for (int u = 0; u < kGroup; ++u) {
                    const int ks = kk[u] < 0 ? kk[0] : kk[u];
                    const float4 q = s1[ks];
                    const float4 c = s2[ks];
#pragma unroll
                    for (int p = 0; p < NP; ++p) {
                        if (ok[u][p]) {
                            contrib = true;
                            const float alpha = fminf(kAlphaMax, ar[u][p]);
                            const float om = 1.0f - alpha;
                            const float iom = __fdividef(1.0f, om); // om in [0.01, 1): fast reciprocal
                            const float Ti = T[p] * iom;
                            const float wgt = alpha * Ti;
                            float *gu = g + 10 * u;
                            gu[6] += wgt * dC0[p];
                            gu[7] += wgt * dC1[p];
                            gu[8] += wgt * dC2[p];
                            gu[9] += wgt * dD[p];
                            const float dal = dC0[p] * (c.x * Ti - S0[p] * iom) + dC1[p] * (c.y * Ti - S1[p] * iom) +
                                              dC2[p] * (c.z * Ti - S2[p] * iom) + dD[p] * (c.w * Ti - SD[p] * iom);
                            S0[p] += c.x * wgt;
                            S1[p] += c.y * wgt;
                            S2[p] += c.z * wgt;
                            SD[p] += c.w * wgt;
                            T[p] = Ti;
                            if (ar[u][p] < kAlphaMax) {
                                const float dx = dxs[u][p], dy = dys[u][p];
                                gu[5] += dal * ex[u][p]; // d alpha / d opacity = exp(power)
                                const float gp = dal * alpha;
                                // w = Q d: dpower/dd = -w, dpower/dSigma2 = w w^T / 2
                                const float wx = q.x * dx + q.y * dy, wy = q.y * dx + q.z * dy;
                                gu[0] += -gp * wx;
                                gu[1] += -gp * wy;
                                const float hg = 0.5f * gp;
                                gu[2] += hg * wx * wx;
                                gu[3] += hg * wx * wy;
                                gu[4] += hg * wy * wy;
                            }
                        }
                    }
                }
                }
            }
            if (__any_sync(0xffffffffu, contrib)) {
                const float tot = warp_transpose_sum32(g);
                const int u = lane / 10, j = lane - 10 * u;
                if (lane < 10 * kGroup && i1 - u >= 0) atomicAdd(acc + clist[i1 - u] * kAccStride + j, tot);
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < ncl; i += nthr) {
            const int k = (int)clist[i];
            const float4 *ak = reinterpret_cast<const float4 *>(acc + k * kAccStride);
            const float4 x0 = ak[0], x1 = ak[1], x2 = ak[2];
            if (x0.x != 0.f || x0.y != 0.f || x0.z != 0.f || x0.w != 0.f || x1.x != 0.f || x1.y != 0.f ||
                x1.z != 0.f || x1.w != 0.f || x2.x != 0.f || x2.y != 0.f) {
                float4 *dst = reinterpret_cast<float4 *>(w.d_rec + (size_t)(ibc[k] & kKeyRecord) * kGradStride);
                atomicAdd(dst + 0, x0);
                atomicAdd(dst + 1, x1);
                atomicAdd(dst + 2, x2);
            }
        }
        __syncthreads();
    }
    cp_async_wait<0>();
}

// Sums v[0..31] over each 8-lane quarter of the warp with 28 shuffles
// (butterfly transpose over lane bits 4, 2, 1): on return, lane 8q + m holds
// in v[0..3] the quarter's totals of v[4m .. 4m + 3].
__device__ __forceinline__ void quarter_transpose_sum32(float (&v)[32])
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 4, m = 32; o > 0; o >>= 1, m >>= 1) {
        const bool up = lane & o;
#pragma unroll
        for (int i = 0; i < m / 2; ++i) {
            const float keep = up ? v[i + m / 2] : v[i], send = up ? v[i] : v[i + m / 2];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
}

// 2 x 1 pixels per lane with a Gaussian list per 4 x 4 quarter (the layout of
// the forward's blendq_tile): per batch, back to front, the entries some pixel
// of the tile blended are gathered; every warp lists, per quarter, those its
// quarter blended (the forward's quarter bits), and the quarters walk their own
// lists in lockstep, kGroup entries at a time; the gradient sums of a group are
// reduced per quarter (8 lanes) and added to the batch's shared accumulator.
__device__ __forceinline__ void blendq_backward_tile(const Ws &w, const gs_camera *cams, const float *d_rgb,
                                                    const float *d_depth, int bin, uint32_t seg_lo, uint32_t seg_hi,
                                                    int64_t ck_slot, float4 *sm, float *acc, uint32_t *sidx,
                                                    uint32_t *clist, uint32_t *spq, uint8_t *qls,
                                                    uint32_t *smax_last)
{
    const Table *tb = w.tb;
    const int B = tb->batch_depth;
    const int nthr = blockDim.x;
    const int v = bin / tb->tiles_per_view;
    const int t = bin - v * tb->tiles_per_view;
    const int tyi = t / tb->tiles_x, txi = t - tyi * tb->tiles_x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = lane >> 3, mq = lane & 7;
    const int wx = tb->tile_w >> 3;
    const int tx0 = txi * tb->tile_w, ty0 = tyi * tb->tile_h;
    const int i0 = tx0 + (warp % wx) * 8 + (q & 1) * 4 + (mq & 1) * 2;
    const int j0 = ty0 + (warp / wx) * 8 + (q >> 1) * 4 + (mq >> 1);
    const int W = tb->W, H = tb->H;
    const gs_camera &cam = cams[v];
    const float pyc = pix_c(j0, cam.cy);
    const float2 npx2 = make_float2(-pix_c(i0, cam.cx), -pix_c(i0 + 1, cam.cx));
    const size_t HW = (size_t)W * H;
    uint32_t start, n;
    bin_range(w, bin, start, n);
    const unsigned long long *keys = w.keys + start;
    const uint32_t *pqb = w.pq + start;
    const uint32_t R = (uint32_t)tb->n_records;
    const int qs = qlist_stride(B);
    uint8_t *ql = qls + warp * 4 * qs;

    float T[2], dC0[2], dC1[2], dC2[2], dD[2], S0[2], S1[2], S2[2], SD[2];
    uint32_t last[2];
    uint32_t tlast = 0;
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const int i = i0 + p, j = j0;
        T[p] = 1.0f; dC0[p] = dC1[p] = dC2[p] = dD[p] = 0.f; S0[p] = S1[p] = S2[p] = SD[p] = 0.f;
        last[p] = 0;
        if (i < W && j < H) {
            const size_t px = (size_t)j * W + i;
            T[p] = w.pix_T[(size_t)v * HW + px];
            last[p] = w.pix_last[(size_t)v * HW + px];
            dC0[p] = d_rgb[(3 * (size_t)v + 0) * HW + px];
            dC1[p] = d_rgb[(3 * (size_t)v + 1) * HW + px];
            dC2[p] = d_rgb[(3 * (size_t)v + 2) * HW + px];
            dD[p] = d_depth[(size_t)v * HW + px];
            S0[p] = T[p] * tb->bg[0];
            S1[p] = T[p] * tb->bg[1];
            S2[p] = T[p] * tb->bg[2];
        }
        tlast = max(tlast, last[p]);
    }
    if (threadIdx.x == 0) *smax_last = 0;
    __syncthreads();
    const uint32_t wl = __reduce_max_sync(0xffffffffu, tlast);
    if (lane == 0) atomicMax(smax_last, wl);
    __syncthreads();
    const uint32_t tile_last = min(*smax_last, n);
    if (seg_lo >= tile_last) return; // nothing blended in this segment
    const uint32_t n_proc = min(tile_last, seg_hi);
    if (n_proc < tile_last) {
        // start from the checkpoint before position seg_hi
        const int tpx = tb->tile_w * tb->tile_h;
        const int lpx = (j0 - ty0) * tb->tile_w + (i0 - tx0);
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            const int i = i0 + p, j = j0;
            if (i < W && j < H) {
                const float4 ck = w.ck_C[(size_t)ck_slot * tpx + lpx + p];
                const float ckd = w.ck_D[(size_t)ck_slot * tpx + lpx + p];
                const float4 fin = w.pix_C[(size_t)v * HW + (size_t)j * W + i];
                T[p] = ck.x;
                S0[p] = fin.x - ck.y;
                S1[p] = fin.y - ck.z;
                S2[p] = fin.z - ck.w;
                SD[p] = fin.w - ckd;
            }
        }
    }
    // both pixels as packed FP32 pairs; the colour and depth terms of dL/dalpha
    // enter through one running dot product per pixel, ndcs = -(dC . S), S the
    // colour and depth behind the current pair (S grows by c wgt, so ndcs falls
    // by wgt (dC . c))
    float2 T2 = make_float2(T[0], T[1]);
    const float2 dc0 = make_float2(dC0[0], dC0[1]), dc1 = make_float2(dC1[0], dC1[1]),
                 dc2 = make_float2(dC2[0], dC2[1]), dd = make_float2(dD[0], dD[1]);
    float2 ndcs;
    {
        float x[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) x[e] = -(dC0[e] * S0[e] + dC1[e] * S1[e] + dC2[e] * S2[e] + dD[e] * SD[e]);
        ndcs = make_float2(x[0], x[1]);
    }
    const int nb = (int)((n_proc - seg_lo + B - 1) / B);
    // batch b covers [lo_b, hi_b), hi_b = n_proc - b B, lo_b >= seg_lo
    auto lo_of = [&](int b) {
        const int32_t x = (int32_t)n_proc - (b + 1) * B;
        return x < (int32_t)seg_lo ? (int32_t)seg_lo : x;
    };
    auto hi_of = [&](int b) { return (int32_t)n_proc - b * B; };
    unsigned long long kr[kMaxPerB];
    auto load_keys = [&](int b) {
        const int32_t lo = lo_of(b), cnt = hi_of(b) - lo;
#pragma unroll
        for (int qq = 0; qq < kMaxPerB; ++qq) {
            const int e = threadIdx.x + qq * nthr;
            kr[qq] = (b < nb && e < cnt) ? keys[lo + e] : 0ull;
        }
    };
    auto issue = [&](int b) {
        float4 *buf = sm + (b & 1) * 3 * B;
        uint32_t *ib = sidx + (b & 1) * B;
        uint32_t *pb = spq + (b & 1) * B;
        const int32_t lo = lo_of(b), cnt = hi_of(b) - lo;
#pragma unroll
        for (int qq = 0; qq < kMaxPerB; ++qq) {
            const int e = threadIdx.x + qq * nthr;
            if (e < cnt) {
                const uint32_t word = (uint32_t)kr[qq], fl = word & kKeyBlended;
                uint32_t rec = word & kKeyRecord;
                if (rec >= R) rec = 0; // only after a capacity overflow
                if (fl) { // pairs that no pixel blended are never read
                    const float4 *src = w.rec + 3 * (size_t)rec;
                    cp_async16(buf + e, src);
                    cp_async16(buf + B + e, src + 1);
                    cp_async16(buf + 2 * B + e, src + 2);
                    pb[e] = pqb[lo + e];
                }
                ib[e] = rec | fl;
            }
        }
    };
    if (nb > 0) {
        load_keys(0);
        issue(0);
        cp_async_commit();
        load_keys(1);
    }
    const unsigned lt = (1u << lane) - 1u;
    for (int b = 0; b < nb; ++b) {
        if (b + 1 < nb) issue(b + 1);
        cp_async_commit();
        if (b + 2 < nb) load_keys(b + 2);
        const int32_t lo = lo_of(b), cnt = hi_of(b) - lo;
        for (int k = threadIdx.x; k < cnt * kAccStride; k += nthr) acc[k] = 0.0f;
        cp_async_wait<1>();
        __syncthreads();
        const uint32_t *ibc = sidx + (b & 1) * B;
        const uint32_t *pbc = spq + (b & 1) * B;
        if (threadIdx.x < 32) { // the batch's blended entries, in list order
            uint32_t base = 0;
            for (int c0 = 0; c0 < cnt; c0 += 32) {
                const int k = c0 + lane;
                const bool f = k < cnt && (ibc[k] & kKeyBlended);
                const unsigned bal = __ballot_sync(0xffffffffu, f);
                if (f) clist[base + __popc(bal & lt)] = (uint32_t)k;
                base += __popc(bal);
            }
            if (lane == 0) clist[B] = base;
        }
        __syncthreads();
        const int ncl = (int)clist[B];
        // this warp's quarter lists: the blended entries each quarter blended
        int len[4] = {0, 0, 0, 0};
        for (int c0 = 0; c0 < ncl; c0 += 32) {
            const int i = c0 + lane;
            const uint32_t k = i < ncl ? clist[i] : 0u;
            const uint32_t qb = i < ncl ? (pbc[k] >> (8 * warp)) & 15u : 0u;
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) {
                const bool hit = (qb >> qq) & 1u;
                const unsigned bal = __ballot_sync(0xffffffffu, hit);
                if (hit) ql[qq * qs + len[qq] + __popc(bal & lt)] = (uint8_t)k;
                len[qq] += __popc(bal);
            }
        }
        __syncwarp();
        const int mylen = q == 0 ? len[0] : q == 1 ? len[1] : q == 2 ? len[2] : len[3];
        const int maxlen = max(max(len[0], len[1]), max(len[2], len[3]));
        const uint8_t *myl = ql + q * qs;
        const float4 *s0 = sm + (b & 1) * 3 * B, *s1 = s0 + B, *s2 = s0 + 2 * B;
        // the slot a lane past its list's end reads: a gathered record, so that
        // the branch-free gradient phase multiplies finite values by its zero
        // weights (the slots of pairs no pixel blended hold stale data)
        const int ksafe = ncl > 0 ? (int)clist[0] : 0;
        // groups of kGroup entries per quarter, back to front: falloff and
        // alpha first (independent of T), then the sequential transmittance
        // rebuild and gradients, then one quarter reduction of the group's
        // 10 x kGroup sums
        for (int s = 0; s < maxlen; s += kGroup) {
            int kk[kGroup]; // batch entries of the group (-1: past this quarter's list)
#pragma unroll
            for (int u = 0; u < kGroup; ++u) kk[u] = s + u < mylen ? (int)myl[mylen - 1 - s - u] : -1;
            float g[32];
#pragma unroll
            for (int x = 0; x < 32; ++x) g[x] = 0.f;
            bool contrib = false;
            float ar[kGroup][2], ex[kGroup][2], dxs[kGroup][2], dys[kGroup];
            bool ok[kGroup][2];
#pragma unroll
            for (int u = 0; u < kGroup; ++u) {
                const int k = kk[u], ks = k < 0 ? ksafe : k;
                const float4 a = s0[ks];
                const float4 qv = s1[ks];
                const float dy = __fsub_rn(a.y, pyc);
                const float2 dx2 = __fadd2_rn(make_float2(a.x, a.x), npx2); // = a.x - pxc
                const float2 p2 = gauss_power2(qv.x, qv.y, qv.z, dx2, dy);
                dxs[u][0] = dx2.x;
                dxs[u][1] = dx2.y;
                dys[u] = dy;
                const float pw[2] = {p2.x, p2.y};
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    ex[u][p] = __expf(pw[p]);
                    ar[u][p] = __fmul_rn(qv.w, ex[u][p]); // = raw_alpha(qv.w, power)
                    ok[u][p] = k >= 0 && (uint32_t)(lo + k) < last[p] && fabsf(dxs[u][p]) <= a.z &&
                               fabsf(dy) <= a.w && pw[p] <= 0.0f && fminf(kAlphaMax, ar[u][p]) >= kAlphaMin;
                    if (!ok[u][p]) ex[u][p] = 0.f; // finite where a zero weight multiplies it
                }
            }
            // every pixel of the group: a pixel that the pair does not reach
            // gets alpha = 0 and adds exact zeros
            float2 G[kGroup][10];
#pragma unroll
            for (int u = 0; u < kGroup; ++u)
#pragma unroll
                for (int x = 0; x < 10; ++x) G[u][x] = make_float2(0.f, 0.f);
#pragma unroll
            for (int u = 0; u < kGroup; ++u) {
                const int ks = kk[u] < 0 ? ksafe : kk[u];
                const float4 qv = s1[ks];
                const float4 c = s2[ks];
                contrib = contrib || ok[u][0] || ok[u][1]; // branch-free: a lane that blends neither pixel adds zeros
                const float2 cx = make_float2(c.x, c.x), cy = make_float2(c.y, c.y), cz = make_float2(c.z, c.z),
                             az = make_float2(c.w, c.w);
                const float2 qx = make_float2(qv.x, qv.x), qy = make_float2(qv.y, qv.y);
                const float2 nal = make_float2(ok[u][0] ? -fminf(kAlphaMax, ar[u][0]) : 0.f,
                                               ok[u][1] ? -fminf(kAlphaMax, ar[u][1]) : 0.f);
                const float2 om = __fadd2_rn(make_float2(1.f, 1.f), nal);
                const float2 iom = make_float2(__fdividef(1.0f, om.x), __fdividef(1.0f, om.y));
                const float2 Ti = __fmul2_rn(T2, iom);
                const float2 nwgt = __fmul2_rn(nal, Ti);
                G[u][6] = __ffma2_rn(nwgt, dc0, G[u][6]);
                G[u][7] = __ffma2_rn(nwgt, dc1, G[u][7]);
                G[u][8] = __ffma2_rn(nwgt, dc2, G[u][8]);
                G[u][9] = __ffma2_rn(nwgt, dd, G[u][9]);
                const float2 dcc = __ffma2_rn(dd, az, __ffma2_rn(dc2, cz, __ffma2_rn(dc1, cy, __fmul2_rn(dc0, cx))));
                const float2 dal = __ffma2_rn(ndcs, iom, __fmul2_rn(dcc, Ti));
                ndcs = __ffma2_rn(nwgt, dcc, ndcs);
                T2 = Ti;
                // the 0.99 clamp passes no gradient to opacity and footprint
                const float2 dalm = make_float2(ar[u][0] < kAlphaMax ? dal.x : 0.f, ar[u][1] < kAlphaMax ? dal.y : 0.f);
                const float2 dx = make_float2(dxs[u][0], dxs[u][1]);
                const float dy1 = dys[u];
                G[u][5] = __ffma2_rn(dalm, make_float2(ex[u][0], ex[u][1]), G[u][5]);
                const float2 ngp = __fmul2_rn(dalm, nal); // -dL/dalpha * alpha
                // w = Q d (Q the conic): dpower/dd = -w and dpower/dSigma2 = w w^T / 2
                const float qyd = qv.y * dy1, qzd = qv.z * dy1;
                const float2 wxv = __ffma2_rn(qx, dx, make_float2(qyd, qyd));
                const float2 wyv = __ffma2_rn(qy, dx, make_float2(qzd, qzd));
                G[u][0] = __ffma2_rn(ngp, wxv, G[u][0]);
                G[u][1] = __ffma2_rn(ngp, wyv, G[u][1]);
                const float2 nhw = __fmul2_rn(__fmul2_rn(ngp, make_float2(-0.5f, -0.5f)), wxv);
                G[u][2] = __ffma2_rn(nhw, wxv, G[u][2]);
                G[u][3] = __ffma2_rn(nhw, wyv, G[u][3]);
                G[u][4] = __ffma2_rn(__fmul2_rn(__fmul2_rn(ngp, make_float2(-0.5f, -0.5f)), wyv), wyv, G[u][4]);
            }
#pragma unroll
            for (int u = 0; u < kGroup; ++u) {
#pragma unroll
                for (int x = 0; x < 6; ++x) g[10 * u + x] = G[u][x].x + G[u][x].y;
#pragma unroll
                for (int x = 6; x < 10; ++x) g[10 * u + x] = -(G[u][x].x + G[u][x].y);
            }
            if (__any_sync(0xffffffffu, contrib)) {
                quarter_transpose_sum32(g);
                // lane 8q + mq holds the quarter's sums of g[4 mq .. 4 mq + 3]
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int x = 4 * mq + j, u = x / 10, comp = x - 10 * u;
                    const int k = u == 0 ? kk[0] : u == 1 ? kk[1] : u == 2 ? kk[2] : -1;
                    if (x < 10 * kGroup && k >= 0 && g[j] != 0.0f) atomicAdd(acc + k * kAccStride + comp, g[j]);
                }
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < ncl; i += nthr) {
            const int k = (int)clist[i];
            const float4 *ak = reinterpret_cast<const float4 *>(acc + k * kAccStride);
            const float4 x0 = ak[0], x1 = ak[1], x2 = ak[2];
            if (x0.x != 0.f || x0.y != 0.f || x0.z != 0.f || x0.w != 0.f || x1.x != 0.f || x1.y != 0.f ||
                x1.z != 0.f || x1.w != 0.f || x2.x != 0.f || x2.y != 0.f) {
                float4 *dst = reinterpret_cast<float4 *>(w.d_rec + (size_t)(ibc[k] & kKeyRecord) * kGradStride);
                atomicAdd(dst + 0, x0);
                atomicAdd(dst + 1, x1);
                atomicAdd(dst + 2, x2);
            }
        }
        __syncthreads();
    }
    cp_async_wait<0>();
}

// Sums v[0..19] over each 4-lane group of the warp with 15 shuffles
// (butterfly transpose over lane bits 2, 1): on return, lane 4g + m holds in
// v[0..4] the group's totals of v[5m .. 5m + 4].
__device__ __forceinline__ void quad_transpose_sum20(float (&v)[20])
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 2, m = 20; o > 0; o >>= 1, m >>= 1) {
        const bool up = lane & o;
#pragma unroll
        for (int i = 0; i < m / 2; ++i) {
            const float keep = up ? v[i + m / 2] : v[i], send = up ? v[i] : v[i + m / 2];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
}

constexpr int kGroup4 = 2; // entries per 4-lane reduction (20 sums)
// Batch depth of the 4-lane walk, whatever the forward's: one-warp CTAs need
// small batch buffers to keep 16 warps per SM (measured: 64 against 128,
// 3.72 against 4.54 ms at 64 envs); the backward's batches are its own.
constexpr int kQ4Batch = 64;

// The quarter walk with 2 x 2 pixels per lane: the tile's 4 x 4 quarters of
// the forward (four per forward warp) walked by 4 lanes each, eight per warp,
// so one warp takes the quarters of two forward warps.  Same lists, same
// per-pixel arithmetic as blendq_backward_tile; the gradient sums of a group
// are reduced over 4 lanes instead of 8 (a quarter of the shuffles per pixel).
__device__ __forceinline__ void blendq4_backward_tile(const Ws &w, const gs_camera *cams, const float *d_rgb,
                                                     const float *d_depth, int bin, uint32_t seg_lo, uint32_t seg_hi,
                                                     int64_t ck_slot, float4 *sm, float *acc, uint32_t *sidx,
                                                     uint32_t *clist, uint32_t *spq, uint8_t *qls,
                                                     uint32_t *smax_last)
{
    const Table *tb = w.tb;
    const int B = min(tb->batch_depth, kQ4Batch);
    const int nthr = blockDim.x;
    const int v = bin / tb->tiles_per_view;
    const int t = bin - v * tb->tiles_per_view;
    const int tyi = t / tb->tiles_x, txi = t - tyi * tb->tiles_x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int Q = lane >> 2, m = lane & 3;  // quarter of the warp (0..7), lane in it
    const int fw = 2 * warp + (Q >> 2), qq = Q & 3; // the forward warp and its quarter
    const int wx = tb->tile_w >> 3;
    const int tx0 = txi * tb->tile_w, ty0 = tyi * tb->tile_h;
    const int i0 = tx0 + (fw % wx) * 8 + (qq & 1) * 4 + (m & 1) * 2;
    const int j0 = ty0 + (fw / wx) * 8 + (qq >> 1) * 4 + (m >> 1) * 2;
    const int W = tb->W, H = tb->H;
    const gs_camera &cam = cams[v];
    const float pyc[2] = {pix_c(j0, cam.cy), pix_c(j0 + 1, cam.cy)};
    const float2 npx2 = make_float2(-pix_c(i0, cam.cx), -pix_c(i0 + 1, cam.cx));
    const size_t HW = (size_t)W * H;
    uint32_t start, n;
    bin_range(w, bin, start, n);
    const unsigned long long *keys = w.keys + start;
    const uint32_t *pqb = w.pq + start;
    const uint32_t R = (uint32_t)tb->n_records;
    const int qs = qlist_stride(B);
    uint8_t *ql = qls + warp * 8 * qs;

    // per pixel (row r, column p): T, dL/dC, dL/dD, the colour and depth behind
    float T[2][2], dC0[2][2], dC1[2][2], dC2[2][2], dD[2][2], S0[2][2], S1[2][2], S2[2][2], SD[2][2];
    uint32_t last[2][2];
    uint32_t tlast = 0;
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            const int i = i0 + p, j = j0 + r;
            T[r][p] = 1.0f; dC0[r][p] = dC1[r][p] = dC2[r][p] = dD[r][p] = 0.f;
            S0[r][p] = S1[r][p] = S2[r][p] = SD[r][p] = 0.f;
            last[r][p] = 0;
            if (i < W && j < H) {
                const size_t px = (size_t)j * W + i;
                T[r][p] = w.pix_T[(size_t)v * HW + px];
                last[r][p] = w.pix_last[(size_t)v * HW + px];
                dC0[r][p] = d_rgb[(3 * (size_t)v + 0) * HW + px];
                dC1[r][p] = d_rgb[(3 * (size_t)v + 1) * HW + px];
                dC2[r][p] = d_rgb[(3 * (size_t)v + 2) * HW + px];
                dD[r][p] = d_depth[(size_t)v * HW + px];
                S0[r][p] = T[r][p] * tb->bg[0];
                S1[r][p] = T[r][p] * tb->bg[1];
                S2[r][p] = T[r][p] * tb->bg[2];
            }
            tlast = max(tlast, last[r][p]);
        }
    if (threadIdx.x == 0) *smax_last = 0;
    __syncthreads();
    const uint32_t wl = __reduce_max_sync(0xffffffffu, tlast);
    if (lane == 0) atomicMax(smax_last, wl);
    __syncthreads();
    const uint32_t tile_last = min(*smax_last, n);
    if (seg_lo >= tile_last) return; // nothing blended in this segment
    const uint32_t n_proc = min(tile_last, seg_hi);
    if (n_proc < tile_last) {
        // start from the checkpoint before position seg_hi
        const int tpx = tb->tile_w * tb->tile_h;
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                const int i = i0 + p, j = j0 + r;
                if (i < W && j < H) {
                    const int lpx = (j - ty0) * tb->tile_w + (i - tx0);
                    const float4 ck = w.ck_C[(size_t)ck_slot * tpx + lpx];
                    const float ckd = w.ck_D[(size_t)ck_slot * tpx + lpx];
                    const float4 fin = w.pix_C[(size_t)v * HW + (size_t)j * W + i];
                    T[r][p] = ck.x;
                    S0[r][p] = fin.x - ck.y;
                    S1[r][p] = fin.y - ck.z;
                    S2[r][p] = fin.z - ck.w;
                    SD[r][p] = fin.w - ckd;
                }
            }
    }
    // per row, both pixels as packed FP32 pairs (as blendq_backward_tile)
    float2 T2[2], dc0[2], dc1[2], dc2[2], dd[2], ndcs[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        T2[r] = make_float2(T[r][0], T[r][1]);
        dc0[r] = make_float2(dC0[r][0], dC0[r][1]);
        dc1[r] = make_float2(dC1[r][0], dC1[r][1]);
        dc2[r] = make_float2(dC2[r][0], dC2[r][1]);
        dd[r] = make_float2(dD[r][0], dD[r][1]);
        float x[2];
#pragma unroll
        for (int e = 0; e < 2; ++e)
            x[e] = -(dC0[r][e] * S0[r][e] + dC1[r][e] * S1[r][e] + dC2[r][e] * S2[r][e] + dD[r][e] * SD[r][e]);
        ndcs[r] = make_float2(x[0], x[1]);
    }
    const int nb = (int)((n_proc - seg_lo + B - 1) / B);
    // batch b covers [lo_b, hi_b), hi_b = n_proc - b B, lo_b >= seg_lo
    auto lo_of = [&](int b) {
        const int32_t x = (int32_t)n_proc - (b + 1) * B;
        return x < (int32_t)seg_lo ? (int32_t)seg_lo : x;
    };
    auto hi_of = [&](int b) { return (int32_t)n_proc - b * B; };
    unsigned long long kr[kMaxPerB];
    auto load_keys = [&](int b) {
        const int32_t lo = lo_of(b), cnt = hi_of(b) - lo;
#pragma unroll
        for (int qq2 = 0; qq2 < kMaxPerB; ++qq2) {
            const int e = threadIdx.x + qq2 * nthr;
            kr[qq2] = (b < nb && e < cnt) ? keys[lo + e] : 0ull;
        }
    };
    auto issue = [&](int b) {
        float4 *buf = sm + (b & 1) * 3 * B;
        uint32_t *ib = sidx + (b & 1) * B;
        uint32_t *pb = spq + (b & 1) * B;
        const int32_t lo = lo_of(b), cnt = hi_of(b) - lo;
#pragma unroll
        for (int qq2 = 0; qq2 < kMaxPerB; ++qq2) {
            const int e = threadIdx.x + qq2 * nthr;
            if (e < cnt) {
                const uint32_t word = (uint32_t)kr[qq2], fl = word & kKeyBlended;
                uint32_t rec = word & kKeyRecord;
                if (rec >= R) rec = 0; // only after a capacity overflow
                if (fl) { // pairs that no pixel blended are never read
                    const float4 *src = w.rec + 3 * (size_t)rec;
                    cp_async16(buf + e, src);
                    cp_async16(buf + B + e, src + 1);
                    cp_async16(buf + 2 * B + e, src + 2);
                    pb[e] = pqb[lo + e];
                }
                ib[e] = rec | fl;
            }
        }
    };
    if (nb > 0) {
        load_keys(0);
        issue(0);
        cp_async_commit();
        load_keys(1);
    }
    const unsigned lt = (1u << lane) - 1u;
    for (int b = 0; b < nb; ++b) {
        if (b + 1 < nb) issue(b + 1);
        cp_async_commit();
        if (b + 2 < nb) load_keys(b + 2);
        const int32_t lo = lo_of(b), cnt = hi_of(b) - lo;
        for (int k = threadIdx.x; k < cnt * kAccStride; k += nthr) acc[k] = 0.0f;
        cp_async_wait<1>();
        __syncthreads();
        const uint32_t *ibc = sidx + (b & 1) * B;
        const uint32_t *pbc = spq + (b & 1) * B;
        if (threadIdx.x < 32) { // the batch's blended entries, in list order
            uint32_t base = 0;
            for (int c0 = 0; c0 < cnt; c0 += 32) {
                const int k = c0 + lane;
                const bool f = k < cnt && (ibc[k] & kKeyBlended);
                const unsigned bal = __ballot_sync(0xffffffffu, f);
                if (f) clist[base + __popc(bal & lt)] = (uint32_t)k;
                base += __popc(bal);
            }
            if (lane == 0) clist[B] = base;
        }
        __syncthreads();
        const int ncl = (int)clist[B];
        // this warp's eight quarter lists: bytes 2 warp and 2 warp + 1 of the
        // forward's per-warp quarter bits
        int len[8];
#pragma unroll
        for (int x = 0; x < 8; ++x) len[x] = 0;
        for (int c0 = 0; c0 < ncl; c0 += 32) {
            const int i = c0 + lane;
            const uint32_t k = i < ncl ? clist[i] : 0u;
            const uint32_t word = i < ncl ? pbc[k] >> (16 * warp) : 0u;
            const uint32_t qb = (word & 15u) | ((word >> 4) & 0xf0u);
#pragma unroll
            for (int x = 0; x < 8; ++x) {
                const bool hit = (qb >> x) & 1u;
                const unsigned bal = __ballot_sync(0xffffffffu, hit);
                if (hit) ql[x * qs + len[x] + __popc(bal & lt)] = (uint8_t)k;
                len[x] += __popc(bal);
            }
        }
        __syncwarp();
        int mylen = len[0], maxlen = len[0];
#pragma unroll
        for (int x = 1; x < 8; ++x) {
            mylen = Q == x ? len[x] : mylen;
            maxlen = max(maxlen, len[x]);
        }
        const uint8_t *myl = ql + Q * qs;
        const float4 *s0 = sm + (b & 1) * 3 * B, *s1 = s0 + B, *s2 = s0 + 2 * B;
        // the slot a lane past its list's end reads: a gathered record, so that
        // the branch-free gradient phase multiplies finite values by its zero
        // weights (the slots of pairs no pixel blended hold stale data)
        const int ksafe = ncl > 0 ? (int)clist[0] : 0;
        // groups of kGroup4 entries per quarter, back to front: falloff and
        // alpha of the lane's four pixels first, then per row the sequential
        // transmittance rebuild and gradients (branch-free), then one 4-lane
        // reduction of the group's 10 x kGroup4 sums
        for (int s = 0; s < maxlen; s += kGroup4) {
            int kk[kGroup4]; // batch entries of the group (-1: past this quarter's list)
#pragma unroll
            for (int u = 0; u < kGroup4; ++u) kk[u] = s + u < mylen ? (int)myl[mylen - 1 - s - u] : -1;
            float g[20];
#pragma unroll
            for (int x = 0; x < 20; ++x) g[x] = 0.f;
            bool contrib = false;
            float ar[kGroup4][2][2], ex[kGroup4][2][2], dxs[kGroup4][2], dys[kGroup4][2];
            bool ok[kGroup4][2][2];
#pragma unroll
            for (int u = 0; u < kGroup4; ++u) {
                const int k = kk[u], ks = k < 0 ? ksafe : k;
                const float4 a = s0[ks];
                const float4 qv = s1[ks];
                const float2 dx2 = __fadd2_rn(make_float2(a.x, a.x), npx2); // = a.x - pxc
                dxs[u][0] = dx2.x;
                dxs[u][1] = dx2.y;
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const float dy = __fsub_rn(a.y, pyc[r]);
                    dys[u][r] = dy;
                    const float2 p2 = gauss_power2(qv.x, qv.y, qv.z, dx2, dy);
                    const float pw[2] = {p2.x, p2.y};
#pragma unroll
                    for (int p = 0; p < 2; ++p) {
                        ex[u][r][p] = __expf(pw[p]);
                        ar[u][r][p] = __fmul_rn(qv.w, ex[u][r][p]); // = raw_alpha(qv.w, power)
                        ok[u][r][p] = k >= 0 && (uint32_t)(lo + k) < last[r][p] && fabsf(dxs[u][p]) <= a.z &&
                                      fabsf(dy) <= a.w && pw[p] <= 0.0f && fminf(kAlphaMax, ar[u][r][p]) >= kAlphaMin;
                        if (!ok[u][r][p]) ex[u][r][p] = 0.f; // finite where a zero weight multiplies it
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < kGroup4; ++u) {
                const int ks = kk[u] < 0 ? ksafe : kk[u];
                const float4 qv = s1[ks];
                const float4 c = s2[ks];
                const float2 cx = make_float2(c.x, c.x), cy = make_float2(c.y, c.y), cz = make_float2(c.z, c.z),
                             az = make_float2(c.w, c.w);
                const float2 qx = make_float2(qv.x, qv.x), qy = make_float2(qv.y, qv.y);
                const float2 dx = make_float2(dxs[u][0], dxs[u][1]);
                float2 Gs[10];
#pragma unroll
                for (int x = 0; x < 10; ++x) Gs[x] = make_float2(0.f, 0.f);
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    contrib = contrib || ok[u][r][0] || ok[u][r][1];
                    const float2 nal = make_float2(ok[u][r][0] ? -fminf(kAlphaMax, ar[u][r][0]) : 0.f,
                                                   ok[u][r][1] ? -fminf(kAlphaMax, ar[u][r][1]) : 0.f);
                    const float2 om = __fadd2_rn(make_float2(1.f, 1.f), nal);
                    const float2 iom = make_float2(__fdividef(1.0f, om.x), __fdividef(1.0f, om.y));
                    const float2 Ti = __fmul2_rn(T2[r], iom);
                    const float2 nwgt = __fmul2_rn(nal, Ti);
                    Gs[6] = __ffma2_rn(nwgt, dc0[r], Gs[6]);
                    Gs[7] = __ffma2_rn(nwgt, dc1[r], Gs[7]);
                    Gs[8] = __ffma2_rn(nwgt, dc2[r], Gs[8]);
                    Gs[9] = __ffma2_rn(nwgt, dd[r], Gs[9]);
                    const float2 dcc =
                        __ffma2_rn(dd[r], az, __ffma2_rn(dc2[r], cz, __ffma2_rn(dc1[r], cy, __fmul2_rn(dc0[r], cx))));
                    const float2 dal = __ffma2_rn(ndcs[r], iom, __fmul2_rn(dcc, Ti));
                    ndcs[r] = __ffma2_rn(nwgt, dcc, ndcs[r]);
                    T2[r] = Ti;
                    // the 0.99 clamp passes no gradient to opacity and footprint
                    const float2 dalm = make_float2(ar[u][r][0] < kAlphaMax ? dal.x : 0.f,
                                                    ar[u][r][1] < kAlphaMax ? dal.y : 0.f);
                    const float dy1 = dys[u][r];
                    Gs[5] = __ffma2_rn(dalm, make_float2(ex[u][r][0], ex[u][r][1]), Gs[5]);
                    const float2 ngp = __fmul2_rn(dalm, nal); // -dL/dalpha * alpha
                    // w = Q d (Q the conic): dpower/dd = -w and dpower/dSigma2 = w w^T / 2
                    const float qyd = qv.y * dy1, qzd = qv.z * dy1;
                    const float2 wxv = __ffma2_rn(qx, dx, make_float2(qyd, qyd));
                    const float2 wyv = __ffma2_rn(qy, dx, make_float2(qzd, qzd));
                    Gs[0] = __ffma2_rn(ngp, wxv, Gs[0]);
                    Gs[1] = __ffma2_rn(ngp, wyv, Gs[1]);
                    const float2 nhw = __fmul2_rn(__fmul2_rn(ngp, make_float2(-0.5f, -0.5f)), wxv);
                    Gs[2] = __ffma2_rn(nhw, wxv, Gs[2]);
                    Gs[3] = __ffma2_rn(nhw, wyv, Gs[3]);
                    Gs[4] = __ffma2_rn(__fmul2_rn(__fmul2_rn(ngp, make_float2(-0.5f, -0.5f)), wyv), wyv, Gs[4]);
                }
#pragma unroll
                for (int x = 0; x < 6; ++x) g[10 * u + x] = Gs[x].x + Gs[x].y;
#pragma unroll
                for (int x = 6; x < 10; ++x) g[10 * u + x] = -(Gs[x].x + Gs[x].y);
            }
            if (__any_sync(0xffffffffu, contrib)) {
                quad_transpose_sum20(g);
                // lane 4Q + m holds the quarter's sums of g[5 m .. 5 m + 4]
#pragma unroll
                for (int j = 0; j < 5; ++j) {
                    const int x = 5 * m + j, u = x / 10, comp = x - 10 * u;
                    const int k = u == 0 ? kk[0] : kk[1];
                    if (k >= 0 && g[j] != 0.0f) atomicAdd(acc + k * kAccStride + comp, g[j]);
                }
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < ncl; i += nthr) {
            const int k = (int)clist[i];
            const float4 *ak = reinterpret_cast<const float4 *>(acc + k * kAccStride);
            const float4 x0 = ak[0], x1 = ak[1], x2 = ak[2];
            if (x0.x != 0.f || x0.y != 0.f || x0.z != 0.f || x0.w != 0.f || x1.x != 0.f || x1.y != 0.f ||
                x1.z != 0.f || x1.w != 0.f || x2.x != 0.f || x2.y != 0.f) {
                float4 *dst = reinterpret_cast<float4 *>(w.d_rec + (size_t)(ibc[k] & kKeyRecord) * kGradStride);
                atomicAdd(dst + 0, x0);
                atomicAdd(dst + 1, x1);
                atomicAdd(dst + 2, x2);
            }
        }
        __syncthreads();
    }
    cp_async_wait<0>();
}

// Overwrite mode: every gradient row is first set to zero (the preprocess
// backward then writes the rows of the Gaussians some view sees).  The clearing
// is split into items of kZeroFloats floats that the persistent blend-backward
// CTAs take one at a time between their tiles, so that the store stream to HBM
// runs under the issue-bound blend instead of after it.  The 16-byte aligned
// body of an item is written by TMA bulk copies from a zeroed shared-memory
// buffer (one thread issues them; the load/store pipeline the blend needs for
// its shared-memory traffic stays free), the unaligned ends by plain stores.
constexpr int64_t kZeroFloats = 1 << 16;
// Bytes of zeros in shared memory, the size of each bulk copy: 4 KB measured
// fastest on GB300 (1 KB copies left the engine's issue rate on the critical
// path, 8 KB and more cost resident CTAs).
constexpr int kZeroBuf = 4096;

__device__ __forceinline__ void bulk_zero(char *dst, uint32_t bytes, uint32_t zbuf_saddr, uint64_t policy)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group.L2::cache_hint [%0], [%1], %2, %3;\n" ::"l"(dst),
                 "r"(zbuf_saddr), "r"(bytes), "l"(policy)
                 : "memory");
}

__device__ __noinline__ void zero_item(const ZeroWork &zw, uint32_t z, uint32_t zbuf_saddr)
{
    int a = 0;
    while (a + 1 < kZeroArrays && zw.first[a + 1] <= z) ++a;
    float *p = zw.p[a];
    const int64_t lo = (int64_t)(z - zw.first[a]) * kZeroFloats, hi = min(zw.n[a], lo + kZeroFloats);
    // plain stores up to the first 16-byte boundary and after the last
    const int64_t a4 = min(hi, lo + (int64_t)((((16 - (reinterpret_cast<uintptr_t>(p + lo) & 15)) & 15)) >> 2));
    const int64_t n4 = (hi - a4) >> 2;
    if (lo + (int64_t)threadIdx.x < a4) p[lo + threadIdx.x] = 0.f;
    const int64_t t0 = a4 + 4 * n4;
    if (t0 + (int64_t)threadIdx.x < hi) p[t0 + threadIdx.x] = 0.f;
    if (threadIdx.x == 0 && n4 > 0) {
        // the zeros stream through L2 ahead of the blend's records: evict them first
        uint64_t policy;
        asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(policy));
        char *d = reinterpret_cast<char *>(p + a4);
        for (int64_t off = 0, nb = n4 * 16; off < nb; off += kZeroBuf)
            bulk_zero(d + off, (uint32_t)min((int64_t)kZeroBuf, nb - off), zbuf_saddr, policy);
        asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
    }
}

// Q4: 2 x 1 pixels per lane in the forward, 2 x 2 in the backward
// (blendq4_backward_tile; the CTA has half the forward's threads)
template <int PX, int PY, bool Q4>
__global__ void blend_backward_kernel(const gs_camera *__restrict__ cams, Ws w, const float *__restrict__ d_rgb,
                                      const float *__restrict__ d_depth, ZeroWork zw)
{
    extern __shared__ float4 smem_b[];
    __shared__ uint32_t smax_last, item;
    constexpr bool Q = PX == 2 && PY == 1; // quarter lists (blendq_backward_tile)
    const int B = Q4 ? min(w.tb->batch_depth, kQ4Batch) : w.tb->batch_depth;
    float *acc = reinterpret_cast<float *>(smem_b + 2 * 3 * B); // [B][kAccStride]
    uint32_t *sidx = reinterpret_cast<uint32_t *>(acc + B * kAccStride); // [2][B]
    uint32_t *clist = sidx + 2 * B;                                        // [B + 1]
    uint32_t *spq = clist + B + 1;                                         // Q: [2][B] quarter bits
    uint8_t *qls = reinterpret_cast<uint8_t *>(spq + (Q ? 2 * B : 0));     // Q: per warp 4 quarter lists
    const int qbytes = Q ? (int)(blockDim.x >> 5) * (Q4 ? 8 : 4) * qlist_stride(B) : 0;
    // zeros for the clearing items' bulk copies (16-byte aligned, after the lists)
    const uint32_t zoff = ((uint32_t)(reinterpret_cast<char *>(qls + qbytes) - reinterpret_cast<char *>(smem_b)) +
                           15u) & ~15u;
    float4 *zbuf = reinterpret_cast<float4 *>(reinterpret_cast<char *>(smem_b) + zoff);
    const uint32_t zbuf_saddr = (uint32_t)__cvta_generic_to_shared(zbuf);
    if (zw.total) {
        for (int i = threadIdx.x; i < kZeroBuf / 16; i += blockDim.x) zbuf[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); // visible to the bulk copies
    }
    // items: the kSeg-long segments of the heavy bins (largest bins first),
    // then every other bin whole
    const uint32_t nhi = w.hdr->n_heavy_items, nh = w.hdr->n_heavy;
    const uint32_t n_items = nhi + (uint32_t)w.tb->n_bins;
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&w.hdr->n_backward, 1u); // d_rec is dirty from here on
    // the first clear_ctas CTAs (one per two SMs) clear first, so that the
    // store stream runs from the start beside the heavy tiles; the others take
    // tiles, then what is left of the clearing
    for (bool clearing = zw.total && blockIdx.x < zw.clear_ctas; clearing;) {
        __syncthreads();
        if (threadIdx.x == 0) item = atomicAdd(&w.hdr->queue_zero, 1u);
        __syncthreads();
        if (item >= zw.total) break;
        zero_item(zw, item, zbuf_saddr);
    }
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) item = atomicAdd(&w.hdr->queue_bwd, 1u);
        __syncthreads();
        if (item >= n_items) break;
        if (item < nhi) {
            uint32_t lo = 0, hi = nh - 1; // heavy bin: last h with heavy_seg[h] <= item
            while (lo < hi) {
                const uint32_t mid = (lo + hi + 1) >> 1;
                if (w.heavy_seg[mid] <= item) lo = mid;
                else hi = mid - 1;
            }
            const uint32_t s = item - w.heavy_seg[lo];
            if constexpr (Q4)
                blendq4_backward_tile(w, cams, d_rgb, d_depth, (int)w.heavy[lo], s * kSeg, (s + 1) * kSeg,
                                      (int64_t)w.heavy_seg[lo] + s, smem_b, acc, sidx, clist, spq, qls, &smax_last);
            else if constexpr (Q)
                blendq_backward_tile(w, cams, d_rgb, d_depth, (int)w.heavy[lo], s * kSeg, (s + 1) * kSeg,
                                     (int64_t)w.heavy_seg[lo] + s, smem_b, acc, sidx, clist, spq, qls, &smax_last);
            else
                blend_backward_tile<PX, PY>(w, cams, d_rgb, d_depth, (int)w.heavy[lo], s * kSeg, (s + 1) * kSeg,
                                            (int64_t)w.heavy_seg[lo] + s, smem_b, acc, sidx, clist, &smax_last);
        } else {
            const uint32_t b = item - nhi;
            if (w.bin_count[b] + w.bin_fcount[b] < w.hdr->heavy_min) {
                if constexpr (Q4)
                    blendq4_backward_tile(w, cams, d_rgb, d_depth, (int)b, 0u, 0xffffffffu, 0, smem_b, acc, sidx,
                                          clist, spq, qls, &smax_last);
                else if constexpr (Q)
                    blendq_backward_tile(w, cams, d_rgb, d_depth, (int)b, 0u, 0xffffffffu, 0, smem_b, acc, sidx,
                                         clist, spq, qls, &smax_last);
                else
                    blend_backward_tile<PX, PY>(w, cams, d_rgb, d_depth, (int)b, 0u, 0xffffffffu, 0, smem_b, acc,
                                                sidx, clist, &smax_last);
            }
        }
    }
    for (;;) { // clearing items left when the tiles ran out
        __syncthreads();
        if (threadIdx.x == 0) item = zw.total ? atomicAdd(&w.hdr->queue_zero, 1u) : zw.total;
        __syncthreads();
        if (item >= zw.total) break;
        zero_item(zw, item, zbuf_saddr);
    }
    // the bulk copies read the shared buffer until they complete
    if (zw.total && threadIdx.x == 0) asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory");
}

// ---------------------------------------------------------------------------
// preprocess backward
// ---------------------------------------------------------------------------

// dL/d(dir) += sum_k grad(Y_k) * w_k for the degree-3 basis.
__device__ __forceinline__ void sh_dir_vjp(float x, float y, float z, const float (&wk)[16], float &gx, float &gy,
                                           float &gz)
{
    const float xx = x * x, yy = y * y, zz = z * z;
    gx += -kSH1 * wk[3];
    gy += -kSH1 * wk[1];
    gz += kSH1 * wk[2];
    gx += kSH2a * y * wk[4]; gy += kSH2a * x * wk[4];
    gy += -kSH2a * z * wk[5]; gz += -kSH2a * y * wk[5];
    gx += -2.f * kSH2b * x * wk[6]; gy += -2.f * kSH2b * y * wk[6]; gz += 4.f * kSH2b * z * wk[6];
    gx += -kSH2a * z * wk[7]; gz += -kSH2a * x * wk[7];
    gx += 2.f * kSH2c * x * wk[8]; gy += -2.f * kSH2c * y * wk[8];
    gx += -6.f * kSH3a * x * y * wk[9]; gy += -kSH3a * (3.f * xx - 3.f * yy) * wk[9];
    gx += kSH3b * y * z * wk[10]; gy += kSH3b * x * z * wk[10]; gz += kSH3b * x * y * wk[10];
    gx += 2.f * kSH3c * x * y * wk[11]; gy += -kSH3c * (4.f * zz - xx - 3.f * yy) * wk[11];
    gz += -8.f * kSH3c * y * z * wk[11];
    gx += -6.f * kSH3d * x * z * wk[12]; gy += -6.f * kSH3d * y * z * wk[12];
    gz += kSH3d * (6.f * zz - 3.f * xx - 3.f * yy) * wk[12];
    gx += -kSH3c * (4.f * zz - 3.f * xx - yy) * wk[13]; gy += 2.f * kSH3c * x * y * wk[13];
    gz += -8.f * kSH3c * x * z * wk[13];
    gx += 2.f * kSH3e * x * z * wk[14]; gy += -2.f * kSH3e * y * z * wk[14]; gz += kSH3e * (xx - yy) * wk[14];
    gx += -kSH3a * (3.f * xx - 3.f * yy) * wk[15]; gy += 6.f * kSH3a * x * y * wk[15];
}

struct GaussInB {
    const float *means, *log_scales, *quats, *ologits, *cov3d;
    const void *sh;
    // fused LBS (gs_render_avatars_backward): the avatar rows are posed again
    // here, as the forward's preprocess posed them, from their canonical rows
    const float *av_means, *av_log_scales, *av_quats, *av_weights, *av_G;
    const uint16_t *av_ids;
    const int32_t *av_of;
    int32_t n_avatars, n_joints;
};

// Streams the 48 SH coefficients of Gaussian g and returns, per basis
// function, sum_ch k[i][ch] * gch[ch].
template <int SHT>
__device__ __forceinline__ void sh_weighted(const void *sh, int64_t g, const float (&gch)[3], float (&wk)[16])
{
#pragma unroll
    for (int i = 0; i < 16; ++i) wk[i] = 0.f;
    if (SHT == GS_SH_F32) {
        const float4 *p = reinterpret_cast<const float4 *>(sh) + g * 12;
#pragma unroll
        for (int i = 0; i < 12; ++i) {
            const float4 v = __ldcg(p + i);
            const float c[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) wk[(4 * i + j) / 3] += c[j] * gch[(4 * i + j) % 3];
        }
    } else {
        const uint4 *p = reinterpret_cast<const uint4 *>(sh) + g * 6;
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            const uint4 v = __ldcg(p + i);
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
                wk[(8 * i + 2 * j) / 3] += lo * gch[(8 * i + 2 * j) % 3];
                wk[(8 * i + 2 * j + 1) / 3] += hi * gch[(8 * i + 2 * j + 1) % 3];
            }
        }
    }
}

// Full chain for one Gaussian seen by at least one view: screen-space
// gradients of each visible view back to the Gaussian's parameters.  The
// per-Gaussian rows are scattered (a quarter of the rows are seen), so they
// are loaded through L2 only (ld.global.cg): an L1 fill would pull whole
// 128-byte lines of mostly unseen neighbours.
template <int SHT, bool OVERWRITE, bool FUSED>
__device__ __forceinline__ void gaussian_backward(const gs_camera *__restrict__ cams, const GaussInB &gin, const Ws &w,
                                                  const Table *tb, const GradOut &o, int64_t g, int e)
{
    const int vb = tb->env_view_begin[e], ve = tb->env_view_begin[e + 1];
    const int64_t local = g - tb->env_off[e];
    const bool posed = FUSED && g >= tb->env_cov_begin[e];
    const bool use_cov = posed || (gin.cov3d != nullptr && g >= tb->env_cov_begin[e]);
    float mx, my, mz;
    float S[6];
    float3 ls = make_float3(0.f, 0.f, 0.f);
    float4 q = make_float4(1.f, 0.f, 0.f, 0.f);
    if (FUSED && posed) {
        // posed mean and covariance by LBS, bit for bit the forward's
        const int64_t i = tb->env_av_base[e] + (g - tb->env_cov_begin[e]);
        const int a = clamp_avatar(__ldg(gin.av_of + i), gin.n_avatars);
        const ushort4 id = clamp_ids(__ldg(reinterpret_cast<const ushort4 *>(gin.av_ids) + i), gin.n_joints);
        const float4 wt = __ldg(reinterpret_cast<const float4 *>(gin.av_weights) + i);
        float mu[3];
        lbs_gaussian(gin.av_G + (size_t)a * gin.n_joints * 12, id, wt,
                     make_float3(__ldcg(gin.av_means + 3 * i), __ldcg(gin.av_means + 3 * i + 1),
                                 __ldcg(gin.av_means + 3 * i + 2)),
                     make_float3(__ldcg(gin.av_log_scales + 3 * i), __ldcg(gin.av_log_scales + 3 * i + 1),
                                 __ldcg(gin.av_log_scales + 3 * i + 2)),
                     __ldcg(reinterpret_cast<const float4 *>(gin.av_quats) + i), mu, S);
        mx = mu[0];
        my = mu[1];
        mz = mu[2];
    } else {
        mx = __ldcg(gin.means + 3 * g);
        my = __ldcg(gin.means + 3 * g + 1);
        mz = __ldcg(gin.means + 3 * g + 2);
        if (use_cov) {
#pragma unroll
            for (int i = 0; i < 6; ++i) S[i] = __ldcg(gin.cov3d + 6 * g + i);
        } else {
            ls = make_float3(__ldcg(gin.log_scales + 3 * g), __ldcg(gin.log_scales + 3 * g + 1),
                             __ldcg(gin.log_scales + 3 * g + 2));
            q = __ldcg(reinterpret_cast<const float4 *>(gin.quats) + g);
            sigma_from_sq(ls, q, S);
        }
    }
    float op = 0.f; // from the record rows (the forward wrote it there)
    float gS[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float gm0 = 0.f, gm1 = 0.f, gm2 = 0.f, go = 0.f;
    bool first_sh = true;
    float4 *dsh4 = reinterpret_cast<float4 *>(o.sh + 48 * g);
    const int W = tb->W, H = tb->H;
    for (int kv = vb; kv < ve; ++kv) {
        const int v = tb->env_views[kv];
        const uint32_t rec = (uint32_t)(tb->view_rec_off[v] + local);
        if (!((__ldcg(w.vis + (rec >> 5)) >> (rec & 31)) & 1u)) continue;
        const float4 *gr4 = reinterpret_cast<const float4 *>(w.d_rec + (size_t)rec * kGradStride);
        const float4 r0 = __ldcg(gr4), r1 = __ldcg(gr4 + 1), r2 = __ldcg(gr4 + 2), r3 = __ldcg(gr4 + 3);
        const uint32_t clamped = __float_as_uint(r3.x); // colour channels clamped at 0
        op = r2.z;
        // a channel clamped at 0 passes no gradient
        const float gch[3] = {(clamped & 1u) ? 0.f : r1.z, (clamped & 2u) ? 0.f : r1.w, (clamped & 4u) ? 0.f : r2.x};
        // (uc, vc, Sigma2 xx, Sigma2 xy, Sigma2 yy, opacity, r, g, b, z): the 2D
        // covariance part as the symmetric matrix dL/dSigma2 (xy = half of dL/db)
        const float g_u = r0.x, g_v = r0.y, G00 = r0.z, G01 = r0.w, G11 = r1.x, g_op = r1.y;
        const float g_z = r2.y;
        const gs_camera &cam = cams[v];
        const float zk = depth_key(mx, my, mz, cam);
        Proj pj;
        project_ewa(mx, my, mz, zk, S, cam, W, H, pj);

        const float px = pj.px, py = pj.py, ipz = 1.0f / pj.pz, ipz2 = ipz * ipz;
        float gpx = g_u * cam.fx * ipz, gpy = g_v * cam.fy * ipz;
        float gpz = -g_u * cam.fx * px * ipz2 - g_v * cam.fy * py * ipz2 + g_z;
        const float *t = pj.t;
        // dL/dSigma = T^T G2 T (symmetric)
        const float h0 = G00 * t[0] + G01 * t[3], h1 = G00 * t[1] + G01 * t[4], h2 = G00 * t[2] + G01 * t[5];
        const float k0 = G01 * t[0] + G11 * t[3], k1 = G01 * t[1] + G11 * t[4], k2 = G01 * t[2] + G11 * t[5];
        gS[0] += t[0] * h0 + t[3] * k0;
        gS[1] += t[0] * h1 + t[3] * k1;
        gS[2] += t[0] * h2 + t[3] * k2;
        gS[3] += t[1] * h1 + t[4] * k1;
        gS[4] += t[1] * h2 + t[4] * k2;
        gS[5] += t[2] * h2 + t[5] * k2;
        // dL/dT = 2 G2 T Sigma ; rows x = 0, 1
        const float TS00 = t[0] * S[0] + t[1] * S[1] + t[2] * S[2], TS01 = t[0] * S[1] + t[1] * S[3] + t[2] * S[4],
                    TS02 = t[0] * S[2] + t[1] * S[4] + t[2] * S[5];
        const float TS10 = t[3] * S[0] + t[4] * S[1] + t[5] * S[2], TS11 = t[3] * S[1] + t[4] * S[3] + t[5] * S[4],
                    TS12 = t[3] * S[2] + t[4] * S[4] + t[5] * S[5];
        const float gT00 = 2.f * (G00 * TS00 + G01 * TS10), gT01 = 2.f * (G00 * TS01 + G01 * TS11),
                    gT02 = 2.f * (G00 * TS02 + G01 * TS12);
        const float gT10 = 2.f * (G01 * TS00 + G11 * TS10), gT11 = 2.f * (G01 * TS01 + G11 * TS11),
                    gT12 = 2.f * (G01 * TS02 + G11 * TS12);
        // T = J W: dL/dJ = dL/dT W^T (entries J00, J02, J11, J12)
        const float gJ00 = gT00 * cam.R[0] + gT01 * cam.R[1] + gT02 * cam.R[2];
        const float gJ02 = gT00 * cam.R[6] + gT01 * cam.R[7] + gT02 * cam.R[8];
        const float gJ11 = gT10 * cam.R[3] + gT11 * cam.R[4] + gT12 * cam.R[5];
        const float gJ12 = gT10 * cam.R[6] + gT11 * cam.R[7] + gT12 * cam.R[8];
        gpz += -gJ00 * cam.fx * ipz2 - gJ11 * cam.fy * ipz2;
        if (!pj.clampx) {
            gpx += -gJ02 * cam.fx * ipz2;
            gpz += 2.f * gJ02 * cam.fx * px * ipz2 * ipz;
        } else {
            gpz += gJ02 * cam.fx * pj.tx * ipz2;
        }
        if (!pj.clampy) {
            gpy += -gJ12 * cam.fy * ipz2;
            gpz += 2.f * gJ12 * cam.fy * py * ipz2 * ipz;
        } else {
            gpz += gJ12 * cam.fy * pj.ty * ipz2;
        }
        // p = W d
        float gd0 = cam.R[0] * gpx + cam.R[3] * gpy + cam.R[6] * gpz;
        float gd1 = cam.R[1] * gpx + cam.R[4] * gpy + cam.R[7] * gpz;
        float gd2 = cam.R[2] * gpx + cam.R[5] * gpy + cam.R[8] * gpz;
        // colour: SH coefficients get Y(dir) x gch, the direction gets grad(Y) . (k gch)
        float idn;
        const float3 dir = view_dir(pj.d0, pj.d1, pj.d2, idn);
        const float x = dir.x, y = dir.y, z = dir.z;
        float Y[16];
        sh_basis(x, y, z, Y);
#pragma unroll
        for (int i = 0; i < 12; ++i) {
            float vals[4];
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) vals[jj] = Y[(4 * i + jj) / 3] * gch[(4 * i + jj) % 3];
            float4 val = make_float4(vals[0], vals[1], vals[2], vals[3]);
            if (!(OVERWRITE && first_sh)) {
                const float4 cur = dsh4[i];
                val = make_float4(cur.x + val.x, cur.y + val.y, cur.z + val.z, cur.w + val.w);
            }
            dsh4[i] = val;
        }
        first_sh = false;
        float wk[16];
        sh_weighted<SHT>(gin.sh, g, gch, wk);
        float gx = 0.f, gy = 0.f, gz = 0.f;
        sh_dir_vjp(x, y, z, wk, gx, gy, gz);
        const float dot = gx * x + gy * y + gz * z;
        gd0 += (gx - x * dot) * idn;
        gd1 += (gy - y * dot) * idn;
        gd2 += (gz - z * dot) * idn;
        gm0 += gd0;
        gm1 += gd1;
        gm2 += gd2;
        go += g_op;
    }
    if (OVERWRITE) {
        o.means[3 * g] = gm0;
        o.means[3 * g + 1] = gm1;
        o.means[3 * g + 2] = gm2;
        o.ologits[g] = go * op * (1.0f - op);
    } else {
        o.means[3 * g] += gm0;
        o.means[3 * g + 1] += gm1;
        o.means[3 * g + 2] += gm2;
        o.ologits[g] += go * op * (1.0f - op);
    }
    if (use_cov) {
        if (o.cov3d) {
            float *dc = o.cov3d + 6 * g;
            const float v6[6] = {gS[0], 2.f * gS[1], 2.f * gS[2], gS[3], 2.f * gS[4], gS[5]};
            for (int i = 0; i < 6; ++i) dc[i] = OVERWRITE ? v6[i] : dc[i] + v6[i];
        }
        return;
    }
    // Sigma = M M^T, M = R diag(s): dL/dM = 2 gS M
    const float qn = sqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w), iq = 1.0f / qn;
    const float qw = q.x * iq, qx = q.y * iq, qy = q.z * iq, qz = q.w * iq;
    float R[9];
    quat_rot(qw, qx, qy, qz, R);
    const float sc[3] = {expf(ls.x), expf(ls.y), expf(ls.z)};
    const float Gs[9] = {gS[0], gS[1], gS[2], gS[1], gS[3], gS[4], gS[2], gS[4], gS[5]};
    float gR[9], gsv[3];
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) {
        float gscc = 0.f;
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            // (gS M)[r][cc] with M[k][cc] = R[k][cc] sc[cc]
            const float gM = 2.f * (Gs[3 * r] * R[cc] + Gs[3 * r + 1] * R[3 + cc] + Gs[3 * r + 2] * R[6 + cc]) * sc[cc];
            gscc += gM * R[3 * r + cc];
            gR[3 * r + cc] = gM * sc[cc];
        }
        gsv[cc] = gscc * sc[cc];
    }
    for (int i = 0; i < 3; ++i) o.log_scales[3 * g + i] = OVERWRITE ? gsv[i] : o.log_scales[3 * g + i] + gsv[i];
    const float gw = gR[1] * (-2 * qz) + gR[2] * (2 * qy) + gR[3] * (2 * qz) + gR[5] * (-2 * qx) + gR[6] * (-2 * qy) +
                     gR[7] * (2 * qx);
    const float gx = gR[1] * (2 * qy) + gR[2] * (2 * qz) + gR[3] * (2 * qy) + gR[4] * (-4 * qx) + gR[5] * (-2 * qw) +
                     gR[6] * (2 * qz) + gR[7] * (2 * qw) + gR[8] * (-4 * qx);
    const float gy = gR[0] * (-4 * qy) + gR[1] * (2 * qx) + gR[2] * (2 * qw) + gR[3] * (2 * qx) + gR[5] * (2 * qz) +
                     gR[6] * (-2 * qw) + gR[7] * (2 * qz) + gR[8] * (-4 * qy);
    const float gz = gR[0] * (-4 * qz) + gR[1] * (-2 * qw) + gR[2] * (2 * qx) + gR[3] * (2 * qw) + gR[4] * (-4 * qz) +
                     gR[5] * (2 * qy) + gR[6] * (2 * qx) + gR[7] * (2 * qy);
    const float dq = gw * qw + gx * qx + gy * qy + gz * qz;
    const float4 gq4 = make_float4((gw - qw * dq) * iq, (gx - qx * dq) * iq, (gy - qy * dq) * iq, (gz - qz * dq) * iq);
    float4 *dqo = reinterpret_cast<float4 *>(o.quats) + g;
    if (OVERWRITE) {
        *dqo = gq4;
    } else {
        const float4 cur = *dqo;
        *dqo = make_float4(cur.x + gq4.x, cur.y + gq4.y, cur.z + gq4.z, cur.w + gq4.w);
    }
}


// Chunked like the forward preprocess: every lane checks whether any view sees
// its Gaussian (the rows of an unseen one are not touched: in overwrite mode
// the blend backward has cleared them); the seen ones go through a per-warp
// ring queue and are processed 32 at a time, so that the
// long chain runs on full warps.
constexpr int kBwdWarpQ = 64;


template <int SHT, bool OVERWRITE, bool FUSED>
__global__ void __launch_bounds__(256, 2) preprocess_backward_kernel(const gs_camera *__restrict__ cams, GaussInB gin,
                                                                     Ws w, GradOut o, const __grid_constant__ Table tbp)
{
    __shared__ uint32_t qs[8][kBwdWarpQ];
    // the table as a kernel parameter: constant-bank operands, never reloaded
    // after the gradient stores
    const Table *tb = &tbp;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    uint32_t *q = qs[warp];
    int lo = 0, hi = tb->n_envs - 1; // env of the chunk (chunks never straddle envs)
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tb->chunk_off[mid] <= (int)blockIdx.x) lo = mid;
        else hi = mid - 1;
    }
    const int64_t g0 = tb->env_off[lo] + (int64_t)(blockIdx.x - tb->chunk_off[lo]) * tb->chunk;
    const int64_t g1 = min(g0 + tb->chunk, tb->env_off[lo + 1]);
    int head = 0, tail = 0;
    const int64_t env_base = tb->env_off[lo];
    const int vb = tb->env_view_begin[lo], ve = tb->env_view_begin[lo + 1];
    for (int64_t base = g0 + warp * 32; base < g1; base += 32 * nwarps) {
        const int64_t g = base + lane;
        bool seen = false;
        if (g < g1) {
            const int64_t local = g - env_base;
            for (int kv = vb; kv < ve && !seen; ++kv) {
                const uint32_t rec = (uint32_t)(tb->view_rec_off[tb->env_views[kv]] + local);
                seen = (__ldg(w.vis + (rec >> 5)) >> (rec & 31)) & 1u;
            }
        }
        const unsigned bal = __ballot_sync(0xffffffffu, seen);
        if (seen) q[(tail + __popc(bal & ((1u << lane) - 1u))) & (kBwdWarpQ - 1)] = (uint32_t)(g - g0);
        tail += __popc(bal);
        __syncwarp();
        if (tail - head >= 32) {
            const int64_t gg = g0 + q[(head + lane) & (kBwdWarpQ - 1)];
            head += 32;
            __syncwarp();
            gaussian_backward<SHT, OVERWRITE, FUSED>(cams, gin, w, tb, o, gg, lo);
        }
    }
    if (lane < tail - head)
        gaussian_backward<SHT, OVERWRITE, FUSED>(cams, gin, w, tb, o, g0 + q[(head + lane) & (kBwdWarpQ - 1)], lo);
}

// ---------------------------------------------------------------------------
// Record gradient rows: the forward leaves the rows of visible records at zero;
// a second backward of the same forward finds them filled by the first and
// clears them here (the gradient part only: opacity and clamp bits stay).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) clear_record_grads_kernel(Ws w, int64_t n_words)
{
    if (w.hdr->n_backward == 0) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_words * 32;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t bits = w.vis[i >> 5];
        if (!((bits >> (i & 31)) & 1u)) continue;
        float4 *row = reinterpret_cast<float4 *>(w.d_rec + (size_t)i * kGradStride);
        row[0] = row[1] = make_float4(0.f, 0.f, 0.f, 0.f);
        *reinterpret_cast<float2 *>(row + 2) = make_float2(0.f, 0.f); // the opacity stays
    }
}

void launch_clear_record_grads(const Ws &w, int64_t n_records, int n_sms, cudaStream_t s)
{
    const int64_t n_words = (n_records + 31) / 32;
    clear_record_grads_kernel<<<n_sms * 4, 256, 0, s>>>(w, n_words);
}

// ---------------------------------------------------------------------------
// popcount of the visibility mask (statistics only)
// ---------------------------------------------------------------------------
__global__ void count_visible_kernel(Ws w, int64_t n_words)
{
    uint32_t c = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_words; i += (int64_t)gridDim.x * blockDim.x)
        c += __popc(w.vis[i]);
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(&w.hdr->n_visible, c);
}

void launch_count_visible(const Ws &w, int64_t n_words, cudaStream_t s)
{
    count_visible_kernel<<<256, 256, 0, s>>>(w, n_words);
}

// q_warps: warps of a quarter-list CTA (2 x 1 pixels per lane), else 0
static int blend_bwd_smem(int batch_depth, int q_warps)
{
    int base = 2 * 3 * batch_depth * (int)sizeof(float4) + batch_depth * kAccStride * 4 + 2 * batch_depth * 4 +
               (batch_depth + 1) * 4;
    if (q_warps) base += 2 * batch_depth * 4 + q_warps * 4 * qlist_stride(batch_depth);
    return ((base + 15) & ~15) + kZeroBuf;
}

// The clearing items of the gradient arrays of n Gaussians (none for NULL).
static ZeroWork zero_work(const GradOut *clear, int64_t n)
{
    ZeroWork zw;
    memset(&zw, 0, sizeof(zw));
    if (!clear) return zw;
    float *ps[kZeroArrays] = {clear->sh, clear->means, clear->ologits, clear->log_scales, clear->quats, clear->cov3d};
    const int64_t ns[kZeroArrays] = {48 * n, 3 * n, n, 3 * n, 4 * n, clear->cov3d ? 6 * n : 0};
    uint32_t acc = 0;
    for (int a = 0; a < kZeroArrays; ++a) {
        zw.p[a] = ps[a];
        zw.n[a] = ps[a] ? ns[a] : 0;
        zw.first[a] = acc;
        acc += (uint32_t)((zw.n[a] + kZeroFloats - 1) / kZeroFloats);
    }
    zw.total = acc;
    return zw;
}

// gs_zero_gradients: the same clearing items outside the blend backward, for
// a stream beside the forward.  Each CTA zeroes its 4 KB source and takes the
// items in turn.
__global__ void __launch_bounds__(128) zero_gradients_kernel(ZeroWork zw)
{
    __shared__ __align__(16) float4 zbuf[kZeroBuf / 16];
    for (int i = threadIdx.x; i < kZeroBuf / 16; i += blockDim.x) zbuf[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); // visible to the bulk copies
    __syncthreads();
    const uint32_t saddr = (uint32_t)__cvta_generic_to_shared(zbuf);
    for (uint32_t z = blockIdx.x; z < zw.total; z += gridDim.x) zero_item(zw, z, saddr);
    if (threadIdx.x == 0) asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory");
}

void launch_zero_gradients(const GradOut &o, int64_t n, int n_ctas, cudaStream_t s)
{
    const ZeroWork zw = zero_work(&o, n);
    if (zw.total) zero_gradients_kernel<<<(unsigned)std::min<uint32_t>((uint32_t)n_ctas, zw.total), 128, 0, s>>>(zw);
}

// threads: the forward's CTA size; Q4 launches half of them (2 x 2 pixels per lane)
template <int PX, int PY, bool Q4>
static void launch_bb(const gs_camera *cams, const Ws &w, const float *d_rgb, const float *d_depth, int n_bins,
                      int threads, int batch_depth, int n_sms, const ZeroWork &zw, cudaStream_t s)
{
    const int bd = Q4 ? std::min(batch_depth, kQ4Batch) : batch_depth;
    const int smem = blend_bwd_smem(bd, PX == 2 && PY == 1 ? threads / 32 : 0);
    const int bt = Q4 ? threads / 2 : threads;
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, blend_backward_kernel<PX, PY, Q4>, bt, smem);
    int grid = n_sms * (nb > 0 ? nb : 1);
    if (grid > n_bins) grid = n_bins;
    blend_backward_kernel<PX, PY, Q4><<<grid, bt, smem, s>>>(cams, w, d_rgb, d_depth, zw);
}

template <int PX, int PY>
static int bb_limit_t()
{
    cudaFuncAttributes a;
    if (cudaFuncGetAttributes(&a, blend_backward_kernel<PX, PY, false>) != cudaSuccess) return 0;
    return a.maxThreadsPerBlock;
}

int blend_backward_thread_limit(int px, int py)
{
    if (px == 2 && py == 2) return bb_limit_t<2, 2>();
    if (px == 2) return bb_limit_t<2, 1>();
    if (py == 2) return bb_limit_t<1, 2>();
    return bb_limit_t<1, 1>();
}

void launch_blend_backward(const gs_camera *cams, const Ws &w, const float *d_rgb, const float *d_depth, int n_bins,
                           int px, int py, int threads, int batch_depth, int n_sms, const GradOut *clear, int64_t n,
                           cudaStream_t s)
{
    // 2 x 1 pixels per lane with an even number of forward warps: the backward
    // walks each quarter with 4 lanes of 2 x 2 pixels, in batches of at most
    // kQ4Batch (its staging needs the depth <= kMaxPerB x its threads)
    const bool q4 = px == 2 && py == 1 && (threads / 32) % 2 == 0 &&
                    std::min(batch_depth, kQ4Batch) <= kMaxPerB * (threads / 2);
    ZeroWork zw = zero_work(clear, n);
    // CTAs that clear before taking tiles, measured fastest: one per SM with the
    // one-warp CTAs of the 4-lane walk (a quarter or twice that: slower), one
    // per two SMs otherwise (all SMs, twice that: slower)
    if (clear) zw.clear_ctas = (uint32_t)(q4 ? n_sms : (n_sms + 1) / 2);
    if (px == 2 && py == 2) launch_bb<2, 2, false>(cams, w, d_rgb, d_depth, n_bins, threads, batch_depth, n_sms, zw, s);
    else if (q4) launch_bb<2, 1, true>(cams, w, d_rgb, d_depth, n_bins, threads, batch_depth, n_sms, zw, s);
    else if (px == 2) launch_bb<2, 1, false>(cams, w, d_rgb, d_depth, n_bins, threads, batch_depth, n_sms, zw, s);
    else if (py == 2) launch_bb<1, 2, false>(cams, w, d_rgb, d_depth, n_bins, threads, batch_depth, n_sms, zw, s);
    else launch_bb<1, 1, false>(cams, w, d_rgb, d_depth, n_bins, threads, batch_depth, n_sms, zw, s);
}

template <bool OW, bool FUSED>
static void launch_pb(const Table &tb, const GaussInB &gin, int sh_dtype, const gs_camera *cams, const Ws &w,
                      const GradOut &o, unsigned grid, cudaStream_t s)
{
    switch (sh_dtype) {
    case GS_SH_F16: preprocess_backward_kernel<GS_SH_F16, OW, FUSED><<<grid, 256, 0, s>>>(cams, gin, w, o, tb); break;
    case GS_SH_BF16: preprocess_backward_kernel<GS_SH_BF16, OW, FUSED><<<grid, 256, 0, s>>>(cams, gin, w, o, tb); break;
    default: preprocess_backward_kernel<GS_SH_F32, OW, FUSED><<<grid, 256, 0, s>>>(cams, gin, w, o, tb); break;
    }
}

void launch_preprocess_backward(const Table &tb, const gs_gaussians *g, const gs_camera *cams, const Ws &w,
                                const GradOut &o, int n_chunks, bool overwrite, cudaStream_t s, const gs_avatars *av,
                                const float *joint_G)
{
    const unsigned grid = (unsigned)n_chunks;
    if (!grid) return;
    GaussInB gin{g->means, g->log_scales, g->quats, g->opacity_logits, g->cov3d, g->sh,
                 nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 0, 0};
    const bool fused = av && joint_G;
    if (fused) {
        gin.av_means = av->means; gin.av_log_scales = av->log_scales; gin.av_quats = av->quats;
        gin.av_weights = av->weights; gin.av_G = joint_G; gin.av_ids = av->joint_ids; gin.av_of = av->avatar_of;
        gin.n_avatars = av->n_avatars; gin.n_joints = av->n_joints;
    }
    if (overwrite) {
        if (fused) launch_pb<true, true>(tb, gin, g->sh_dtype, cams, w, o, grid, s);
        else launch_pb<true, false>(tb, gin, g->sh_dtype, cams, w, o, grid, s);
    } else {
        if (fused) launch_pb<false, true>(tb, gin, g->sh_dtype, cams, w, o, grid, s);
        else launch_pb<false, false>(tb, gin, g->sh_dtype, cams, w, o, grid, s);
    }
}

cudaError_t configure_backward_kernels()
{
    const int smem = blend_bwd_smem(256, 8);
    const void *ks[] = {reinterpret_cast<const void *>(blend_backward_kernel<1, 1, false>),
                        reinterpret_cast<const void *>(blend_backward_kernel<2, 1, false>),
                        reinterpret_cast<const void *>(blend_backward_kernel<2, 1, true>),
                        reinterpret_cast<const void *>(blend_backward_kernel<1, 2, false>),
                        reinterpret_cast<const void *>(blend_backward_kernel<2, 2, false>)};
    cudaError_t e = cudaSuccess;
    for (const void *k : ks)
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    return e;
}

} // namespace gs
