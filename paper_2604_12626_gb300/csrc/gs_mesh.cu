// gs_mesh.cu -- the triangle-mesh layer of a mixed scene (sm_103a): the mesh
// pass whose colour and depth the composite of Sec. 3.2 merges with the
// Gaussian pass, rasterised here in CUDA (no graphics API).
//
//   mesh_setup_kernel   one thread per (view, triangle): view transform, near
//                       cull, screen vertices, 1/z, signed area and the pixel
//                       bounding box -> a 96-byte record
//   mesh_raster_kernel  one CTA per (view, 16x16 tile), one thread per pixel:
//                       the boxes of 256 triangles at a time tested against
//                       the tile, the records of those that meet it gathered
//                       into shared memory in index order; inside test on the
//                       edge functions, perspective-correct depth and colour,
//                       nearest depth kept (the lower triangle index on a tie)
#include <cmath>

#include "gs_internal.cuh"
#include "gs_launch.h"

namespace gs {

constexpr int kMeshTile = 16;
constexpr int kMeshBatch = 256;

// (sx0, sy0, sx1, sy1) (sx2, sy2, iz0, iz1) (iz2, area, box_x, box_y) (c0) (c1) (c2)
// box_x = x0 | x1 << 16 (x0 = 0xffff: culled), colours (r, g, b, 0)
struct MeshRec {
    float4 a, b, c, c0, c1, c2;
};

__global__ void __launch_bounds__(256) mesh_setup_kernel(MeshIn in, const gs_camera *__restrict__ cams, MeshTable t,
                                                         MeshRec *__restrict__ rec)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= t.view_rec_off[t.n_views]) return;
    int v = 0;
    while (r >= t.view_rec_off[v + 1]) ++v; // few views: linear
    const int e = t.view_env[v];
    const int64_t tri = t.env_off[e] + (r - t.view_rec_off[v]);
    const gs_camera &cam = cams[v];
    float sx[3], sy[3], iz[3];
    bool ok = true;
    float4 col[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        int32_t vi = in.tris[3 * tri + k];
        vi = vi < 0 ? 0 : (vi >= in.n_verts ? (int32_t)in.n_verts - 1 : vi);
        const float d0 = __fsub_rn(in.verts[3 * vi], cam.C[0]), d1 = __fsub_rn(in.verts[3 * vi + 1], cam.C[1]),
                    d2 = __fsub_rn(in.verts[3 * vi + 2], cam.C[2]);
        const float qx = cam.R[0] * d0 + cam.R[1] * d1 + cam.R[2] * d2;
        const float qy = cam.R[3] * d0 + cam.R[4] * d1 + cam.R[5] * d2;
        const float qz = cam.R[6] * d0 + cam.R[7] * d1 + cam.R[8] * d2;
        ok = ok && qz > t.near_plane;
        sx[k] = cam.fx * qx / qz + cam.cx;
        sy[k] = cam.fy * qy / qz + cam.cy;
        iz[k] = 1.0f / qz;
        col[k] = make_float4(in.colors[3 * vi], in.colors[3 * vi + 1], in.colors[3 * vi + 2], 0.f);
    }
    const float area = (sx[1] - sx[0]) * (sy[2] - sy[0]) - (sy[1] - sy[0]) * (sx[2] - sx[0]);
    ok = ok && area != 0.0f && isfinite(area);
    int x0 = 0xffff, x1 = 0, y0 = 0xffff, y1 = 0; // culled: a box no tile intersects
    if (ok) {
        // pixel box, one pixel of slack against rounding (the edge test decides)
        const float lx = fminf(sx[0], fminf(sx[1], sx[2])), hx = fmaxf(sx[0], fmaxf(sx[1], sx[2]));
        const float ly = fminf(sy[0], fminf(sy[1], sy[2])), hy = fmaxf(sy[0], fmaxf(sy[1], sy[2]));
        x0 = (int)fmaxf(0.f, floorf(lx) - 1.f);
        x1 = (int)fminf((float)(t.W - 1), ceilf(hx) + 1.f);
        y0 = (int)fmaxf(0.f, floorf(ly) - 1.f);
        y1 = (int)fminf((float)(t.H - 1), ceilf(hy) + 1.f);
        if (x0 > x1 || y0 > y1) x0 = 0xffff, x1 = 0, y0 = 0xffff, y1 = 0;
    }
    MeshRec m;
    m.a = make_float4(sx[0], sy[0], sx[1], sy[1]);
    m.b = make_float4(sx[2], sy[2], iz[0], iz[1]);
    m.c = make_float4(iz[2], area, __uint_as_float((uint32_t)x0 | ((uint32_t)x1 << 16)),
                      __uint_as_float((uint32_t)y0 | ((uint32_t)y1 << 16)));
    m.c0 = col[0];
    m.c1 = col[1];
    m.c2 = col[2];
    rec[r] = m;
}

__global__ void __launch_bounds__(kMeshTile *kMeshTile) mesh_raster_kernel(MeshTable t, const MeshRec *__restrict__ rec,
                                                                          float *rgb, float *depth)
{
    __shared__ MeshRec s[kMeshBatch]; // records of the batch whose box meets this tile, in index order
    __shared__ int n_hit, warp_n[kMeshTile * kMeshTile / 32];
    const int v = blockIdx.y;
    const int tiles_x = (t.W + kMeshTile - 1) / kMeshTile;
    const int tx0 = (blockIdx.x % tiles_x) * kMeshTile, ty0 = (blockIdx.x / tiles_x) * kMeshTile;
    const int i = tx0 + (threadIdx.x % kMeshTile), j = ty0 + (threadIdx.x / kMeshTile);
    const float px = (float)i, py = (float)j;
    float best = INFINITY, r0 = t.bg[0], r1 = t.bg[1], r2 = t.bg[2];
    const int64_t lo = t.view_rec_off[v], hi = t.view_rec_off[v + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t b0 = lo; b0 < hi; b0 += kMeshBatch) {
        const int cnt = (int)min((int64_t)kMeshBatch, hi - b0);
        __syncthreads();
        // each thread tests one triangle's box (16 of the record's 96 bytes)
        // against the tile; the hits are compacted in index order (warp
        // ballots, then a scan over the warps) and only their records gathered
        bool h = false;
        if ((int)threadIdx.x < cnt) {
            const float4 mc = rec[b0 + threadIdx.x].c;
            const uint32_t bx = __float_as_uint(mc.z), by = __float_as_uint(mc.w);
            const int x0 = (int)(bx & 0xffffu), x1 = (int)(bx >> 16), y0 = (int)(by & 0xffffu), y1 = (int)(by >> 16);
            h = !(x1 < tx0 || x0 > tx0 + kMeshTile - 1 || y1 < ty0 || y0 > ty0 + kMeshTile - 1);
        }
        const unsigned bal = __ballot_sync(0xffffffffu, h);
        if (lane == 0) warp_n[warp] = __popc(bal);
        __syncthreads();
        if (threadIdx.x == 0) {
            int acc = 0;
            for (int q = 0; q < kMeshTile * kMeshTile / 32; ++q) {
                const int c = warp_n[q];
                warp_n[q] = acc;
                acc += c;
            }
            n_hit = acc;
        }
        __syncthreads();
        if (h) s[warp_n[warp] + __popc(bal & ((1u << lane) - 1u))] = rec[b0 + threadIdx.x];
        __syncthreads();
        const int nh = n_hit;
        for (int q = 0; q < nh; ++q) {
            const int k = q;
            const float4 A = s[k].a, B = s[k].b, C = s[k].c;
            const float X[3] = {A.x, A.z, B.x}, Y[3] = {A.y, A.w, B.y};
            float e[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const int c = (a + 1) % 3;
                e[a] = (X[c] - X[a]) * (py - Y[a]) - (Y[c] - Y[a]) * (px - X[a]);
            }
            const float area = C.y;
            const bool in = area > 0.f ? (e[0] >= 0.f && e[1] >= 0.f && e[2] >= 0.f)
                                       : (e[0] <= 0.f && e[1] <= 0.f && e[2] <= 0.f);
            if (!in) continue;
            const float w0 = e[1] / area * B.z, w1 = e[2] / area * B.w, w2 = e[0] / area * C.x;
            const float z = 1.0f / (w0 + w1 + w2);
            if (z < best) {
                best = z;
                const float4 c0 = s[k].c0, c1 = s[k].c1, c2 = s[k].c2;
                r0 = z * (w0 * c0.x + w1 * c1.x + w2 * c2.x);
                r1 = z * (w0 * c0.y + w1 * c1.y + w2 * c2.y);
                r2 = z * (w0 * c0.z + w1 * c1.z + w2 * c2.z);
            }
        }
    }
    if (i < t.W && j < t.H) {
        const size_t HW = (size_t)t.W * t.H, p = (size_t)j * t.W + i;
        rgb[(3 * (size_t)v + 0) * HW + p] = r0;
        rgb[(3 * (size_t)v + 1) * HW + p] = r1;
        rgb[(3 * (size_t)v + 2) * HW + p] = r2;
        depth[(size_t)v * HW + p] = best < INFINITY ? best : 0.0f;
    }
}

size_t mesh_record_bytes() { return sizeof(MeshRec); }

void launch_mesh(const MeshIn &in, const gs_camera *cams, const MeshTable &t, void *rec, float *rgb, float *depth,
                 cudaStream_t s)
{
    const int64_t R = t.view_rec_off[t.n_views];
    if (R > 0)
        mesh_setup_kernel<<<(unsigned)((R + 255) / 256), 256, 0, s>>>(in, cams, t, static_cast<MeshRec *>(rec));
    const int tiles = ((t.W + kMeshTile - 1) / kMeshTile) * ((t.H + kMeshTile - 1) / kMeshTile);
    mesh_raster_kernel<<<dim3(tiles, t.n_views), kMeshTile * kMeshTile, 0, s>>>(t, static_cast<const MeshRec *>(rec),
                                                                                   rgb, depth);
}

} // namespace gs
