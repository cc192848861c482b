/*
 * gs.h -- C ABI of libgs: batched Gaussian-splatting RGB-D rendering with
 * drivable LBS avatars, hand-written CUDA for sm_103a (GB300).
 *
 * The paper (Habitat-GS) renders scene Gaussians with a CUDA tile-based 3D
 * Gaussian Splatting rasteriser producing colour and depth (Sec. 3.1, Sec. 3.2),
 * and deforms canonical avatar Gaussians with a CUDA linear-blend-skinning
 * kernel over per-frame SMPL-X joint matrices before rasterising all avatars in
 * one pass (Sec. 3.2 last paragraph, Sec. 3.3, Sec. 3.3.1).  This header is the
 * boundary of that hot path; everything behind it runs in this library's own
 * kernels.
 *
 * Conventions (all entry points):
 *  - Every pointer argument named as "device" is a caller-owned device pointer;
 *    the library never allocates device memory and never frees anything.  All
 *    scratch lives in a caller-provided workspace (see gs_render_workspace_size).
 *  - Arrays are dense, row-major, float32 unless stated, and must be 16-byte
 *    aligned (GS_ERR_ALIGNMENT otherwise), except gs_gaussians.means,
 *    log_scales, opacity_logits and cov3d, which need 4 bytes, so that one env
 *    of a concatenated batch can be passed as a slice.  Struct arguments are
 *    host memory.
 *  - Work is enqueued on `stream` (a cudaStream_t; NULL is the legacy default
 *    stream).  No call synchronises the stream except gs_get_status and
 *    gs_render_stats, and no call reads device memory from the host, so
 *    gs_render / gs_render_backward / gs_render_avatars(_backward) /
 *    gs_deform_avatars(_backward) can be captured into a CUDA graph.
 *  - Returns GS_OK or a negative gs_status.  Errors the device detects (pair
 *    capacity exceeded) set a status word in the workspace, which gs_render
 *    clears when it starts and gs_render_backward leaves as it is; read it with
 *    gs_get_status.  Outputs of such a call are unspecified but every write
 *    stays in bounds.
 *  - Camera convention: world->camera rotation R (rows: right, down, forward;
 *    OpenCV), camera centre C in world coordinates, so p = R (mu - C).  Pixel
 *    (i, j) has its centre at image coordinates (i, j).
 */
#ifndef GS_H
#define GS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t gs_status;
#define GS_OK 0
#define GS_ERR_INVALID_ARG (-1)
#define GS_ERR_ALIGNMENT (-2)
#define GS_ERR_WORKSPACE_TOO_SMALL (-3)
#define GS_ERR_CAPACITY (-4)
#define GS_ERR_CUDA (-5)
#define GS_ERR_TIMEOUT (-6)
#define GS_ERR_UNSUPPORTED (-7)

/* storage type of the SH coefficients (arithmetic is always float32) */
#define GS_SH_F32 0
#define GS_SH_F16 1
#define GS_SH_BF16 2

/* gs_render_config.flags */
#define GS_FLAG_PERSISTENT 1      /* blend with a persistent grid over an (view, tile) work queue */
#define GS_FLAG_NORMALIZE_DEPTH 2 /* depth = D / (1 - T), 0 where 1 - T < 1e-4 (forward only) */
#define GS_FLAG_GRAD_OVERWRITE 4  /* gs_render_backward writes every gradient row (zeros where a
                                     Gaussian is seen by no view) instead of adding to it */
#define GS_FLAG_COUNT_EVALS 8     /* the forward also counts blend evaluations into
                                     gs_stats.n_evaluations and n_covered (one atomic per warp
                                     and tile) and lists every Gaussian for the tiles its square
                                     footprint touches (the same images, slower) */
#define GS_FLAG_AVATAR_CANONICAL_SH 16 /* gs_render_avatars: evaluate an avatar Gaussian's SH at
                                     A3^-1 (mu' - C) normalised, the view direction in its
                                     canonical frame (A3: linear part of its skinning matrix);
                                     without it, at the world view direction */
#define GS_FLAG_GRAD_PRECLEARED 32 /* gs_render_backward / gs_render_avatars_backward write the rows
                                      of the Gaussians some view sees and leave every other row as
                                      it is: on arrays set to zero beforehand (gs_zero_gradients,
                                      e.g. on a stream beside gs_render) the result of
                                      GS_FLAG_GRAD_OVERWRITE without its clearing */

#define GS_MAX_ENVS 512
#define GS_MAX_VIEWS 512

/* A pinhole camera, 64 bytes: p = R (mu - C); u = fx px/pz + cx, v = fy py/pz + cy. */
typedef struct {
    float R[9]; /* world->camera rotation, row-major */
    float C[3]; /* camera centre, world coordinates */
    float fx, fy, cx, cy;
} gs_camera;

/* The Gaussians of all environments, concatenated env after env (device).
 * Gaussian k of env e sits at index env_offsets[e] + k.  Within an env the
 * Gaussians from env_cov3d_begin[e] on (typically the posed avatars) take their
 * covariance from cov3d instead of (log_scales, quats). */
typedef struct {
    const float *means;          /* [N,3] world positions */
    const float *log_scales;     /* [N,3] log of the per-axis standard deviation */
    const float *quats;          /* [N,4] rotation (w, x, y, z), normalised by the kernel */
    const float *opacity_logits; /* [N] opacity = sigmoid(logit) */
    const void *sh;              /* [N,16,3] degree-3 SH, coefficient-major, channel fastest */
    int32_t sh_dtype;            /* GS_SH_F32 / GS_SH_F16 / GS_SH_BF16 */
    int32_t reserved;
    const float *cov3d;          /* [N,6] (xx, xy, xz, yy, yz, zz) or NULL */
    int64_t n;                   /* total Gaussians N */
} gs_gaussians;

/* Batch structure (host arrays; copied into the workspace by every call). */
typedef struct {
    int32_t n_envs;                 /* E, 1..GS_MAX_ENVS */
    int32_t n_views;                /* V, 1..GS_MAX_VIEWS; several views may share an env */
    const int64_t *env_offsets;     /* host [E+1], env_offsets[0] = 0, env_offsets[E] = N */
    const int64_t *env_cov3d_begin; /* host [E] absolute index, or NULL (no cov3d use) */
    const int32_t *view_env;        /* host [V] env of each view */
} gs_batch;

typedef struct {
    int32_t width, height;     /* image size shared by all views */
    int32_t tile_w, tile_h;    /* blend tile; 0 -> 16 x 16 */
    int32_t batch_depth;       /* Gaussians staged per shared-memory batch, 32..256 and at most
                                  4 x the CTA's threads; 0 -> 256 */
    int32_t flags;             /* GS_FLAG_* */
    float bg[3];               /* background colour added with the final transmittance */
    float near_plane;          /* Gaussians with FP32 view depth <= near are culled; 0 -> 0.2 */
    int64_t pair_capacity;     /* max (tile, Gaussian) pairs; 0 -> 4 x records + 65536 */
    int32_t pix_x, pix_y;      /* pixels per blend thread, each 1 or 2 (0 -> 1); the CTA has
                                  (tile_w / pix_x) x (tile_h / pix_y) threads, a multiple of 32.
                                  2 x 1: a warp per 8 x 8 block with a Gaussian list per 4 x 4
                                  quarter; tile_w, tile_h multiples of 8 and at most 4 warps
                                  (GS_ERR_UNSUPPORTED otherwise) */
} gs_render_config;

/* Per-call counters, read back by gs_render_stats (synchronises). */
typedef struct {
    int64_t n_records;  /* (view, Gaussian) records considered */
    int64_t n_visible;  /* records that passed near, conic and footprint culling */
    int64_t n_pairs;    /* (tile, Gaussian) pairs generated */
    int64_t max_bin;    /* largest pair count of one (view, tile) */
    int32_t status;     /* device status word (0 or a GS_ERR_* code) */
    int32_t reserved;
    int64_t n_evaluations; /* with GS_FLAG_COUNT_EVALS: sum over pixels of the covered Gaussians
                              examined in depth order up to and including the one that stops the
                              pixel (Sec. 3.2 blending rule); else 0 */
    int64_t n_covered;     /* with GS_FLAG_COUNT_EVALS: sum over pixels of the covered Gaussians up
                              to and including the last one blended (the adjoint's walk); else 0 */
} gs_stats;

/* Canonical avatar Gaussians for LBS (device). */
typedef struct {
    const float *means;         /* [M,3] canonical positions */
    const float *log_scales;    /* [M,3] */
    const float *quats;         /* [M,4] (w, x, y, z) */
    const uint16_t *joint_ids;  /* [M,4] joint index per skin weight, < n_joints */
    const float *weights;       /* [M,4] skin weights, used as given (no renormalisation) */
    const int32_t *avatar_of;   /* [M] avatar of each Gaussian, < n_avatars */
    const int64_t *dest;        /* [M] output index of each Gaussian, or NULL for 0..M-1 */
    int64_t m;
    int32_t n_avatars, n_joints; /* n_joints <= 64 */
} gs_avatars;

/* Workspace bytes needed by gs_render / gs_render_backward for this config
 * and batch (the backward reuses the forward's workspace). */
gs_status gs_render_workspace_size(const gs_render_config *cfg, const gs_batch *batch, size_t *bytes);

/* Forward render of V views (Sec. 3.2: CUDA 3DGS rasterisation to colour and
 * depth).  Pipeline: EWA projection + SH-3 colour per (view, Gaussian), binning
 * of (tile, depth key) pairs, per-tile sort by (FP32 view depth, index), tile
 * ranges, front-to-back blending (alpha = min(0.99, o exp(power)), skip alpha <
 * 1/255, stop before T < 1e-4).  A Gaussian covers pixel (i, j) iff
 * |i - u| <= r and |j - v| <= r, r = ceil(3 sqrt(lambda_max)).  A Gaussian is
 * listed only for the tiles where its alpha can reach 1/255 (a window inside
 * the square, with margins for FP32 rounding), which changes no output.
 *   cams          device [V] gs_camera
 *   out_rgb       device [V,3,H,W]  C + T bg
 *   out_depth     device [V,H,W]    sum z alpha T (raw), or normalised (flag)
 *   out_T         device [V,H,W]    final transmittance
 *   out_ncontrib  device [V,H,W] int32: the number of Gaussians blended into
 *                 that pixel
 * The workspace keeps what the backward needs.  A tile whose CTA
 * ((tile_w / pix_x) x (tile_h / pix_y) threads) exceeds what the blend kernels'
 * registers allow is rejected with GS_ERR_UNSUPPORTED (e.g. 32x32 at 1x1). */
gs_status gs_render(const gs_gaussians *g, const gs_batch *batch, const gs_camera *cams, const gs_render_config *cfg,
                    void *workspace, size_t workspace_bytes, float *out_rgb, float *out_depth, float *out_T,
                    int32_t *out_ncontrib, void *stream);

/* gs_render with the avatars posed inside the preprocess (Sec. 3.3: LBS of
 * the canonical avatar Gaussians, fused into the projection so that the posed
 * mean and covariance are never written to or read from memory).  The batch
 * must give env_cov3d_begin: rows [env_cov3d_begin[e], env_offsets[e+1]) of
 * env e are avatar Gaussians, and they are the canonical rows of `av` in env
 * order (env 0's first, then env 1's ...; av->dest must be NULL, av->m their
 * total).  For those rows g->means is read but ignored and g->log_scales,
 * g->quats, g->cov3d are not used; opacity and SH are g's rows as for the
 * scene.  joint_G: device [n_avatars, n_joints, 3, 4].  The result equals
 * gs_deform_avatars into those rows followed by gs_render; its adjoint is
 * gs_render_avatars_backward. */
gs_status gs_render_avatars(const gs_gaussians *g, const gs_batch *batch, const gs_avatars *av, const float *joint_G,
                            const gs_camera *cams, const gs_render_config *cfg, void *workspace,
                            size_t workspace_bytes, float *out_rgb, float *out_depth, float *out_T,
                            int32_t *out_ncontrib, void *stream);

/* Adjoint of gs_render_avatars (Sec. 3.3's LBS fused into the projection, and
 * its gradient through the skinning), for L with dL/drgb = d_rgb and dL/ddepth
 * = d_depth as in gs_render_backward.  Must follow gs_render_avatars with the
 * same arguments and an untouched workspace.  The preprocess backward poses
 * the avatar rows again by LBS (the same FP32 values as the forward: nothing
 * posed is read from memory), and the LBS adjoint then carries their
 * gradients to the canonical Gaussians and the joint matrices.
 *   d_means, d_log_scales, d_quats, d_opacity_logits, d_sh: as for
 *     gs_render_backward (ADDED, or overwritten under GS_FLAG_GRAD_OVERWRITE),
 *     all rows; an avatar row of d_means receives dL/d(posed mean), its rows
 *     of d_log_scales and d_quats are left as they are (accumulate) or zero
 *     (overwrite);
 *   d_cov3d: device [N,6], required: avatar rows receive dL/d(posed
 *     covariance) (xx, xy, xz, yy, yz, zz; an off-diagonal entry holds the
 *     gradient of both of its symmetric entries);
 *   d_canon_means [M,3], d_canon_log_scales [M,3], d_canon_quats [M,4],
 *   d_joint_G [n_avatars, n_joints, 3, 4]: device, 16-byte aligned, ADDED to
 *     (as gs_deform_avatars_backward does).
 * The result equals gs_render_backward of the posed rows followed by
 * gs_deform_avatars_backward, up to the order of floating-point atomics. */
gs_status gs_render_avatars_backward(const gs_gaussians *g, const gs_batch *batch, const gs_avatars *av,
                                     const float *joint_G, const gs_camera *cams, const gs_render_config *cfg,
                                     void *workspace, size_t workspace_bytes, const float *d_rgb,
                                     const float *d_depth, float *d_means, float *d_log_scales, float *d_quats,
                                     float *d_opacity_logits, float *d_sh, float *d_cov3d, float *d_canon_means,
                                     float *d_canon_log_scales, float *d_canon_quats, float *d_joint_G,
                                     void *stream);

/* gs_render without a workspace, for callers that cannot allocate device
 * memory -- for instance a sensor plugin inside a host simulator whose device
 * memory is owned by another framework's allocator, or a real-time path that
 * must not allocate after start-up.  The paper has no counterpart; it is an
 * addition of this library.
 * The scratch is a file-scope device array of GS_STATIC_SCRATCH_BYTES (64 MiB)
 * inside libgs, present on every GPU that loads the library until the process
 * exits.  Inputs and outputs are as for gs_render.  Problems whose workspace
 * (gs_render_workspace_size) exceeds the array are rejected with
 * GS_ERR_WORKSPACE_TOO_SMALL before any work is enqueued; 64 MiB holds about
 * 195k (view, Gaussian) records at 256x256 with the default pair capacity.
 * Allocates nothing: no cudaMalloc/cudaFree, no library allocation, and no
 * profiling events.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress), so make that first call before any stream
 * capture.  Under CUDA's lazy module loading (the default) that first call is
 * also when the 64 MiB are reserved on the device, so make it at start-up (or
 * set CUDA_MODULE_LOADING=EAGER to reserve them when the library loads); a
 * lookup that fails returns GS_ERR_CUDA and is tried again by the next call.
 * Every call on a device shares the one array and leaves its contents behind
 * (the call clears what must start at zero itself), so calls whose work
 * overlaps on the GPU -- two streams, or two threads -- race; serialise them.
 * The backward cannot follow this call (its state lives in the shared array).
 * A device-detected error (pair capacity exceeded) is read with
 * gs_render_static_status. */
#define GS_STATIC_SCRATCH_BYTES (64ll << 20)
gs_status gs_render_static(const gs_gaussians *g, const gs_batch *batch, const gs_camera *cams,
                           const gs_render_config *cfg, float *out_rgb, float *out_depth, float *out_T,
                           int32_t *out_ncontrib, void *stream);

/* gs_get_status for gs_render_static, whose status word lives in the static
 * array (the caller has no workspace pointer): synchronises `stream`, returns
 * the device status the last gs_render_static call on the current device left
 * (GS_OK or GS_ERR_CAPACITY) in *device_status and clears it.  The paper has
 * no counterpart.  Allocates nothing. */
gs_status gs_render_static_status(void *stream, int32_t *device_status);

/* Adjoint of gs_render for L with dL/drgb = d_rgb [V,3,H,W] and dL/ddepth =
 * d_depth [V,H,W] (device; raw depth only).  Must follow gs_render with the
 * same arguments and an untouched workspace.  Gradients are ADDED to the
 * outputs (device) -- or overwrites them with GS_FLAG_GRAD_OVERWRITE --:
 * d_means [N,3], d_log_scales [N,3], d_quats [N,4],
 * d_opacity_logits [N], d_sh [N,16,3] float32 whatever the SH storage type,
 * d_cov3d [N,6] or NULL (written for Gaussians that use cov3d).  The discrete
 * decisions are held fixed; the 0.99 clamp and the colour clamp at 0 pass zero
 * gradient where active. */
gs_status gs_render_backward(const gs_gaussians *g, const gs_batch *batch, const gs_camera *cams,
                             const gs_render_config *cfg, void *workspace, size_t workspace_bytes,
                             const float *d_rgb, const float *d_depth, float *d_means, float *d_log_scales,
                             float *d_quats, float *d_opacity_logits, float *d_sh, float *d_cov3d, void *stream);

/* Sets the parameter-gradient arrays of n Gaussians to zero -- d_sh
 * [n,16,3], d_means [n,3], d_opacity_logits [n], d_log_scales [n,3], d_quats
 * [n,4], d_cov3d [n,6] or NULL (device, 16-byte aligned) -- with TMA bulk
 * stores from n_ctas CTAs of 128 threads (n_ctas < 1: one per two SMs).  The
 * clearing that GS_FLAG_GRAD_OVERWRITE does inside the backward, as a call of
 * its own: enqueued on a second stream while gs_render runs (the blend leaves
 * HBM mostly idle), it takes the store stream off the backward, which then
 * runs with GS_FLAG_GRAD_PRECLEARED after an event joins the streams.  The
 * paper has no counterpart.  Asynchronous. */
gs_status gs_zero_gradients(int64_t n, float *d_means, float *d_log_scales, float *d_quats, float *d_opacity_logits,
                            float *d_sh, float *d_cov3d, int32_t n_ctas, void *stream);

/* Linear blend skinning (Sec. 3.3): A = sum_k w_k G[avatar][j_k] (3x4),
 * mean' = A[:, :3] mean + A[:, 3], cov' = A[:, :3] Sigma A[:, :3]^T with
 * Sigma = R(q) diag(exp(2 s)) R(q)^T.  joint_G: device [A, n_joints, 3, 4].
 * Writes out_means[dest[i]] ([.,3]) and out_cov3d[dest[i]] ([.,6]). */
gs_status gs_deform_avatars(const gs_avatars *av, const float *joint_G, float *out_means, float *out_cov3d,
                            void *stream);

/* Adjoint of gs_deform_avatars: reads d_means[dest[i]], d_cov3d[dest[i]] and
 * ADDS to d_canon_means [M,3], d_canon_log_scales [M,3], d_canon_quats [M,4]
 * and d_joint_G [A, n_joints, 3, 4] (device). */
gs_status gs_deform_avatars_backward(const gs_avatars *av, const float *joint_G, const float *d_means,
                                     const float *d_cov3d, float *d_canon_means, float *d_canon_log_scales,
                                     float *d_canon_quats, float *d_joint_G, void *stream);

/* Nearest-fragment composite of two RGB-D layers (Sec. 3.2: the full-screen
 * pass that merges the 3DGS colour and depth with the mesh pass, and the
 * avatars' Gaussian pass with the scene's).  Per pixel
 *   (C, D) = (D_a < D_b) ? (C_a, D_a) : (C_b, D_b),
 * where a depth that is not a positive finite number -- a pixel the layer
 * does not cover, e.g. gs_render's normalised depth 0 -- compares as
 * +infinity (so the second layer is kept when neither covers the pixel).
 *   rgb_a, rgb_b, rgb_out        device [V,3,H,W] float32
 *   depth_a, depth_b, depth_out  device [V,H,W] float32
 * All 16-byte aligned; the outputs may alias either input (element-wise).
 * For a Gaussian layer pass gs_render's depth under GS_FLAG_NORMALIZE_DEPTH. */
gs_status gs_composite_nearest(const float *rgb_a, const float *depth_a, const float *rgb_b, const float *depth_b,
                               int32_t n_views, int32_t height, int32_t width, float *rgb_out, float *depth_out,
                               void *stream);

/* A triangle mesh with per-vertex colours (device): the mesh layer of a scene
 * that mixes meshes with 3DGS assets (Sec. 3.2). */
typedef struct {
    const float *vertices;    /* [V,3] world positions */
    const float *colors;      /* [V,3] linear RGB */
    const int32_t *triangles; /* [T,3] vertex indices */
    int64_t n_vertices, n_triangles;
} gs_mesh;

/* Workspace bytes of gs_render_mesh: 96 bytes per (view, triangle of its env). */
gs_status gs_mesh_workspace_size(const gs_batch *batch, size_t *bytes);

/* The mesh pass (Sec. 3.2: the colour and depth of the mesh layer that the
 * full-screen composite merges with the Gaussian pass), rasterised by CUDA
 * kernels instead of a graphics API.  Per view, with the camera of gs_render:
 * q = R (P - C); a triangle with a vertex at q.z <= near_plane (<= 0: 0.2) is
 * culled (no clipping); a pixel is covered when its centre lies inside or on
 * the edge of the projected triangle; depth is the perspective-correct
 * view-space z, colour the perspective-correct interpolation of the vertex
 * colours; the smallest depth wins, the lower triangle index on a tie.
 * batch: env_offsets index TRIANGLES (env e's triangles [env_offsets[e],
 * env_offsets[e+1])), view_env as for gs_render (host).  Uncovered pixels get
 * bg (host float[3], NULL for black) and depth 0, so the output is a layer
 * for gs_composite_nearest.  out_rgb [V,3,H,W], out_depth [V,H,W] (device). */
gs_status gs_render_mesh(const gs_mesh *mesh, const gs_batch *batch, const gs_camera *cams, int32_t width,
                         int32_t height, const float *bg, float near_plane, void *workspace, size_t workspace_bytes,
                         float *out_rgb, float *out_depth, void *stream);

/* Skinning matrices of A avatars by forward kinematics of one joint tree
 * (Sec. 3.3.1: the per-frame SMPL-X joint matrices that drive the LBS kernel):
 *   G_0 = [R_root R_0 | t_root],  G_j = G_parent(j) [R_j | J_j - J_parent(j)],
 *   M_j = G_j [I | -J_j]   (3x4 row-major, the joint_G of gs_deform_avatars)
 *   local_rot     device [A,J,3,3]  local joint rotations R_j
 *   root          device [A,3,4]    [R_root | t_root]
 *   rest          device [J,3]      rest-pose joint positions J_j
 *   parents_host  HOST [J] int32    parent of each joint, parents[j] < j for
 *                                   j > 0 (parents[0] is ignored)
 *   out           device [A,J,3,4]
 * 1 <= J <= 64; GS_ERR_INVALID_ARG for a parent that is not below its child. */
gs_status gs_forward_kinematics(const float *local_rot, const float *root, const float *rest,
                                const int32_t *parents_host, int32_t n_avatars, int32_t n_joints, float *out,
                                void *stream);

/* Proxy capsules of posed avatars (Sec. 3.3.2: collision capsules derived from
 * the skeletal bones, posed per frame, approximate each avatar's body for the
 * navigation side).  Capsule j of avatar a is the segment from the posed
 * position of parent(j) to that of j (the root: both ends at the root, a
 * sphere) with radius radius[j]; the posed position of joint j is
 * M_j [J_j; 1], M_j its skinning matrix (the matrices gs_deform_avatars takes)
 * and J_j its rest position.
 *   joint_M       device [A,J,3,4] skinning matrices
 *   rest          device [J,3] rest joint positions
 *   parents_host  host [J] parent of each joint, parents[j] < j for j > 0
 *   radius        device [J] capsule radius per joint (metres)
 *   out_caps      device [A,J,8] (ax, ay, az, radius, bx, by, bz, 0), 16-byte aligned
 * 1 <= J <= 64; GS_ERR_INVALID_ARG for a parent that is not below its child. */
gs_status gs_avatar_capsules(const float *joint_M, const float *rest, const int32_t *parents_host,
                             const float *radius, int32_t n_avatars, int32_t n_joints, float *out_caps, void *stream);

/* The two avatar queries of Sec. 3.4: the distance to the nearest avatar
 * capsule, and whether a candidate step is blocked (the planner clips motion
 * that would enter a capsule, Sec. 3.3.2).  Query q belongs to env
 * query_env[q], whose capsules are rows [env_cap_off[e], env_cap_off[e+1]) of
 * caps; the agent is a sphere of radius agent_radius moved from p0[q] to
 * p1[q].  Per query:
 *   out_dist     [Q] float32: min over the env's capsules of |p0 - axis| - radius
 *                (negative inside; +inf for an env without capsules)
 *   out_nearest  [Q] int32: that capsule's row within the env (the lowest on
 *                ties), -1 without capsules
 *   out_tclip    [Q] float32 or NULL: the smallest t in [0, 1] at which the
 *                sphere at p0 + t (p1 - p0) touches a capsule (0 when it starts
 *                in contact), 1 when it touches none
 *   out_blocked  [Q] uint8 or NULL: 1 when the step touches a capsule
 *   caps         device [C,8] rows as gs_avatar_capsules writes them, 16-byte aligned
 *   env_cap_off  device [n_envs+1] int64; query_env device [Q] int32 (entries
 *                outside [0, n_envs) read as an env without capsules)
 *   p0, p1       device [Q,3]; p1 NULL: no step (tclip 1 unless p0 is in contact) */
gs_status gs_capsule_query(const float *caps, const int64_t *env_cap_off, int32_t n_envs, const int32_t *query_env,
                           const float *p0, const float *p1, float agent_radius, int64_t n_queries, float *out_dist,
                           int32_t *out_nearest, float *out_tclip, uint8_t *out_blocked, void *stream);

/* Joint matrices at the current simulation time (Sec. 3.3.1: the per-frame/* Joint matrices at the current simulation time (Sec. 3.3.1: the per-frame
 * matrices are interpolated at the simulation time).  For avatar a at the
 * fractional frame position t[a]: f = clamp(floor(t), 0, F-1),
 * w = clamp(t - f, 0, 1), out = (1 - w) M[f] + w M[min(f+1, F-1)] -- linear in
 * the matrices, as LBS itself blends them.
 *   frames  device [A,F,J,3,4], t device [A] float32, out device [A,J,3,4] */
gs_status gs_interpolate_joints(const float *frames, const float *t, int32_t n_avatars, int32_t n_frames,
                                int32_t n_joints, float *out, void *stream);

/* Synchronises `stream`, returns the device status of the workspace (set by
 * the last gs_render and any gs_render_backward after it) in *device_status
 * (GS_OK or GS_ERR_CAPACITY) and clears it. */
gs_status gs_get_status(void *workspace, size_t workspace_bytes, void *stream, int32_t *device_status);

/* Synchronises `stream` and copies the last call's counters. */
gs_status gs_render_stats(const void *workspace, size_t workspace_bytes, void *stream, gs_stats *out);

/* Times gs_render for each (tile_w, tile_h, batch_depth, pix_x, pix_y) candidate
 * on the given inputs (CUDA events on `stream`, `reps` timed runs after one
 * warm-up) and writes the fastest into cfg.  Candidates whose workspace does
 * not fit workspace_bytes are skipped.  Results do not depend on the
 * candidate (the footprint is per pixel), only the time does.
 * candidates: host [n_candidates][5]; best_ms receives the best time. */
gs_status gs_autotune(const gs_gaussians *g, const gs_batch *batch, const gs_camera *cams, gs_render_config *cfg,
                      void *workspace, size_t workspace_bytes, float *out_rgb, float *out_depth, float *out_T,
                      int32_t *out_ncontrib, const int32_t *candidates, int32_t n_candidates, int32_t reps,
                      float *best_ms, void *stream);

/* Device addresses of the workspace sections a gs_render call leaves behind,
 * for inspection (tests, statistics).  Host-only arithmetic on `workspace`;
 * nothing is read or written.  Layouts:
 *   records    [R][12] float: (uc, vc, hx, hy, A, B, C, opacity, red, green, blue, z)
 *              where uc = u - cx, vc = v - cy, (hx, hy) the half widths of the pixel
 *              window (pixels with |i - cx - uc| <= hx and |j - cy - vc| <= hy: the
 *              square footprint r, narrowed to where alpha can reach 1/255; r itself
 *              under GS_FLAG_COUNT_EVALS), z the FP32 depth key;
 *              R = n_records, record of (view v, local index k) at view_rec_off[v] + k
 *   vis        [ceil(R/32)] uint32 visibility bits
 *   keys       [pair_capacity] uint64 (depth bits << 32 | record), sorted per bin;
 *              after the blend, bit 31 (the record word's top bit) is set on
 *              the pairs that some pixel of their tile blended
 *   bin_start  [n_bins + 1] uint32, bin = view * tiles_per_view + ty * tiles_x + tx
 *   quarters   at 2 x 1 pixels per thread (else NULL): [pair_capacity] uint32 beside
 *              the keys; on a pair whose key has bit 31 set, byte w holds (bits 0-3)
 *              the 4 x 4 quarters of warp w's 8 x 8 block that blended it (warps in
 *              row-major order over the tile's blocks, quarter q at (4 (q & 1),
 *              4 (q >> 1)) in the block); stale elsewhere */
typedef struct {
    void *records, *vis, *keys, *bin_start, *quarters;
    int64_t n_records, pair_capacity;
    int32_t n_bins, tiles_x, tiles_y, tiles_per_view;
} gs_ws_sections;

gs_status gs_workspace_sections(const gs_render_config *cfg, const gs_batch *batch, void *workspace,
                                gs_ws_sections *out);

/* Stage profiling.  While enabled, every gs_render / gs_render_backward /
 * gs_deform_avatars(_backward) call records a CUDA event pair on its stream
 * around each kernel (not while the stream is being captured).
 * gs_profile_read synchronises on those events and returns, per stage, the
 * summed milliseconds and the number of launches since the last read, then
 * resets.  Stages: 0 setup, 1 preprocess, 2 scan, 3 scatter, 4 sort (every
 * bin, or 4096-key chunk of a larger bin), 5 merge (bins of more than 4096
 * pairs), 6 blend, 7 blend_backward, 8 preprocess_backward, 9 deform,
 * 10 deform_backward (GS_N_STAGES).  Not thread-safe. */
#define GS_N_STAGES 11
gs_status gs_profile_enable(int32_t enable);
gs_status gs_profile_read(float *stage_ms, int32_t *stage_launches);

/* Measurement of the special-function unit's exp2 throughput, the roofline
 * of the one transcendental per blend evaluation (alpha = o e^power, Sec. 3.2's
 * 3DGS blending).  Launches n_blocks CTAs of 256 threads; each thread runs
 * eight independent chains of `iters` steps x <- 2^(-x) (ex2.approx.ftz), so
 * one launch performs n_blocks * 256 * iters * 8 exp2 operations; time it with
 * events on `stream`.  out: device float[n_blocks * 256], written (the chains'
 * sums, so the work is not elided).  GS_ERR_INVALID_ARG for n_blocks < 1,
 * iters < 1 or a null out.  Asynchronous. */
gs_status gs_exp2_rate(int32_t n_blocks, int32_t iters, float *out, void *stream);

/* The CUDA error behind the last GS_ERR_CUDA (a cudaError_t value), 0 if none. */
int32_t gs_last_cuda_error(void);

int32_t gs_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GS_H */
