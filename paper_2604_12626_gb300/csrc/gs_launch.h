// gs_launch.h -- host-side launchers of the kernels (internal to libgs).
#pragma once

#include <cuda_runtime.h>

#include "gs_internal.cuh"

namespace gs {

cudaError_t configure_forward_kernels();
cudaError_t configure_backward_kernels();

void launch_setup(const Table &tb, const Ws &w, cudaStream_t s);
// hist_words: (view, tile) counters a chunk keeps in shared memory, at least
// min(kHistCap, most views of an env x tiles per view)
void launch_preprocess(const Table &tb, const gs_gaussians *g, const gs_camera *cams, const Ws &w, int n_chunks,
                       int hist_words, cudaStream_t s, const gs_avatars *av = nullptr, const float *joint_G = nullptr);
void launch_scan(const Ws &w, cudaStream_t s);
// chunk: Gaussians per chunk (the record list it keeps in shared memory)
void launch_scatter(const gs_camera *cams, const Ws &w, int n_chunks, int hist_words, int chunk, cudaStream_t s);
cudaError_t configure_sort_kernels();
void launch_exp2_rate(int n_blocks, int iters, float *out, cudaStream_t s);
int merge_passes_for_capacity(int64_t pair_capacity);
void launch_sort_chunks(const Ws &w, int n_sms, cudaStream_t s);
void launch_merge_passes(const Ws &w, int n_passes, int n_sms, cudaStream_t s);
// count: the GS_FLAG_COUNT_EVALS variant (evaluation counters in the header)
void launch_blend(const Table &tb, const gs_camera *cams, const Ws &w, float *rgb, float *depth, float *T,
                  int32_t *ncontrib, int n_bins, int px, int py, int threads, int batch_depth, bool persistent,
                  bool count, int n_sms, cudaStream_t s);
// Largest CTA (threads) the blend kernels of this pixels-per-thread variant can
// launch with (register-limited), forward and backward.
int blend_thread_limit(int px, int py);
int blend_backward_thread_limit(int px, int py);
void launch_count_visible(const Ws &w, int64_t n_words, cudaStream_t s);

struct GradOut {
    float *means, *log_scales, *quats, *ologits, *sh, *cov3d;
};

constexpr int kZeroArrays = 6;
struct ZeroWork { // gradient arrays to clear and the first clearing item of each
    float *p[kZeroArrays];
    int64_t n[kZeroArrays];
    uint32_t first[kZeroArrays];
    uint32_t total;
    uint32_t clear_ctas; // CTAs that clear before they take tiles (one per SM)
};
void launch_clear_record_grads(const Ws &w, int64_t n_records, int n_sms, cudaStream_t s);
// gs_zero_gradients: the gradient arrays of n Gaussians set to zero by n_ctas CTAs
void launch_zero_gradients(const GradOut &o, int64_t n, int n_ctas, cudaStream_t s);
// clear: in overwrite mode the gradient arrays (n Gaussians) the blend backward
// sets to zero between its tiles, else nullptr
void launch_blend_backward(const gs_camera *cams, const Ws &w, const float *d_rgb, const float *d_depth, int n_bins,
                           int px, int py, int threads, int batch_depth, int n_sms, const GradOut *clear, int64_t n,
                           cudaStream_t s);
// av, joint_G: the fused path (gs_render_avatars_backward) poses the avatar
// rows again by LBS and writes their posed mean / covariance gradients
void launch_preprocess_backward(const Table &tb, const gs_gaussians *g, const gs_camera *cams, const Ws &w,
                                const GradOut &o, int n_chunks, bool overwrite, cudaStream_t s,
                                const gs_avatars *av = nullptr, const float *joint_G = nullptr);

void launch_deform(const gs_avatars *av, const float *G, float *out_means, float *out_cov, cudaStream_t s);
// rows: the batch layout (device table) that maps canonical avatar rows to
// batch rows when av->dest is NULL (gs_render_avatars_backward), else NULL
void launch_deform_backward(const gs_avatars *av, const float *G, const float *d_means, const float *d_cov,
                            float *d_cm, float *d_cls, float *d_cq, float *d_G, cudaStream_t s,
                            const Table *rows = nullptr);

void launch_composite(const float *rgb_a, const float *depth_a, const float *rgb_b, const float *depth_b,
                      float *rgb_out, float *depth_out, int64_t n_views, int64_t hw, int n_sms, cudaStream_t s);
void launch_fk(const float *local_rot, const float *root, const float *rest, const JointTree &tree, int n_avatars,
               float *out, cudaStream_t s);
void launch_interp(const float *frames, const float *t, int n_avatars, int n_frames, int n_joints, float *out,
                   int n_sms, cudaStream_t s);

void launch_capsules(const float *M, const float *rest, const float *radius, const JointTree &tree, int n_avatars,
                     float *out, cudaStream_t s);
void launch_capsule_query(const float *caps, const int64_t *cap_off, int n_envs, const int32_t *query_env,
                          const float *p0, const float *p1, float agent_r, int64_t n_q, float *out_dist,
                          int32_t *out_near, float *out_t, uint8_t *out_blk, cudaStream_t s);

size_t mesh_record_bytes();
void launch_mesh(const MeshIn &in, const gs_camera *cams, const MeshTable &t, void *rec, float *rgb, float *depth,
                 cudaStream_t s);

// Records a CUDA error for gs_last_cuda_error and returns GS_ERR_CUDA.
gs_status record_cuda_error(cudaError_t e);

// While alive on this thread, the calls made by this thread record no stage
// profiling events.
struct ProfileSuppress {
    ProfileSuppress();
    ~ProfileSuppress();
    bool prev;
};

} // namespace gs
