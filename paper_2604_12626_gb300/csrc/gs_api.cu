// gs_api.cu -- the extern "C" entry points of libgs (include/gs.h).
//
// Host side only: argument checks, the workspace layout, the batch table and
// the launch sequence.  No call allocates device memory, and only
// gs_get_status / gs_render_stats synchronise.
#include <cuda_runtime.h>

#include <cstdint>
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "gs.h"
#include "gs_internal.cuh"
#include "gs_launch.h"

namespace {

using namespace gs;

thread_local int32_t g_last_cuda_error = 0;

gs_status cuda_fail(cudaError_t e)
{
    g_last_cuda_error = (int32_t)e;
    return GS_ERR_CUDA;
}

gs_status check_launch()
{
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GS_OK : cuda_fail(e);
}

// ---------------------------------------------------------------------------
// stage profiling (events around each launch, outside stream capture)
// ---------------------------------------------------------------------------
struct ProfRec {
    int stage;
    cudaEvent_t a, b;
};
bool g_prof = false;
thread_local bool g_prof_suppress = false;
std::vector<ProfRec> g_prof_pending;
std::vector<cudaEvent_t> g_prof_pool;

cudaEvent_t prof_event()
{
    if (!g_prof_pool.empty()) {
        cudaEvent_t e = g_prof_pool.back();
        g_prof_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

bool capturing(cudaStream_t s)
{
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &st);
    return st != cudaStreamCaptureStatusNone;
}

// RAII marker: records an event before and after the launches in its scope.
struct Stage {
    int stage;
    cudaStream_t s;
    cudaEvent_t a = nullptr;
    Stage(int st, cudaStream_t str) : stage(st), s(str)
    {
        if (g_prof && !g_prof_suppress && !capturing(s)) {
            a = prof_event();
            cudaEventRecord(a, s);
        }
    }
    ~Stage()
    {
        if (a) {
            cudaEvent_t b = prof_event();
            cudaEventRecord(b, s);
            g_prof_pending.push_back(ProfRec{stage, a, b});
        }
    }
};

constexpr int kMaxDevices = 64;
std::once_flag g_once[kMaxDevices];
cudaError_t g_init_err[kMaxDevices];
int g_sms[kMaxDevices];

gs_status device_init(int *sms)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e);
    if (dev < 0 || dev >= kMaxDevices) return GS_ERR_UNSUPPORTED;
    std::call_once(g_once[dev], [dev]() {
        cudaError_t r = configure_forward_kernels();
        if (r == cudaSuccess) r = configure_backward_kernels();
        if (r == cudaSuccess) r = configure_sort_kernels();
        int n = 0;
        if (r == cudaSuccess) r = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        g_sms[dev] = n;
        g_init_err[dev] = r;
    });
    if (g_init_err[dev] != cudaSuccess) return cuda_fail(g_init_err[dev]);
    *sms = g_sms[dev];
    return GS_OK;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Plan {
    int W, H, tw, th, px, py, threads, tiles_x, tiles_y, tpv, n_bins, B, flags;
    int64_t N, R, cap;
    int64_t max_view; // most records of one view: no bin holds more pairs
    float near_plane;
    // byte offsets
    size_t o_hdr, o_tb, o_rec, o_vis, o_cnt, o_fcnt, o_start, o_cur, o_big, o_heavy, o_rel, o_keys, o_scr, o_pT, o_pL,
        o_drec, o_hseg, o_hof, o_pC, o_ckC, o_ckD, o_pq, total;
    int chunk, n_chunks;
};

gs_status make_plan(const gs_render_config *cfg, const gs_batch *b, Plan &p)
{
    if (!cfg || !b) return GS_ERR_INVALID_ARG;
    if (b->n_envs < 1 || b->n_envs > GS_MAX_ENVS || b->n_views < 1 || b->n_views > GS_MAX_VIEWS)
        return GS_ERR_INVALID_ARG;
    if (!b->env_offsets || !b->view_env) return GS_ERR_INVALID_ARG;
    if (cfg->width < 1 || cfg->height < 1 || cfg->width > 16384 || cfg->height > 16384) return GS_ERR_INVALID_ARG;
    p.W = cfg->width;
    p.H = cfg->height;
    p.tw = cfg->tile_w > 0 ? cfg->tile_w : 16;
    p.th = cfg->tile_h > 0 ? cfg->tile_h : 16;
    p.px = cfg->pix_x > 0 ? cfg->pix_x : 1;
    p.py = cfg->pix_y > 0 ? cfg->pix_y : 1;
    if (p.px > 2 || p.py > 2 || p.tw % p.px || p.th % p.py) return GS_ERR_INVALID_ARG;
    p.threads = (p.tw / p.px) * (p.th / p.py);
    if (p.threads > 1024 || p.threads % 32 != 0) return GS_ERR_INVALID_ARG;
    // 2 x 1 pixels per lane: 8 x 8 blocks per warp, at most 4 warps (the
    // per-pair quarter bits of a tile fill one 32-bit word)
    if (p.px == 2 && p.py == 1 && (p.tw % 8 || p.th % 8 || p.threads > 128)) return GS_ERR_UNSUPPORTED;
    p.B = cfg->batch_depth > 0 ? cfg->batch_depth : 256;
    if (p.B < 32 || p.B > 256 || p.B > 4 * p.threads) return GS_ERR_INVALID_ARG;
    p.flags = cfg->flags;
    p.near_plane = cfg->near_plane > 0.0f ? cfg->near_plane : 0.2f;
    p.tiles_x = (p.W + p.tw - 1) / p.tw;
    p.tiles_y = (p.H + p.th - 1) / p.th;
    p.tpv = p.tiles_x * p.tiles_y;
    const int64_t nb = (int64_t)p.tpv * b->n_views;
    if (nb > (int64_t)1 << 30) return GS_ERR_INVALID_ARG;
    p.n_bins = (int)nb;
    if (b->env_offsets[0] != 0) return GS_ERR_INVALID_ARG;
    for (int e = 0; e < b->n_envs; ++e)
        if (b->env_offsets[e + 1] < b->env_offsets[e]) return GS_ERR_INVALID_ARG;
    p.N = b->env_offsets[b->n_envs];
    int64_t R = 0, max_view = 0;
    for (int v = 0; v < b->n_views; ++v) {
        const int e = b->view_env[v];
        if (e < 0 || e >= b->n_envs) return GS_ERR_INVALID_ARG;
        R += b->env_offsets[e + 1] - b->env_offsets[e];
        max_view = std::max(max_view, b->env_offsets[e + 1] - b->env_offsets[e]);
    }
    p.max_view = max_view;
    if (R >= ((int64_t)1 << 31)) return GS_ERR_UNSUPPORTED;
    p.R = R;
    p.cap = cfg->pair_capacity > 0 ? cfg->pair_capacity : 4 * R + 65536;
    if (p.cap > ((int64_t)1 << 31) - 1) p.cap = ((int64_t)1 << 31) - 1;
    const int64_t npix = (int64_t)b->n_views * p.W * p.H;
    size_t o = 0;
    p.o_hdr = o; o = align256(o + sizeof(Header));
    p.o_tb = o; o = align256(o + sizeof(Table));
    p.o_rec = o; o = align256(o + (size_t)R * 48);
    p.o_vis = o; o = align256(o + (size_t)((R + 31) / 32 + 1) * 4);
    p.o_cnt = o; o = align256(o + (size_t)nb * 4);
    p.o_fcnt = o; o = align256(o + (size_t)nb * 4);
    p.o_start = o; o = align256(o + (size_t)(nb + 1) * 4);
    p.o_cur = o; o = align256(o + (size_t)nb * 4);
    p.o_big = o; o = align256(o + (size_t)(2 * (p.cap / kSortChunk) + 2) * 8);
    p.o_heavy = o; o = align256(o + (size_t)4096 * 4);
    p.chunk = chunk_of(p.N);
    int64_t nch = 0;
    for (int e = 0; e < b->n_envs; ++e) nch += (b->env_offsets[e + 1] - b->env_offsets[e] + p.chunk - 1) / p.chunk;
    if (nch > (int64_t)1 << 30) return GS_ERR_UNSUPPORTED;
    p.n_chunks = (int)nch;
    p.o_rel = o; o = align256(o + (size_t)p.n_chunks * kHistCap * 4);
    p.o_keys = o; o = align256(o + (size_t)p.cap * 8);
    p.o_scr = o; o = align256(o + (size_t)p.cap * 8);
    p.o_pT = o; o = align256(o + (size_t)npix * 4);
    p.o_pL = o; o = align256(o + (size_t)npix * 4);
    p.o_drec = o; o = align256(o + (size_t)R * kGradStride * 4);
    p.o_hseg = o; o = align256(o + (size_t)(kHeavyCap + 1) * 4);
    p.o_hof = o; o = align256(o + (size_t)nb * 4);
    p.o_pC = o; o = align256(o + (size_t)npix * 16);
    // checkpoint slots: every heavy bin has at most count / kSeg boundaries
    const size_t slots = (size_t)(p.cap / kSeg) + kHeavyCap + 1;
    const size_t tpx = (size_t)p.tw * p.th;
    p.o_ckC = o; o = align256(o + slots * tpx * 16);
    p.o_ckD = o; o = align256(o + slots * tpx * 4);
    p.o_pq = o; o = align256(o + (p.px == 2 && p.py == 1 ? (size_t)p.cap * 4 : 0));
    p.total = o;
    return GS_OK;
}

Ws ws_ptrs(void *base, const Plan &p)
{
    char *b = static_cast<char *>(base);
    Ws w;
    w.hdr = reinterpret_cast<Header *>(b + p.o_hdr);
    w.tb = reinterpret_cast<Table *>(b + p.o_tb);
    w.rec = reinterpret_cast<float4 *>(b + p.o_rec);
    w.vis = reinterpret_cast<uint32_t *>(b + p.o_vis);
    w.bin_count = reinterpret_cast<uint32_t *>(b + p.o_cnt);
    w.bin_start = reinterpret_cast<uint32_t *>(b + p.o_start);
    w.bin_cursor = reinterpret_cast<uint32_t *>(b + p.o_cur);
    w.big_list = reinterpret_cast<unsigned long long *>(b + p.o_big);
    w.heavy = reinterpret_cast<uint32_t *>(b + p.o_heavy);
    w.bin_fcount = reinterpret_cast<uint32_t *>(b + p.o_fcnt);
    w.rel = reinterpret_cast<uint32_t *>(b + p.o_rel);
    w.keys = reinterpret_cast<unsigned long long *>(b + p.o_keys);
    w.scratch = reinterpret_cast<unsigned long long *>(b + p.o_scr);
    w.pix_T = reinterpret_cast<float *>(b + p.o_pT);
    w.pix_last = reinterpret_cast<uint32_t *>(b + p.o_pL);
    w.d_rec = reinterpret_cast<float *>(b + p.o_drec);
    w.heavy_seg = reinterpret_cast<uint32_t *>(b + p.o_hseg);
    w.heavy_of = reinterpret_cast<int32_t *>(b + p.o_hof);
    w.pix_C = reinterpret_cast<float4 *>(b + p.o_pC);
    w.ck_C = reinterpret_cast<float4 *>(b + p.o_ckC);
    w.ck_D = reinterpret_cast<float *>(b + p.o_ckD);
    w.pq = reinterpret_cast<uint32_t *>(b + p.o_pq);
    return w;
}

void fill_table(const Plan &p, const gs_batch *b, const gs_render_config *cfg, int n_sms, Table &t)
{
    std::memset(&t, 0, sizeof(Table));
    t.n_envs = b->n_envs;
    t.n_views = b->n_views;
    t.W = p.W; t.H = p.H; t.tile_w = p.tw; t.tile_h = p.th; t.pix_x = p.px; t.pix_y = p.py;
    t.tiles_x = p.tiles_x; t.tiles_y = p.tiles_y; t.tiles_per_view = p.tpv; t.n_bins = p.n_bins;
    t.batch_depth = p.B;
    t.flags = p.flags;
    t.n_records = p.R;
    t.pair_capacity = p.cap;
    t.n_gauss = p.N;
    (void)n_sms;
    t.chunk = p.chunk;
    t.n_chunks = p.n_chunks;
    t.chunk_off[0] = 0;
    for (int e = 0; e < b->n_envs; ++e)
        t.chunk_off[e + 1] =
            t.chunk_off[e] + (int32_t)((b->env_offsets[e + 1] - b->env_offsets[e] + p.chunk - 1) / p.chunk);
    for (int k = 0; k < 3; ++k) t.bg[k] = cfg->bg[k];
    t.near_plane = p.near_plane;
    for (int e = 0; e <= b->n_envs; ++e) t.env_off[e] = b->env_offsets[e];
    for (int e = 0; e < b->n_envs; ++e)
        t.env_cov_begin[e] = b->env_cov3d_begin ? b->env_cov3d_begin[e] : b->env_offsets[e + 1];
    int64_t off = 0;
    for (int v = 0; v < b->n_views; ++v) {
        const int e = b->view_env[v];
        t.view_env[v] = e;
        t.view_rec_off[v] = off;
        off += b->env_offsets[e + 1] - b->env_offsets[e];
    }
    t.view_rec_off[b->n_views] = off;
    // views grouped by env (CSR)
    int cnt = 0;
    for (int e = 0; e < b->n_envs; ++e) {
        t.env_view_begin[e] = cnt;
        for (int v = 0; v < b->n_views; ++v)
            if (b->view_env[v] == e) t.env_views[cnt++] = v;
    }
    t.env_view_begin[b->n_envs] = cnt;
}

// Fused LBS: the avatar rows of env e are canonical rows env_av_base[e] + (g -
// env_cov_begin[e]), env after env; their count must be av->m.
static gs_status set_avatar_rows(Table &t, const gs_batch *b, const gs_avatars *av)
{
    int64_t base = 0;
    for (int e = 0; e < b->n_envs; ++e) {
        t.env_av_base[e] = base;
        base += t.env_off[e + 1] - t.env_cov_begin[e];
    }
    return base == av->m ? GS_OK : GS_ERR_INVALID_ARG;
}

// Arguments of the fused-avatar entry points (gs_render_avatars and its backward).
static gs_status check_avatars_fused(const gs_batch *batch, const gs_avatars *av, const float *joint_G)
{
    if (!batch || !av || !joint_G || !batch->env_cov3d_begin || !batch->env_offsets) return GS_ERR_INVALID_ARG;
    if (av->dest) return GS_ERR_INVALID_ARG;
    if (av->m < 0 || av->n_avatars < 1 || av->n_joints < 1 || av->n_joints > kMaxJoints) return GS_ERR_INVALID_ARG;
    if (av->m > 0 && (!av->means || !av->log_scales || !av->quats || !av->joint_ids || !av->weights || !av->avatar_of))
        return GS_ERR_INVALID_ARG;
    const void *ptrs[] = {av->means, av->log_scales, av->quats, av->joint_ids, av->weights, av->avatar_of, joint_G};
    for (const void *q : ptrs)
        if (q && !aligned16(q)) return GS_ERR_ALIGNMENT;
    if (batch->n_envs < 1 || batch->n_envs > GS_MAX_ENVS) return GS_ERR_INVALID_ARG;
    for (int e = 0; e < batch->n_envs; ++e)
        if (batch->env_cov3d_begin[e] < batch->env_offsets[e] || batch->env_cov3d_begin[e] > batch->env_offsets[e + 1])
            return GS_ERR_INVALID_ARG;
    return GS_OK;
}

gs_status check_gaussians(const gs_gaussians *g, const Plan &p, bool need_sq)
{
    if (!g || !g->means || !g->opacity_logits || !g->sh) return GS_ERR_INVALID_ARG;
    if (g->n != p.N) return GS_ERR_INVALID_ARG;
    if (g->sh_dtype < GS_SH_F32 || g->sh_dtype > GS_SH_BF16) return GS_ERR_INVALID_ARG;
    if (need_sq && (!g->log_scales || !g->quats)) return GS_ERR_INVALID_ARG;
    // rows read with 16-byte vector loads need 16-byte alignment; the rest 4
    const void *p16[] = {g->quats, g->sh};
    for (const void *q : p16)
        if (q && !aligned16(q)) return GS_ERR_ALIGNMENT;
    const void *p4[] = {g->means, g->log_scales, g->opacity_logits, g->cov3d};
    for (const void *q : p4)
        if (q && (reinterpret_cast<uintptr_t>(q) & 3u)) return GS_ERR_ALIGNMENT;
    return GS_OK;
}

gs_status enqueue_forward(const gs_gaussians *g, const gs_batch *b, const gs_camera *cams,
                          const gs_render_config *cfg, void *ws, size_t ws_bytes, float *rgb, float *depth, float *T,
                          int32_t *ncontrib, cudaStream_t s, const gs_avatars *av = nullptr,
                          const float *joint_G = nullptr)
{
    int sms = 0;
    gs_status st = device_init(&sms);
    if (st != GS_OK) return st;
    Plan p;
    st = make_plan(cfg, b, p);
    if (st != GS_OK) return st;
    st = check_gaussians(g, p, true);
    if (st != GS_OK) return st;
    if (!cams || !ws || !rgb || !depth || !T || !ncontrib) return GS_ERR_INVALID_ARG;
    if (p.threads > blend_thread_limit(p.px, p.py)) return GS_ERR_UNSUPPORTED; // CTA too large for the registers
    if (!aligned16(cams) || !aligned16(ws) || !aligned16(rgb) || !aligned16(depth) || !aligned16(T) ||
        !aligned16(ncontrib))
        return GS_ERR_ALIGNMENT;
    if (ws_bytes < p.total) return GS_ERR_WORKSPACE_TOO_SMALL;
    Table t;
    fill_table(p, b, cfg, sms, t);
    if (av && set_avatar_rows(t, b, av) != GS_OK) return GS_ERR_INVALID_ARG;
    Ws w = ws_ptrs(ws, p);
    {
        Stage st0(0, s);
        launch_setup(t, w, s);
        cudaError_t e = cudaMemsetAsync(w.vis, 0, (size_t)((p.R + 31) / 32 + 1) * 4, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(w.bin_count, 0, (size_t)p.n_bins * 4, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(w.bin_fcount, 0, (size_t)p.n_bins * 4, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(w.bin_cursor, 0, (size_t)p.n_bins * 4, s);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    // (view, tile) counters a preprocess / scatter chunk keeps in shared memory
    // (only envs whose views x tiles fit kHistCap keep counters there)
    int64_t hist_words = 0;
    for (int e = 0; e < t.n_envs; ++e) {
        const int64_t h = (int64_t)(t.env_view_begin[e + 1] - t.env_view_begin[e]) * t.tiles_per_view;
        if (h <= kHistCap) hist_words = std::max(hist_words, h);
    }
    {
        Stage st1(1, s);
        launch_preprocess(t, g, cams, w, t.n_chunks, (int)hist_words, s, av, joint_G);
    }
    {
        Stage st2(2, s);
        launch_scan(w, s);
    }
    {
        Stage st3(3, s);
        launch_scatter(cams, w, t.n_chunks, (int)hist_words, t.chunk, s);
    }
    {
        Stage st4(4, s);
        launch_sort_chunks(w, sms, s);
    }
    {
        Stage st5(5, s);
        // one pass per doubling of 4096 up to the largest possible bin
        launch_merge_passes(w, merge_passes_for_capacity(std::min(p.cap, p.max_view)), sms, s);
    }
    const bool persistent = (p.flags & GS_FLAG_PERSISTENT) != 0;
    {
        Stage st6(6, s);
        launch_blend(t, cams, w, rgb, depth, T, ncontrib, p.n_bins, p.px, p.py, p.threads, p.B, persistent,
                     (p.flags & GS_FLAG_COUNT_EVALS) != 0, sms, s);
    }
    return check_launch();
}

} // namespace

namespace gs {

gs_status record_cuda_error(cudaError_t e) { return cuda_fail(e); }

ProfileSuppress::ProfileSuppress() : prev(g_prof_suppress) { g_prof_suppress = true; }
ProfileSuppress::~ProfileSuppress() { g_prof_suppress = prev; }

} // namespace gs

extern "C" {

gs_status gs_render_workspace_size(const gs_render_config *cfg, const gs_batch *batch, size_t *bytes)
{
    if (!bytes) return GS_ERR_INVALID_ARG;
    Plan p;
    gs_status st = make_plan(cfg, batch, p);
    if (st != GS_OK) return st;
    *bytes = p.total;
    return GS_OK;
}

gs_status gs_render(const gs_gaussians *g, const gs_batch *batch, const gs_camera *cams, const gs_render_config *cfg,
                    void *workspace, size_t workspace_bytes, float *out_rgb, float *out_depth, float *out_T,
                    int32_t *out_ncontrib, void *stream)
{
    return enqueue_forward(g, batch, cams, cfg, workspace, workspace_bytes, out_rgb, out_depth, out_T, out_ncontrib,
                           static_cast<cudaStream_t>(stream));
}

// The adjoint of gs_render (av == NULL) or of gs_render_avatars: blend
// backward, then the preprocess backward, which for the fused path poses the
// avatar rows again and writes their posed mean / covariance gradients, then
// the LBS adjoint of those rows into the canonical and joint gradients.
static gs_status enqueue_backward(const gs_gaussians *g, const gs_batch *batch, const gs_camera *cams,
                                  const gs_render_config *cfg, void *workspace, size_t workspace_bytes,
                                  const float *d_rgb, const float *d_depth, float *d_means, float *d_log_scales,
                                  float *d_quats, float *d_opacity_logits, float *d_sh, float *d_cov3d,
                                  cudaStream_t s, const gs_avatars *av = nullptr, const float *joint_G = nullptr,
                                  float *d_canon_means = nullptr, float *d_canon_log_scales = nullptr,
                                  float *d_canon_quats = nullptr, float *d_joint_G = nullptr)
{
    int sms = 0;
    gs_status st = device_init(&sms);
    if (st != GS_OK) return st;
    Plan p;
    st = make_plan(cfg, batch, p);
    if (st != GS_OK) return st;
    st = check_gaussians(g, p, true);
    if (st != GS_OK) return st;
    if (cfg->flags & GS_FLAG_NORMALIZE_DEPTH) return GS_ERR_UNSUPPORTED;
    if (p.threads > blend_backward_thread_limit(p.px, p.py)) return GS_ERR_UNSUPPORTED;
    if (!cams || !workspace || !d_rgb || !d_depth || !d_means || !d_log_scales || !d_quats || !d_opacity_logits ||
        !d_sh)
        return GS_ERR_INVALID_ARG;
    const void *ptrs[] = {cams, workspace, d_rgb, d_depth, d_means, d_log_scales, d_quats, d_opacity_logits, d_sh};
    for (const void *q : ptrs)
        if (!aligned16(q)) return GS_ERR_ALIGNMENT;
    if (d_cov3d && !aligned16(d_cov3d)) return GS_ERR_ALIGNMENT;
    if (workspace_bytes < p.total) return GS_ERR_WORKSPACE_TOO_SMALL;
    Ws w = ws_ptrs(workspace, p);
    // pre-cleared arrays: the overwrite path without its clearing
    const bool precleared = (cfg->flags & GS_FLAG_GRAD_PRECLEARED) != 0;
    const bool overwrite = precleared || (cfg->flags & GS_FLAG_GRAD_OVERWRITE) != 0;
    GradOut o{d_means, d_log_scales, d_quats, d_opacity_logits, d_sh, d_cov3d};
    Table t;
    fill_table(p, batch, cfg, sms, t);
    if (av && set_avatar_rows(t, batch, av) != GS_OK) return GS_ERR_INVALID_ARG;
    {
        Stage st7(7, s);
        // the record gradient rows were zeroed by the forward (visible records
        // only); a repeated backward of the same forward clears them first
        cudaError_t e = cudaMemsetAsync(&w.hdr->queue_bwd, 0, 4, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(&w.hdr->queue_zero, 0, 4, s);
        if (e != cudaSuccess) return cuda_fail(e);
        launch_clear_record_grads(w, p.R, sms, s);
        // overwrite mode: the blend backward also sets every gradient row to
        // zero, between its tiles; the preprocess backward writes the seen rows
        launch_blend_backward(cams, w, d_rgb, d_depth, p.n_bins, p.px, p.py, p.threads, p.B, sms,
                              overwrite && !precleared ? &o : nullptr, p.N, s);
    }
    {
        Stage st8(8, s);
        launch_preprocess_backward(t, g, cams, w, o, p.n_chunks, overwrite, s, av, joint_G);
    }
    if (av && av->m > 0) {
        Stage st10(10, s);
        launch_deform_backward(av, joint_G, d_means, d_cov3d, d_canon_means, d_canon_log_scales, d_canon_quats,
                               d_joint_G, s, w.tb);
    }
    return check_launch();
}

gs_status gs_render_backward(const gs_gaussians *g, const gs_batch *batch, const gs_camera *cams,
                             const gs_render_config *cfg, void *workspace, size_t workspace_bytes,
                             const float *d_rgb, const float *d_depth, float *d_means, float *d_log_scales,
                             float *d_quats, float *d_opacity_logits, float *d_sh, float *d_cov3d, void *stream)
{
    return enqueue_backward(g, batch, cams, cfg, workspace, workspace_bytes, d_rgb, d_depth, d_means, d_log_scales,
                            d_quats, d_opacity_logits, d_sh, d_cov3d, static_cast<cudaStream_t>(stream));
}

gs_status gs_render_avatars_backward(const gs_gaussians *g, const gs_batch *batch, const gs_avatars *av,
                                     const float *joint_G, const gs_camera *cams, const gs_render_config *cfg,
                                     void *workspace, size_t workspace_bytes, const float *d_rgb,
                                     const float *d_depth, float *d_means, float *d_log_scales, float *d_quats,
                                     float *d_opacity_logits, float *d_sh, float *d_cov3d, float *d_canon_means,
                                     float *d_canon_log_scales, float *d_canon_quats, float *d_joint_G,
                                     void *stream)
{
    gs_status st = check_avatars_fused(batch, av, joint_G);
    if (st != GS_OK) return st;
    if (!d_cov3d || !d_canon_means || !d_canon_log_scales || !d_canon_quats || !d_joint_G) return GS_ERR_INVALID_ARG;
    const void *ptrs[] = {d_canon_means, d_canon_log_scales, d_canon_quats, d_joint_G};
    for (const void *q : ptrs)
        if (!aligned16(q)) return GS_ERR_ALIGNMENT;
    if (!g) return GS_ERR_INVALID_ARG;
    gs_gaussians gg = *g;
    gg.cov3d = nullptr; // the avatar rows are posed inside the preprocess backward
    return enqueue_backward(&gg, batch, cams, cfg, workspace, workspace_bytes, d_rgb, d_depth, d_means,
                            d_log_scales, d_quats, d_opacity_logits, d_sh, d_cov3d, static_cast<cudaStream_t>(stream),
                            av, joint_G, d_canon_means, d_canon_log_scales, d_canon_quats, d_joint_G);
}

gs_status gs_deform_avatars(const gs_avatars *av, const float *joint_G, float *out_means, float *out_cov3d,
                            void *stream)
{
    if (!av || !joint_G || !out_means || !out_cov3d) return GS_ERR_INVALID_ARG;
    if (av->m < 0 || av->n_avatars < 1 || av->n_joints < 1 || av->n_joints > 64) return GS_ERR_INVALID_ARG;
    if (av->m == 0) return GS_OK;
    if (!av->means || !av->log_scales || !av->quats || !av->joint_ids || !av->weights || !av->avatar_of)
        return GS_ERR_INVALID_ARG;
    const void *ptrs[] = {av->means, av->log_scales, av->quats, av->joint_ids, av->weights, av->avatar_of,
                          joint_G, out_means, out_cov3d};
    for (const void *q : ptrs)
        if (!aligned16(q)) return GS_ERR_ALIGNMENT;
    {
        Stage st9(9, static_cast<cudaStream_t>(stream));
        launch_deform(av, joint_G, out_means, out_cov3d, static_cast<cudaStream_t>(stream));
    }
    return check_launch();
}

gs_status gs_render_avatars(const gs_gaussians *g, const gs_batch *batch, const gs_avatars *av, const float *joint_G,
                            const gs_camera *cams, const gs_render_config *cfg, void *workspace,
                            size_t workspace_bytes, float *out_rgb, float *out_depth, float *out_T,
                            int32_t *out_ncontrib, void *stream)
{
    if (!g) return GS_ERR_INVALID_ARG;
    gs_status st = check_avatars_fused(batch, av, joint_G);
    if (st != GS_OK) return st;
    gs_gaussians gg = *g;
    gg.cov3d = nullptr; // the avatar rows are posed inside the preprocess
    return enqueue_forward(&gg, batch, cams, cfg, workspace, workspace_bytes, out_rgb, out_depth, out_T,
                           out_ncontrib, static_cast<cudaStream_t>(stream), av, joint_G);
}

static gs_status mesh_table(const gs_batch *b, int32_t W, int32_t H, MeshTable &t)
{
    if (!b || !b->env_offsets || !b->view_env) return GS_ERR_INVALID_ARG;
    if (b->n_envs < 1 || b->n_envs > GS_MAX_ENVS || b->n_views < 1 || b->n_views > GS_MAX_VIEWS) return GS_ERR_INVALID_ARG;
    if (W < 1 || H < 1 || W > 65535 || H > 65535) return GS_ERR_INVALID_ARG;
    std::memset(&t, 0, sizeof(t));
    t.n_views = b->n_views;
    t.W = W;
    t.H = H;
    if (b->env_offsets[0] != 0) return GS_ERR_INVALID_ARG;
    for (int e = 0; e <= b->n_envs; ++e) {
        t.env_off[e] = b->env_offsets[e];
        if (e > 0 && b->env_offsets[e] < b->env_offsets[e - 1]) return GS_ERR_INVALID_ARG;
    }
    int64_t off = 0;
    for (int v = 0; v < b->n_views; ++v) {
        const int e = b->view_env[v];
        if (e < 0 || e >= b->n_envs) return GS_ERR_INVALID_ARG;
        t.view_env[v] = e;
        t.view_rec_off[v] = off;
        off += b->env_offsets[e + 1] - b->env_offsets[e];
    }
    t.view_rec_off[b->n_views] = off;
    return GS_OK;
}

gs_status gs_mesh_workspace_size(const gs_batch *batch, size_t *bytes)
{
    if (!bytes) return GS_ERR_INVALID_ARG;
    MeshTable t;
    const gs_status st = mesh_table(batch, 1, 1, t);
    if (st != GS_OK) return st;
    *bytes = (size_t)t.view_rec_off[t.n_views] * mesh_record_bytes();
    return GS_OK;
}

gs_status gs_render_mesh(const gs_mesh *mesh, const gs_batch *batch, const gs_camera *cams, int32_t width,
                         int32_t height, const float *bg, float near_plane, void *workspace, size_t workspace_bytes,
                         float *out_rgb, float *out_depth, void *stream)
{
    if (!mesh || !cams || !out_rgb || !out_depth) return GS_ERR_INVALID_ARG;
    if (mesh->n_triangles < 0 || mesh->n_vertices < 1 || !mesh->vertices || !mesh->colors || !mesh->triangles)
        return GS_ERR_INVALID_ARG;
    MeshTable t;
    gs_status st = mesh_table(batch, width, height, t);
    if (st != GS_OK) return st;
    if (t.env_off[batch->n_envs] != mesh->n_triangles) return GS_ERR_INVALID_ARG;
    const size_t need = (size_t)t.view_rec_off[t.n_views] * mesh_record_bytes();
    if (need && (!workspace || workspace_bytes < need)) return GS_ERR_WORKSPACE_TOO_SMALL;
    if ((workspace && !aligned16(workspace)) || !aligned16(out_rgb) || !aligned16(out_depth) || !aligned16(cams))
        return GS_ERR_ALIGNMENT;
    const void *p4[] = {mesh->vertices, mesh->colors, mesh->triangles};
    for (const void *q : p4)
        if (reinterpret_cast<uintptr_t>(q) & 3u) return GS_ERR_ALIGNMENT;
    t.near_plane = near_plane > 0.f ? near_plane : 0.2f;
    for (int k = 0; k < 3; ++k) t.bg[k] = bg ? bg[k] : 0.f;
    int sms = 0;
    st = device_init(&sms);
    if (st != GS_OK) return st;
    const MeshIn in{mesh->vertices, mesh->colors, mesh->triangles, mesh->n_vertices, mesh->n_triangles};
    launch_mesh(in, cams, t, workspace, out_rgb, out_depth, static_cast<cudaStream_t>(stream));
    return check_launch();
}

gs_status gs_composite_nearest(const float *rgb_a, const float *depth_a, const float *rgb_b, const float *depth_b,
                               int32_t n_views, int32_t height, int32_t width, float *rgb_out, float *depth_out,
                               void *stream)
{
    if (!rgb_a || !depth_a || !rgb_b || !depth_b || !rgb_out || !depth_out) return GS_ERR_INVALID_ARG;
    if (n_views < 0 || height < 0 || width < 0) return GS_ERR_INVALID_ARG;
    const void *ptrs[] = {rgb_a, depth_a, rgb_b, depth_b, rgb_out, depth_out};
    for (const void *q : ptrs)
        if (!aligned16(q)) return GS_ERR_ALIGNMENT;
    if ((int64_t)n_views * height * width == 0) return GS_OK;
    int sms = 0;
    gs_status st = device_init(&sms);
    if (st != GS_OK) return st;
    launch_composite(rgb_a, depth_a, rgb_b, depth_b, rgb_out, depth_out, n_views, (int64_t)height * width, sms,
                     static_cast<cudaStream_t>(stream));
    return check_launch();
}

gs_status gs_forward_kinematics(const float *local_rot, const float *root, const float *rest,
                                const int32_t *parents_host, int32_t n_avatars, int32_t n_joints, float *out,
                                void *stream)
{
    if (!local_rot || !root || !rest || !parents_host || !out) return GS_ERR_INVALID_ARG;
    if (n_avatars < 0 || n_joints < 1 || n_joints > kMaxJoints) return GS_ERR_INVALID_ARG;
    JointTree tree;
    std::memset(&tree, 0, sizeof(tree));
    tree.n = n_joints;
    tree.parent[0] = -1;
    for (int j = 1; j < n_joints; ++j) {
        const int32_t p = parents_host[j];
        if (p < 0 || p >= j) return GS_ERR_INVALID_ARG;
        tree.parent[j] = (int8_t)p;
        tree.depth[j] = (int8_t)(tree.depth[p] + 1);
        if (tree.depth[j] > tree.max_depth) tree.max_depth = tree.depth[j];
    }
    if (n_avatars == 0) return GS_OK;
    int sms = 0;
    gs_status st = device_init(&sms);
    if (st != GS_OK) return st;
    launch_fk(local_rot, root, rest, tree, n_avatars, out, static_cast<cudaStream_t>(stream));
    return check_launch();
}

gs_status gs_avatar_capsules(const float *joint_M, const float *rest, const int32_t *parents_host,
                             const float *radius, int32_t n_avatars, int32_t n_joints, float *out_caps, void *stream)
{
    if (!joint_M || !rest || !parents_host || !radius || !out_caps) return GS_ERR_INVALID_ARG;
    if (n_avatars < 0 || n_joints < 1 || n_joints > kMaxJoints) return GS_ERR_INVALID_ARG;
    if (!aligned16(out_caps)) return GS_ERR_ALIGNMENT;
    JointTree tree;
    std::memset(&tree, 0, sizeof(tree));
    tree.n = n_joints;
    tree.parent[0] = -1;
    for (int j = 1; j < n_joints; ++j) {
        const int32_t p = parents_host[j];
        if (p < 0 || p >= j) return GS_ERR_INVALID_ARG;
        tree.parent[j] = (int8_t)p;
    }
    if (n_avatars == 0) return GS_OK;
    int sms = 0;
    gs_status st = device_init(&sms);
    if (st != GS_OK) return st;
    launch_capsules(joint_M, rest, radius, tree, n_avatars, out_caps, static_cast<cudaStream_t>(stream));
    return check_launch();
}

gs_status gs_capsule_query(const float *caps, const int64_t *env_cap_off, int32_t n_envs, const int32_t *query_env,
                           const float *p0, const float *p1, float agent_radius, int64_t n_queries, float *out_dist,
                           int32_t *out_nearest, float *out_tclip, uint8_t *out_blocked, void *stream)
{
    if (!env_cap_off || !query_env || !p0 || !out_dist || !out_nearest || n_envs < 1 || n_queries < 0)
        return GS_ERR_INVALID_ARG;
    if (!(agent_radius >= 0.0f)) return GS_ERR_INVALID_ARG;
    if (!caps || !aligned16(caps)) return caps ? GS_ERR_ALIGNMENT : GS_ERR_INVALID_ARG;
    if (n_queries == 0) return GS_OK;
    int sms = 0;
    gs_status st = device_init(&sms);
    if (st != GS_OK) return st;
    launch_capsule_query(caps, env_cap_off, n_envs, query_env, p0, p1, agent_radius, n_queries, out_dist, out_nearest,
                         out_tclip, out_blocked, static_cast<cudaStream_t>(stream));
    return check_launch();
}

gs_status gs_interpolate_joints(const float *frames, const float *t, int32_t n_avatars, int32_t n_frames,
                                int32_t n_joints, float *out, void *stream)
{
    if (!frames || !t || !out) return GS_ERR_INVALID_ARG;
    if (n_avatars < 0 || n_frames < 1 || n_joints < 1 || n_joints > kMaxJoints) return GS_ERR_INVALID_ARG;
    if (n_avatars == 0) return GS_OK;
    int sms = 0;
    gs_status st = device_init(&sms);
    if (st != GS_OK) return st;
    launch_interp(frames, t, n_avatars, n_frames, n_joints, out, sms, static_cast<cudaStream_t>(stream));
    return check_launch();
}

gs_status gs_deform_avatars_backward(const gs_avatars *av, const float *joint_G, const float *d_means,
                                     const float *d_cov3d, float *d_canon_means, float *d_canon_log_scales,
                                     float *d_canon_quats, float *d_joint_G, void *stream)
{
    if (!av || !joint_G || !d_means || !d_cov3d || !d_canon_means || !d_canon_log_scales || !d_canon_quats ||
        !d_joint_G)
        return GS_ERR_INVALID_ARG;
    if (av->m < 0 || av->n_avatars < 1 || av->n_joints < 1 || av->n_joints > 64) return GS_ERR_INVALID_ARG;
    if (av->m == 0) return GS_OK;
    const void *ptrs[] = {av->means, av->log_scales, av->quats, av->joint_ids, av->weights, av->avatar_of, joint_G,
                          d_means, d_cov3d, d_canon_means, d_canon_log_scales, d_canon_quats, d_joint_G};
    for (const void *q : ptrs)
        if (!q || !aligned16(q)) return q ? GS_ERR_ALIGNMENT : GS_ERR_INVALID_ARG;
    {
        Stage st10(10, static_cast<cudaStream_t>(stream));
        launch_deform_backward(av, joint_G, d_means, d_cov3d, d_canon_means, d_canon_log_scales, d_canon_quats,
                               d_joint_G, static_cast<cudaStream_t>(stream));
    }
    return check_launch();
}

gs_status gs_zero_gradients(int64_t n, float *d_means, float *d_log_scales, float *d_quats, float *d_opacity_logits,
                            float *d_sh, float *d_cov3d, int32_t n_ctas, void *stream)
{
    if (n < 0 || !d_means || !d_log_scales || !d_quats || !d_opacity_logits || !d_sh) return GS_ERR_INVALID_ARG;
    const void *ptrs[] = {d_means, d_log_scales, d_quats, d_opacity_logits, d_sh};
    for (const void *q : ptrs)
        if (!aligned16(q)) return GS_ERR_ALIGNMENT;
    if (d_cov3d && !aligned16(d_cov3d)) return GS_ERR_ALIGNMENT;
    if (n == 0) return GS_OK;
    int sms = 0;
    gs_status st = device_init(&sms);
    if (st != GS_OK) return st;
    GradOut o{d_means, d_log_scales, d_quats, d_opacity_logits, d_sh, d_cov3d};
    launch_zero_gradients(o, n, n_ctas > 0 ? n_ctas : (sms + 1) / 2, static_cast<cudaStream_t>(stream));
    return check_launch();
}

gs_status gs_exp2_rate(int32_t n_blocks, int32_t iters, float *out, void *stream)
{
    if (n_blocks < 1 || iters < 1 || !out) return GS_ERR_INVALID_ARG;
    launch_exp2_rate(n_blocks, iters, out, static_cast<cudaStream_t>(stream));
    return check_launch();
}

gs_status gs_get_status(void *workspace, size_t workspace_bytes, void *stream, int32_t *device_status)
{
    if (!workspace || !device_status || workspace_bytes < sizeof(Header)) return GS_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Header *h = static_cast<Header *>(workspace);
    int32_t v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, &h->status, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemsetAsync(&h->status, 0, 4, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e);
    *device_status = v;
    return GS_OK;
}

gs_status gs_render_stats(const void *workspace, size_t workspace_bytes, void *stream, gs_stats *out)
{
    if (!workspace || !out || workspace_bytes < sizeof(Header) + sizeof(Table)) return GS_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const char *b = static_cast<const char *>(workspace);
    Table t;
    cudaError_t e = cudaMemcpyAsync(&t, b + align256(sizeof(Header)), sizeof(Table), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e);
    // rebuild the plan offsets from the table
    Plan p;
    gs_render_config cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cfg.width = t.W; cfg.height = t.H; cfg.tile_w = t.tile_w; cfg.tile_h = t.tile_h;
    cfg.batch_depth = t.batch_depth; cfg.pair_capacity = t.pair_capacity; cfg.flags = t.flags;
    cfg.pix_x = t.pix_x; cfg.pix_y = t.pix_y;
    gs_batch bt;
    bt.n_envs = t.n_envs; bt.n_views = t.n_views;
    bt.env_offsets = t.env_off; bt.env_cov3d_begin = nullptr; bt.view_env = t.view_env;
    gs_status st = make_plan(&cfg, &bt, p);
    if (st != GS_OK) return st;
    if (workspace_bytes < p.total) return GS_ERR_WORKSPACE_TOO_SMALL;
    Ws w = ws_ptrs(const_cast<void *>(workspace), p);
    e = cudaMemsetAsync(&w.hdr->n_visible, 0, 4, s);
    if (e != cudaSuccess) return cuda_fail(e);
    launch_count_visible(w, (p.R + 31) / 32, s);
    Header h;
    e = cudaMemcpyAsync(&h, w.hdr, sizeof(Header), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e);
    out->n_records = t.n_records;
    out->n_visible = h.n_visible;
    out->n_pairs = h.n_pairs;
    out->max_bin = h.max_bin;
    out->status = h.status;
    out->reserved = 0;
    out->n_evaluations = (t.flags & GS_FLAG_COUNT_EVALS) ? (int64_t)h.n_evals : 0;
    out->n_covered = (t.flags & GS_FLAG_COUNT_EVALS) ? (int64_t)h.n_cov : 0;
    return GS_OK;
}

gs_status gs_autotune(const gs_gaussians *g, const gs_batch *batch, const gs_camera *cams, gs_render_config *cfg,
                      void *workspace, size_t workspace_bytes, float *out_rgb, float *out_depth, float *out_T,
                      int32_t *out_ncontrib, const int32_t *candidates, int32_t n_candidates, int32_t reps,
                      float *best_ms, void *stream)
{
    if (!cfg || !candidates || n_candidates < 1 || reps < 1) return GS_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return cuda_fail(e);
    e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(e);
    }
    gs_render_config best = *cfg;
    float best_t = -1.0f;
    gs_status result = GS_OK;
    for (int c = 0; c < n_candidates && result == GS_OK; ++c) {
        gs_render_config k = *cfg;
        k.tile_w = candidates[5 * c];
        k.tile_h = candidates[5 * c + 1];
        k.batch_depth = candidates[5 * c + 2];
        k.pix_x = candidates[5 * c + 3];
        k.pix_y = candidates[5 * c + 4];
        Plan p;
        if (make_plan(&k, batch, p) != GS_OK || p.total > workspace_bytes) continue;
        gs_status st = enqueue_forward(g, batch, cams, &k, workspace, workspace_bytes, out_rgb, out_depth, out_T,
                                       out_ncontrib, s);
        if (st != GS_OK) {
            result = st;
            break;
        }
        e = cudaEventRecord(e0, s);
        for (int r = 0; r < reps && st == GS_OK; ++r)
            st = enqueue_forward(g, batch, cams, &k, workspace, workspace_bytes, out_rgb, out_depth, out_T,
                                 out_ncontrib, s);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            result = cuda_fail(e);
            break;
        }
        if (st != GS_OK) {
            result = st;
            break;
        }
        ms /= (float)reps;
        if (best_t < 0.0f || ms < best_t) {
            best_t = ms;
            best = k;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (result != GS_OK) return result;
    if (best_t < 0.0f) return GS_ERR_WORKSPACE_TOO_SMALL;
    *cfg = best;
    if (best_ms) *best_ms = best_t;
    return GS_OK;
}

gs_status gs_workspace_sections(const gs_render_config *cfg, const gs_batch *batch, void *workspace,
                                gs_ws_sections *out)
{
    if (!workspace || !out) return GS_ERR_INVALID_ARG;
    Plan p;
    gs_status st = make_plan(cfg, batch, p);
    if (st != GS_OK) return st;
    char *b = static_cast<char *>(workspace);
    out->records = b + p.o_rec;
    out->vis = b + p.o_vis;
    out->keys = b + p.o_keys;
    out->bin_start = b + p.o_start;
    out->quarters = (p.px == 2 && p.py == 1) ? b + p.o_pq : nullptr;
    out->n_records = p.R;
    out->pair_capacity = p.cap;
    out->n_bins = p.n_bins;
    out->tiles_x = p.tiles_x;
    out->tiles_y = p.tiles_y;
    out->tiles_per_view = p.tpv;
    return GS_OK;
}

gs_status gs_profile_enable(int32_t enable)
{
    g_prof = enable != 0;
    return GS_OK;
}

gs_status gs_profile_read(float *stage_ms, int32_t *stage_launches)
{
    if (!stage_ms || !stage_launches) return GS_ERR_INVALID_ARG;
    for (int i = 0; i < GS_N_STAGES; ++i) {
        stage_ms[i] = 0.0f;
        stage_launches[i] = 0;
    }
    gs_status result = GS_OK;
    for (const ProfRec &r : g_prof_pending) {
        float ms = 0.0f;
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.a, r.b);
        if (e != cudaSuccess) result = cuda_fail(e);
        if (r.stage >= 0 && r.stage < GS_N_STAGES) {
            stage_ms[r.stage] += ms;
            stage_launches[r.stage] += 1;
        }
        g_prof_pool.push_back(r.a);
        g_prof_pool.push_back(r.b);
    }
    g_prof_pending.clear();
    return result;
}

int32_t gs_last_cuda_error(void) { return g_last_cuda_error; }

int32_t gs_version(void) { return 1; }

} // extern "C"
