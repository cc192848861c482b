// gs_sort.cu -- per-bin depth sort of the (view, tile) pair lists (sm_103a).
//
// After the scatter every bin [bin_start[b], bin_start[b+1]) of `keys` holds
// its pairs in arbitrary order, one 64-bit key each:
//   key = FP32 depth bits << 32 | record index.
// The blend needs them in key order (depth, then record index: the order a
// stable sort of the keys emitted in record order gives, Sec. 3.2's
// front-to-back compositing).  Keys are unique inside a bin.
//
//   sort_chunks_kernel  one CTA sorts up to 4096 keys: a bin of <= 4096 pairs,
//                       or one 4096-long chunk of a larger bin.  LSD radix sort
//                       in shared memory over the depth bits minus the chunk's
//                       smallest (3 passes of 9 bits when they span less than
//                       2^27, else 4 passes of 8 bits over the depth bits),
//                       ranks from warp match masks; keys sharing a depth are
//                       ordered by record index on the way out.
//   sort_small_kernel   bins of 2 .. 512 pairs, one warp each: the same passes
//                       with the keys in registers, warp-level counters and
//                       ranks, no CTA barrier.
//   merge_pass_kernel   bins of more than 4096 pairs: pass p merges sorted runs
//                       of 4096 << p; each CTA writes 4096 outputs, located by
//                       a merge-path search.  Chunk sorts write to keys or to
//                       scratch so that the last pass of every bin ends in keys.
#include "gs_internal.cuh"
#include "gs_launch.h"

namespace gs {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kRadixMax = 512; // digits of up to 9 bits
constexpr int kSmallSort = 512; // bins up to this many pairs: one warp each (sort_small_kernel)

struct SortSmem {
    unsigned long long keys[kSortChunk];
    uint32_t cnt[kSortWarps][kRadixMax];
    uint32_t wsum[kSortWarps];
    uint32_t item, dmin, dmax;
};

__device__ __forceinline__ int ceil_log2(uint32_t x)
{
    return x <= 1u ? 0 : 32 - __clz(x - 1u);
}

// Buffer a bin's keys live in before merge pass p (p = passes: after all).
__device__ __forceinline__ unsigned long long *sort_buf(const Ws &w, int passes, int p)
{
    return ((passes - p) & 1) ? w.scratch : w.keys;
}

// Digit of a key for one LSD pass.  BITS == 8: bits [shift, shift + 8) of the
// 64-bit key.  BITS == 9: bits [shift, shift + 9) of the depth bits minus the
// chunk's smallest (`sub`), capped at kDepthCap so that padding keys sort last.
constexpr uint32_t kDepthCap = (1u << 27) - 1u;

template <int BITS>
__device__ __forceinline__ uint32_t key_digit(unsigned long long key, int shift, uint32_t sub)
{
    if (BITS == 8) return (uint32_t)(key >> shift) & 0xffu;
    return (min((uint32_t)(key >> 32) - sub, kDepthCap) >> shift) & ((1u << BITS) - 1u);
}

// One stable LSD pass over one digit.  Layout: warp w holds positions
// [w 32K, (w+1) 32K), position w 32K + r 32 + lane in register k[r], so
// ranking in (warp, round, lane) order is position order.  On return k[] and
// sm.keys hold the keys in the new order.
template <int K, int BITS>
__device__ __forceinline__ void radix_pass(unsigned long long (&k)[K], int shift, uint32_t sub, SortSmem &sm)
{
    constexpr int R = 1 << BITS, DPT = R / kSortThreads; // digits per thread in the scan
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int i = threadIdx.x; i < kSortWarps * R; i += kSortThreads) sm.cnt[i / R][i % R] = 0u;
    __syncthreads();
    uint32_t loff[(K + 1) / 2]; // ranks < 4096, two per register
#pragma unroll
    for (int r = 0; r < (K + 1) / 2; ++r) loff[r] = 0u;
#pragma unroll
    for (int r = 0; r < K; ++r) {
        const uint32_t d = key_digit<BITS>(k[r], shift, sub);
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int leader = __ffs(peers) - 1;
        uint32_t base = 0;
        if (lane == leader) {
            base = sm.cnt[warp][d];
            sm.cnt[warp][d] = base + (uint32_t)__popc(peers);
        }
        base = __shfl_sync(0xffffffffu, base, leader);
        loff[r >> 1] |= (base + (uint32_t)__popc(peers & lt)) << (16 * (r & 1));
    }
    __syncthreads();
    {
        // exclusive offsets, digit-major then warp: thread t owns digits
        // t DPT .. t DPT + DPT - 1
        uint32_t all = 0;
#pragma unroll
        for (int j = 0; j < DPT; ++j)
#pragma unroll
            for (int q = 0; q < kSortWarps; ++q) all += sm.cnt[q][threadIdx.x * DPT + j];
        uint32_t incl = all;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += v;
        }
        if (lane == 31) sm.wsum[warp] = incl;
        __syncthreads();
        uint32_t run = incl - all;
        for (int q = 0; q < warp; ++q) run += sm.wsum[q];
#pragma unroll
        for (int j = 0; j < DPT; ++j) {
#pragma unroll
            for (int q = 0; q < kSortWarps; ++q) {
                const uint32_t cq = sm.cnt[q][threadIdx.x * DPT + j];
                sm.cnt[q][threadIdx.x * DPT + j] = run;
                run += cq;
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < K; ++r) {
        const uint32_t d = key_digit<BITS>(k[r], shift, sub);
        sm.keys[sm.cnt[warp][d] + ((loff[r >> 1] >> (16 * (r & 1))) & 0xffffu)] = k[r];
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < K; ++r) k[r] = sm.keys[warp * 32 * K + r * 32 + lane];
    __syncthreads();
}

// Bounds [s, e] of the run of keys sharing `key`'s depth around position pos
// of the depth-sorted sm.keys[0..n); false if it is longer than kMaxRun.
constexpr uint32_t kMaxRun = 32;

__device__ __forceinline__ bool run_bounds(const unsigned long long *keys, uint32_t pos, uint32_t n, uint32_t hi,
                                           uint32_t &s, uint32_t &e)
{
    s = pos;
    e = pos;
    while (s > 0 && (uint32_t)(keys[s - 1] >> 32) == hi) {
        --s;
        if (pos - s >= kMaxRun) return false;
    }
    while (e + 1 < n && (uint32_t)(keys[e + 1] >> 32) == hi) {
        ++e;
        if (e - s >= kMaxRun) return false;
    }
    return true;
}

__device__ __forceinline__ bool depth_run(const SortSmem &sm, uint32_t pos, uint32_t n, uint32_t hi, uint32_t &s,
                                          uint32_t &e)
{
    return run_bounds(sm.keys, pos, n, hi, s, e);
}

// Sorts src[0..n) (n <= 256 K) into dst[0..n) (dst may equal src): three or four
// passes over the depth bits; keys sharing a depth are then ordered by record index
// while they are written out, or -- if some run of equal depths is longer than
// kMaxRun -- the whole 64-bit key is sorted again with eight passes.
template <int K>
__device__ void radix_sort_chunk(const unsigned long long *src, unsigned long long *dst, uint32_t n, SortSmem &sm)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned long long k[K];
#pragma unroll
    for (int r = 0; r < K; ++r) {
        const uint32_t pos = (uint32_t)(warp * 32 * K + r * 32 + lane);
        k[r] = pos < n ? src[pos] : ~0ull; // padding sorts last (no real depth has all bits set)
    }
    // the depths of a chunk usually span less than 2^27 - 1 as FP32 bit patterns
    // (0.2 m .. 100 m does): then three 9-bit passes over (depth - smallest)
    // order them, otherwise four 8-bit passes over the depth bits
    if (threadIdx.x == 0) {
        sm.dmin = 0xffffffffu;
        sm.dmax = 0u;
    }
    __syncthreads();
    {
        uint32_t lo = 0xffffffffu, hi = 0u;
#pragma unroll
        for (int r = 0; r < K; ++r) {
            const uint32_t pos = (uint32_t)(warp * 32 * K + r * 32 + lane);
            if (pos < n) {
                lo = min(lo, (uint32_t)(k[r] >> 32));
                hi = max(hi, (uint32_t)(k[r] >> 32));
            }
        }
        lo = __reduce_min_sync(0xffffffffu, lo);
        hi = __reduce_max_sync(0xffffffffu, hi);
        if (lane == 0) {
            atomicMin(&sm.dmin, lo);
            atomicMax(&sm.dmax, hi);
        }
    }
    __syncthreads();
    const uint32_t dmin = sm.dmin, dmax = sm.dmax;
    if (dmax - dmin < kDepthCap) {
#pragma unroll 1
        for (int pass = 0; pass < 3; ++pass) radix_pass<K, 9>(k, 9 * pass, dmin, sm);
    } else {
#pragma unroll 1
        for (int pass = 0; pass < 4; ++pass) radix_pass<K, 8>(k, 32 + 8 * pass, 0u, sm);
    }
    bool long_run = false;
#pragma unroll
    for (int r = 0; r < K; ++r) {
        const uint32_t pos = (uint32_t)(warp * 32 * K + r * 32 + lane);
        const uint32_t hi = (uint32_t)(k[r] >> 32);
        if (pos > 0 && pos < n && (uint32_t)(sm.keys[pos - 1] >> 32) == hi) {
            uint32_t s, e;
            long_run |= !depth_run(sm, pos, n, hi, s, e);
        }
    }
    if (__syncthreads_or(long_run)) {
#pragma unroll 1
        for (int pass = 0; pass < 8; ++pass) radix_pass<K, 8>(k, 8 * pass, 0u, sm);
#pragma unroll
        for (int r = 0; r < K; ++r) {
            const uint32_t pos = (uint32_t)(warp * 32 * K + r * 32 + lane);
            if (pos < n) dst[pos] = k[r];
        }
        return;
    }
#pragma unroll
    for (int r = 0; r < K; ++r) {
        const uint32_t pos = (uint32_t)(warp * 32 * K + r * 32 + lane);
        if (pos >= n) continue;
        const unsigned long long key = k[r];
        const uint32_t hi = (uint32_t)(key >> 32);
        uint32_t at = pos;
        if ((pos > 0 && (uint32_t)(sm.keys[pos - 1] >> 32) == hi) ||
            (pos + 1 < n && (uint32_t)(sm.keys[pos + 1] >> 32) == hi)) {
            uint32_t s, e;
            depth_run(sm, pos, n, hi, s, e);
            uint32_t rank = 0;
            for (uint32_t j = s; j <= e; ++j) rank += (uint32_t)sm.keys[j] < (uint32_t)key;
            at = s + rank;
        }
        dst[at] = key;
    }
}

__device__ __forceinline__ void sort_dispatch(const unsigned long long *src, unsigned long long *dst, uint32_t n,
                                              SortSmem &sm)
{
    if (n <= 256u) radix_sort_chunk<1>(src, dst, n, sm);
    else if (n <= 512u) radix_sort_chunk<2>(src, dst, n, sm);
    else if (n <= 1024u) radix_sort_chunk<4>(src, dst, n, sm);
    else if (n <= 2048u) radix_sort_chunk<8>(src, dst, n, sm);
    else radix_sort_chunk<16>(src, dst, n, sm);
}

// Work items: the 4096-key chunks of the large bins first (their merges wait on
// them), then every bin; a bin of > 4096 pairs or <= 1 pair is skipped there.
__global__ void __launch_bounds__(kSortThreads, 3) sort_chunks_kernel(Ws w)
{
    extern __shared__ __align__(16) unsigned char smem_sort[];
    SortSmem &sm = *reinterpret_cast<SortSmem *>(smem_sort);
    const uint32_t n_big = w.hdr->n_big;
    const uint32_t n_items = n_big + (uint32_t)w.tb->n_bins;
    for (;;) {
        if (threadIdx.x == 0) sm.item = atomicAdd(&w.hdr->big_queue, 1u);
        __syncthreads();
        const uint32_t item = sm.item;
        __syncthreads();
        if (item >= n_items) break;
        uint32_t start, n;
        if (item < n_big) {
            const unsigned long long e = w.big_list[item];
            const int bin = (int)(e >> 32);
            const uint32_t t = (uint32_t)e;
            bin_range(w, bin, start, n);
            const int passes = ceil_log2((n + kSortChunk - 1) / kSortChunk);
            const uint32_t c0 = t * (uint32_t)kSortChunk;
            const uint32_t cn = min((uint32_t)kSortChunk, n - c0);
            sort_dispatch(w.keys + start + c0, sort_buf(w, passes, 0) + start + c0, cn, sm);
        } else {
            bin_range(w, (int)(item - n_big), start, n);
            if (n <= (uint32_t)kSmallSort || n > (uint32_t)kSortChunk) continue; // small bins: sort_small_kernel
            sort_dispatch(w.keys + start, w.keys + start, n, sm);
        }
    }
}

// ---------------------------------------------------------------------------
// Bins of at most kSmallSort pairs: one warp each.  The warp holds the bin's
// keys in registers (K per lane, position r 32 + lane in k[r]) and runs the
// same LSD passes with warp-level counting (shared-memory counters), an
// exclusive scan and stable ranking from match masks, scattering into its own
// shared-memory buffer and reading back in position order -- no CTA barrier.
// Equal depths are ordered by record index on the way out, as in the CTA
// sort; a run of equal depths longer than kMaxRun sorts the whole 64-bit key.
// ---------------------------------------------------------------------------
constexpr int kSmallWarps = 8;

struct SmallSortSmem {
    unsigned long long keys[kSmallWarps][kSmallSort];
    uint32_t cnt[kSmallWarps][kRadixMax];
};

template <int K, int BITS>
__device__ __forceinline__ void warp_radix_pass(unsigned long long (&k)[K], uint32_t n, int shift, uint32_t sub,
                                                unsigned long long *buf, uint32_t *cnt)
{
    constexpr int R = 1 << BITS, PER = R / 32;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int j = 0; j < PER; ++j) cnt[j * 32 + lane] = 0u;
    __syncwarp();
#pragma unroll
    for (int r = 0; r < K; ++r)
        if ((uint32_t)(r * 32 + lane) < n) atomicAdd(cnt + key_digit<BITS>(k[r], shift, sub), 1u);
    __syncwarp();
    {
        // exclusive scan: lane owns digits lane PER .. lane PER + PER - 1
        uint32_t v[PER], sum = 0;
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            v[j] = cnt[lane * PER + j];
            sum += v[j];
        }
        uint32_t incl = sum;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += u;
        }
        uint32_t run = incl - sum;
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            cnt[lane * PER + j] = run;
            run += v[j];
        }
    }
    __syncwarp();
#pragma unroll
    for (int r = 0; r < K; ++r) {
        const bool valid = (uint32_t)(r * 32 + lane) < n;
        const uint32_t d = valid ? key_digit<BITS>(k[r], shift, sub) : 0xffffffffu;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int leader = __ffs(peers) - 1;
        uint32_t base = 0;
        if (valid && lane == leader) {
            base = cnt[d];
            cnt[d] = base + (uint32_t)__popc(peers);
        }
        base = __shfl_sync(0xffffffffu, base, leader);
        if (valid) buf[base + (uint32_t)__popc(peers & lt)] = k[r];
    }
    __syncwarp();
#pragma unroll
    for (int r = 0; r < K; ++r)
        if ((uint32_t)(r * 32 + lane) < n) k[r] = buf[r * 32 + lane];
    __syncwarp();
}

// Sorts keys[0..n) of one bin in place (n <= 32 K) with one warp.
template <int K>
__device__ void warp_sort_bin(unsigned long long *keys, uint32_t n, unsigned long long *buf, uint32_t *cnt)
{
    const int lane = threadIdx.x & 31;
    unsigned long long k[K];
    uint32_t lo = 0xffffffffu, hi = 0u;
#pragma unroll
    for (int r = 0; r < K; ++r) {
        const uint32_t pos = (uint32_t)(r * 32 + lane);
        k[r] = pos < n ? keys[pos] : ~0ull;
        if (pos < n) {
            lo = min(lo, (uint32_t)(k[r] >> 32));
            hi = max(hi, (uint32_t)(k[r] >> 32));
        }
    }
    lo = __reduce_min_sync(0xffffffffu, lo);
    hi = __reduce_max_sync(0xffffffffu, hi);
    if (hi - lo < kDepthCap) {
#pragma unroll 1
        for (int pass = 0; pass < 3; ++pass) warp_radix_pass<K, 9>(k, n, 9 * pass, lo, buf, cnt);
    } else {
#pragma unroll 1
        for (int pass = 0; pass < 4; ++pass) warp_radix_pass<K, 8>(k, n, 32 + 8 * pass, 0u, buf, cnt);
    }
    // buf[0..n) now holds the keys in depth order; runs of equal depths are
    // ordered by record index while they are written out
    bool long_run = false;
#pragma unroll
    for (int r = 0; r < K; ++r) {
        const uint32_t pos = (uint32_t)(r * 32 + lane);
        const uint32_t h = (uint32_t)(k[r] >> 32);
        if (pos > 0 && pos < n && (uint32_t)(buf[pos - 1] >> 32) == h) {
            uint32_t sp, ep;
            long_run |= !run_bounds(buf, pos, n, h, sp, ep);
        }
    }
    if (__any_sync(0xffffffffu, long_run)) {
#pragma unroll 1
        for (int pass = 0; pass < 8; ++pass) warp_radix_pass<K, 8>(k, n, 8 * pass, 0u, buf, cnt);
#pragma unroll
        for (int r = 0; r < K; ++r)
            if ((uint32_t)(r * 32 + lane) < n) keys[r * 32 + lane] = k[r];
        return;
    }
#pragma unroll
    for (int r = 0; r < K; ++r) {
        const uint32_t pos = (uint32_t)(r * 32 + lane);
        if (pos >= n) continue;
        const unsigned long long key = k[r];
        const uint32_t h = (uint32_t)(key >> 32);
        uint32_t at = pos;
        if ((pos > 0 && (uint32_t)(buf[pos - 1] >> 32) == h) || (pos + 1 < n && (uint32_t)(buf[pos + 1] >> 32) == h)) {
            uint32_t sp, ep;
            run_bounds(buf, pos, n, h, sp, ep); // a run of at most kMaxRun keys (checked above)
            uint32_t rank = 0;
            for (uint32_t j = sp; j <= ep; ++j) rank += (uint32_t)buf[j] < (uint32_t)key;
            at = sp + rank;
        }
        keys[at] = key;
    }
}

// Every bin of 2 .. kSmallSort pairs, a warp per bin (bins taken four at a time).
__global__ void __launch_bounds__(kSmallWarps * 32) sort_small_kernel(Ws w)
{
    extern __shared__ __align__(16) unsigned char smem_small[];
    SmallSortSmem &sm = *reinterpret_cast<SmallSortSmem *>(smem_small);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned long long *buf = sm.keys[warp];
    uint32_t *cnt = sm.cnt[warp];
    const uint32_t n_bins = (uint32_t)w.tb->n_bins;
    for (;;) {
        uint32_t b0 = 0;
        if (lane == 0) b0 = atomicAdd(&w.hdr->small_queue, 4u);
        b0 = __shfl_sync(0xffffffffu, b0, 0);
        if (b0 >= n_bins) break;
        for (uint32_t bin = b0; bin < min(b0 + 4u, n_bins); ++bin) {
            uint32_t start, n;
            bin_range(w, (int)bin, start, n);
            if (n <= 1u || n > (uint32_t)kSmallSort) continue;
            unsigned long long *keys = w.keys + start;
            if (n <= 128u) warp_sort_bin<4>(keys, n, buf, cnt);
            else if (n <= 256u) warp_sort_bin<8>(keys, n, buf, cnt);
            else warp_sort_bin<16>(keys, n, buf, cnt);
        }
    }
}

// Merge path with one warp: the number of elements of a[0..na) among the
// first d outputs of merge(a, b) (keys unique).  Each round probes 32 points
// of the remaining range; the first probe whose a-key is not below the
// opposite b-key bounds the answer from above.  About log32 of the range
// dependent global loads instead of log2.
__device__ __forceinline__ uint32_t merge_path_warp(const unsigned long long *a, uint32_t na,
                                                    const unsigned long long *b, uint32_t nb, uint32_t d)
{
    const int lane = threadIdx.x & 31;
    uint32_t lo = d > nb ? d - nb : 0u, hi = min(d, na);
    while (hi > lo) {
        const uint32_t len = hi - lo;
        const uint32_t p = lo + (uint32_t)(((unsigned long long)lane * len) >> 5);
        const bool pr = p < hi && a[p] < b[d - 1 - p];
        const int k = __popc(__ballot_sync(0xffffffffu, pr));
        const uint32_t p_prev = __shfl_sync(0xffffffffu, p, k > 0 ? k - 1 : 0);
        const uint32_t p_next = __shfl_sync(0xffffffffu, p, k < 32 ? k : 31);
        const uint32_t nlo = k > 0 ? p_prev + 1 : lo;
        const uint32_t nhi = k < 32 ? min(p_next, hi) : hi;
        lo = nlo;
        hi = max(nhi, nlo);
    }
    return lo;
}

struct MergeSmem {
    unsigned long long in[kSortChunk];
    unsigned long long out[kSortChunk];
    uint32_t split[2];
};

// One merge pass over all large bins: item (bin, t) writes outputs
// [4096 t, 4096 (t + 1)) of the merge of the two runs of width 4096 << pass
// that contain them.
__global__ void __launch_bounds__(kSortThreads) merge_pass_kernel(Ws w, int pass)
{
    extern __shared__ __align__(16) unsigned char smem_merge[];
    MergeSmem &sm = *reinterpret_cast<MergeSmem *>(smem_merge);
    if (pass >= (int)w.hdr->max_pass) return;
    const uint32_t n_big = w.hdr->n_big;
    for (uint32_t it = blockIdx.x; it < n_big; it += gridDim.x) {
        const unsigned long long e = w.big_list[it];
        const int bin = (int)(e >> 32);
        const uint32_t t = (uint32_t)e;
        uint32_t start, n;
        bin_range(w, bin, start, n);
        const int passes = ceil_log2((n + kSortChunk - 1) / kSortChunk);
        if (pass >= passes) continue;
        const unsigned long long *src = sort_buf(w, passes, pass) + start;
        unsigned long long *dst = sort_buf(w, passes, pass + 1) + start;
        const uint32_t width = (uint32_t)kSortChunk << pass;
        const uint32_t o0 = t * (uint32_t)kSortChunk, o1 = min(n, o0 + (uint32_t)kSortChunk);
        const uint32_t a0 = (o0 / (2 * width)) * (2 * width);
        const uint32_t a1 = min(a0 + width, n), b1 = min(a1 + width, n);
        const uint32_t na = a1 - a0, nb = b1 - a1;
        if (threadIdx.x < 64) { // warp 0: diagonal o0, warp 1: diagonal o1
            const int wq = threadIdx.x >> 5;
            const uint32_t sp = merge_path_warp(src + a0, na, src + a1, nb, (wq == 0 ? o0 : o1) - a0);
            if ((threadIdx.x & 31) == 0) sm.split[wq] = sp;
        }
        __syncthreads();
        const uint32_t i0 = sm.split[0], i1 = sm.split[1];
        const uint32_t j0 = (o0 - a0) - i0, j1 = (o1 - a0) - i1;
        const uint32_t la = i1 - i0, lb = j1 - j0, tot = la + lb;
        for (uint32_t q = threadIdx.x; q < la; q += kSortThreads) sm.in[q] = src[a0 + i0 + q];
        for (uint32_t q = threadIdx.x; q < lb; q += kSortThreads) sm.in[la + q] = src[a1 + j0 + q];
        __syncthreads();
        {
            const unsigned long long *A = sm.in, *B = sm.in + la;
            constexpr uint32_t per = kSortChunk / kSortThreads;
            const uint32_t d0 = min(tot, threadIdx.x * per), d1 = min(tot, d0 + per);
            if (d0 < d1) {
                uint32_t lo = d0 > lb ? d0 - lb : 0u, hi = min(d0, la);
                while (lo < hi) {
                    const uint32_t mid = (lo + hi) >> 1;
                    if (A[mid] < B[d0 - 1 - mid]) lo = mid + 1;
                    else hi = mid;
                }
                uint32_t i = lo, j = d0 - lo;
                for (uint32_t o = d0; o < d1; ++o) {
                    const bool take_a = j >= lb || (i < la && A[i] < B[j]);
                    sm.out[o] = take_a ? A[i++] : B[j++];
                }
            }
        }
        __syncthreads();
        for (uint32_t q = threadIdx.x; q < tot; q += kSortThreads) dst[o0 + q] = sm.out[q];
        __syncthreads();
    }
}

static int g_sort_occ = 1, g_merge_occ = 1, g_small_occ = 1; // resident CTAs per SM

cudaError_t configure_sort_kernels()
{
    cudaError_t e = cudaFuncSetAttribute(sort_chunks_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(SortSmem));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(merge_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(MergeSmem));
    int nb = 0;
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sort_chunks_kernel, kSortThreads, (int)sizeof(SortSmem));
    if (e == cudaSuccess && nb > 0) g_sort_occ = nb;
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, merge_pass_kernel, kSortThreads, (int)sizeof(MergeSmem));
    if (e == cudaSuccess && nb > 0) g_merge_occ = nb;
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(sort_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(SmallSortSmem));
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sort_small_kernel, kSmallWarps * 32,
                                                          (int)sizeof(SmallSortSmem));
    if (e == cudaSuccess && nb > 0) g_small_occ = nb;
    return e;
}

int merge_passes_for_capacity(int64_t pair_capacity)
{
    const int64_t chunks = (pair_capacity + kSortChunk - 1) / kSortChunk;
    int p = 0;
    while (((int64_t)1 << p) < chunks) ++p;
    return p;
}

void launch_sort_chunks(const Ws &w, int n_sms, cudaStream_t s)
{
    sort_chunks_kernel<<<n_sms * g_sort_occ, kSortThreads, sizeof(SortSmem), s>>>(w);
    sort_small_kernel<<<n_sms * g_small_occ, kSmallWarps * 32, sizeof(SmallSortSmem), s>>>(w);
}

void launch_merge_passes(const Ws &w, int n_passes, int n_sms, cudaStream_t s)
{
    for (int p = 0; p < n_passes; ++p)
        merge_pass_kernel<<<n_sms * g_merge_occ, kSortThreads, sizeof(MergeSmem), s>>>(w, p);
}

} // namespace gs
