// sort.cu -- device-wide scans, stream compaction, pair emission and a
// stable LSD radix sort of (u32 key, u32 value) pairs, all with the element
// count read from device memory so that no host round trip is needed.
//
// Role in the method: the camera-space depth order of the Gaussians
// (Sec. 3.1) within every tile of the tile-based rasterizer.
// The sort is done in two stages:
//   1. the visible (view, Gaussian) items are sorted by the float32 bits of
//      their camera depth (4 digit passes over M items; the items start in
//      gid order and the sort is stable, so equal depths keep gid order);
//   2. each item, in that depth order, emits one (tile id, depth position)
//      pair per tile its footprint ellipse meets, and the K pairs are
//      sorted stably by tile id
//      alone (ceil(log2 tiles) bits, 2-3 passes).
// The result is ordered by (tile, depth, gid) -- the per-tile front-to-back
// lists -- while the wide K-sized sort only moves the tile bits.
//
// Partitioning: a fixed grid of G blocks (one wave: G is the SM count times
// the CTAs of the pass that fit on an SM, at most 4); block b owns the
// contiguous segment [b*seg, (b+1)*seg) with seg = ceil(n / G) rounded up
// to the tile size, so a block's output for a digit always precedes block
// b+1's (stability across blocks); inside a block, tiles are taken in order
// and each key is ranked stably within its warp by one ballot per digit
// bit (the lanes holding the same digit, then those before it).  The first
// digit pass's histogram can be counted by the kernel that writes the keys
// (compaction, pair expansion), which saves that pass's upsweep.
#include <algorithm>
#include <atomic>
#include "pvg_internal.cuh"

namespace pvg {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 4;
constexpr int kScanChunk = kScanThreads * kScanItems;  // 1024

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
// keys per thread of the radix passes: 16 for large sorts (fewer tiles,
// fewer barriers per key), 4 when the capacity is at most
// kSmallSort (a block's chain of dependent steps is shorter)
constexpr int kSortItems = 16;
constexpr int kSmallItems = 4;
constexpr uint32_t kSmallSort = 4u << 20;
constexpr uint32_t kLateSortKeys = 12u << 20;  // capacity from which the wide sort reads values late
constexpr int kRadix = kSortRadix;

constexpr uint32_t kEmitChunk = 2048;  // pair outputs per expansion chunk
constexpr int kEmitThreads = 256;
static_assert(kEmitChunk % kEmitThreads == 0, "whole warps per expansion pass");
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// inclusive warp scan
__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

// exclusive block scan over blockDim.x (multiple of 32, <= 1024) values;
// returns the exclusive prefix, *total receives the block sum.  Uses
// 33 words of shared memory.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *smem, uint32_t *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint32_t incl = warp_incl_scan(v);
    if (lane == 31) smem[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < nw ? smem[lane] : 0;
        const uint32_t wi = warp_incl_scan(w);
        if (lane < nw) smem[lane] = wi - w;
        if (lane == 31) smem[32] = wi;
    }
    __syncthreads();
    const uint32_t r = smem[warp] + incl - v;
    *total = smem[32];
    __syncthreads();
    return r;
}

__device__ __forceinline__ void segment_of(uint32_t n, int G, int align, uint32_t *b0, uint32_t *b1) {
    uint32_t seg = (n + G - 1) / G;
    seg = (seg + align - 1) / align * align;
    const uint64_t s = (uint64_t)blockIdx.x * seg;
    *b0 = (uint32_t)(s < n ? s : n);
    const uint64_t e = s + seg;
    *b1 = (uint32_t)(e < n ? e : n);
}

// ---------------------------------------------------------------- scans

// Functor protocol: n() element count, value(i) item's count,
// apply(i, offset) consumes the exclusive prefix.
// inv: set to 0xffffffff for the invisible items (the depth sort's last
// pass writes the visible ones' positions)
struct CompactF {
    const uint32_t *cnt, *zkey;
    uint32_t *keys_out, *vals_out, *inv;
    uint32_t n_items;
    __device__ uint32_t n() const { return n_items; }
    __device__ uint32_t value(uint32_t i) const { return cnt[i] > 0u ? 1u : 0u; }
    __device__ void apply(uint32_t i, uint32_t off, uint32_t v) const {
        if (v) {
            keys_out[off] = zkey[i];
            vals_out[off] = i;
        } else {
            inv[i] = 0xffffffffu;
        }
    }
};

// Count scan of the per-visible-item tile counts.  apply() stores the
// item's first output position and, for every chunk of kEmitChunk outputs
// that starts inside the item's outputs, the item index, so the expansion
// kernel can find each chunk's items without a global search.
struct EmitF {
    const uint32_t *d_m;
    const uint32_t *vis_cnt;
    uint32_t *vis_off;
    uint32_t *chunk_start;
    uint32_t capacity;
    __device__ uint32_t n() const { return *d_m; }
    __device__ uint32_t value(uint32_t m) const { return vis_cnt[m]; }
    __device__ void apply(uint32_t m, uint32_t off, uint32_t v) const {
        vis_off[m] = off;
        if (v == 0) return;
        const uint32_t end = min(off + v, capacity);
        for (uint32_t c = (off + kEmitChunk - 1) / kEmitChunk; c * kEmitChunk < end; c++) chunk_start[c] = m;
    }
};

// zero (optional): nzero words that a later kernel of the sequence
// accumulates into or fills sparsely, zeroed here grid-wide (saving a
// memset node between kernel launches)
template <class F>
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(F f, uint32_t *partials, uint32_t *zero,
                                                              uint32_t nzero) {
    pdl_enter();
    __shared__ uint32_t smem[33];
    if (zero)
        for (uint32_t i = blockIdx.x * kScanThreads + threadIdx.x; i < nzero; i += gridDim.x * kScanThreads)
            zero[i] = 0u;
    uint32_t b0, b1;
    segment_of(f.n(), gridDim.x, kScanChunk, &b0, &b1);
    uint32_t acc = 0;
    for (uint32_t i = b0 + threadIdx.x; i < b1; i += kScanThreads) acc += f.value(i);
    uint32_t total;
    block_excl_scan(acc, smem, &total);
    if (threadIdx.x == 0) partials[blockIdx.x] = total;
}

// exclusive scan of G partials in place (one block of 1024 threads);
// *total = sum; if cap_flag != NULL and total > capacity, set *cap_flag.
__global__ void __launch_bounds__(1024) k_scan_partials(uint32_t *partials, int G, uint32_t *total,
                                                        uint32_t capacity, uint32_t *cap_flag) {
    pdl_enter();
    __shared__ uint32_t smem[33];
    const uint32_t v = threadIdx.x < (unsigned)G ? partials[threadIdx.x] : 0u;
    uint32_t tot;
    const uint32_t ex = block_excl_scan(v, smem, &tot);
    if (threadIdx.x < (unsigned)G) partials[threadIdx.x] = ex;
    if (threadIdx.x == 0) {
        *total = tot;
        if (cap_flag && tot > capacity) *cap_flag = 1u;
    }
}

template <class F>
__global__ void __launch_bounds__(kScanThreads) k_scan_apply(F f, const uint32_t *partials, uint32_t *zero,
                                                             uint32_t nzero) {
    pdl_enter();
    __shared__ uint32_t smem[33];
    if (zero)
        for (uint32_t i = blockIdx.x * kScanThreads + threadIdx.x; i < nzero; i += gridDim.x * kScanThreads)
            zero[i] = 0u;
    uint32_t b0, b1;
    segment_of(f.n(), gridDim.x, kScanChunk, &b0, &b1);
    uint32_t base = partials[blockIdx.x];
    for (uint32_t c0 = b0; c0 < b1; c0 += kScanChunk) {
        // blocked arrangement: thread t owns items c0 + t*4 .. +3
        uint32_t v[kScanItems];
        uint32_t sum = 0;
        const uint32_t first = c0 + threadIdx.x * kScanItems;
#pragma unroll
        for (int k = 0; k < kScanItems; k++) {
            const uint32_t i = first + k;
            v[k] = i < b1 ? f.value(i) : 0u;
            sum += v[k];
        }
        uint32_t total;
        uint32_t off = base + block_excl_scan(sum, smem, &total);
#pragma unroll
        for (int k = 0; k < kScanItems; k++) {
            const uint32_t i = first + k;
            if (i < b1) f.apply(i, off, v[k]);
            off += v[k];
        }
        base += total;
    }
}

// k_scan_apply for the compaction of the visible items, which also writes
// inv[i] = 0xffffffff for the invisible items and counts the first digit
// pass of the depth sort that follows: hist[d * sort_G + b] = keys with
// low byte d in the sort block b that owns their output position (the
// sort's partition of M keys into sort_G segments of whole tiles of
// sort_tile keys).  A block's outputs are contiguous, so its counts are
// summed in shared memory and added with at most 256 atomics per sort
// block they touch.  hist is zeroed by the compaction's reduce kernel.
constexpr int kCompactSpan = 4;  // sort blocks one apply block's outputs can touch (checked; else direct atomics)
__global__ void __launch_bounds__(kScanThreads) k_compact_apply(CompactF f, const uint32_t *partials,
                                                               const uint32_t *d_m, uint32_t *hist, int sort_G,
                                                               uint32_t sort_tile) {
    pdl_enter();
    __shared__ uint32_t smem[33];
    __shared__ uint32_t s_hist[kCompactSpan][kRadix];
    for (int k = threadIdx.x; k < kCompactSpan * kRadix; k += kScanThreads) (&s_hist[0][0])[k] = 0u;
    uint32_t b0, b1;
    segment_of(f.n(), gridDim.x, kScanChunk, &b0, &b1);
    const uint32_t M = *d_m;
    const uint32_t seg = ((M + sort_G - 1) / sort_G + sort_tile - 1) / sort_tile * sort_tile;
    const uint32_t block_base = partials[blockIdx.x];
    const uint32_t sb0 = block_base / max(seg, 1u);  // first sort block of this block's outputs
    uint32_t base = block_base;
    __syncthreads();
    for (uint32_t c0 = b0; c0 < b1; c0 += kScanChunk) {
        uint32_t v[kScanItems];
        uint32_t sum = 0;
        const uint32_t first = c0 + threadIdx.x * kScanItems;
#pragma unroll
        for (int k = 0; k < kScanItems; k++) {
            const uint32_t i = first + k;
            v[k] = i < b1 ? f.value(i) : 0u;
            sum += v[k];
        }
        uint32_t total;
        uint32_t off = base + block_excl_scan(sum, smem, &total);
#pragma unroll
        for (int k = 0; k < kScanItems; k++) {
            const uint32_t i = first + k;
            if (i < b1) {
                f.apply(i, off, v[k]);
                if (v[k]) {
                    const uint32_t d = f.zkey[i] & (kRadix - 1u);
                    const uint32_t sb = off / seg - sb0;
                    if (sb < (uint32_t)kCompactSpan) atomicAdd(&s_hist[sb][d], 1u);
                    else atomicAdd(&hist[(size_t)d * sort_G + sb0 + sb], 1u);
                }
            }
            off += v[k];
        }
        base += total;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kCompactSpan * kRadix; k += kScanThreads) {
        const uint32_t c = (&s_hist[0][0])[k];
        const uint32_t sb = sb0 + (uint32_t)(k / kRadix), d = (uint32_t)(k % kRadix);
        if (c) atomicAdd(&hist[(size_t)d * sort_G + sb], c);
    }
}

int scan_blocks(uint32_t capacity) {
    uint32_t g = (capacity + kScanChunk - 1) / kScanChunk;
    if (g < 1) g = 1;
    if (g > kMaxScanBlocks) g = kMaxScanBlocks;
    return (int)g;
}

// CTAs of the 16-keys-per-thread downsweep (late: the variant with late
// value reads) that fit on one SM (its registers and 43 KB of shared
// memory), at most 4: the grid of the wide sorts stays one wave, since a
// block's tiles run one after another and a second wave of blocks would
// double the pass.  Read once.
int wide_sort_blocks_per_sm(bool late);

int sort_blocks(uint32_t capacity, int tile) {
    uint32_t g = (capacity + tile - 1) / tile;
    const int per_sm = tile == kSortThreads * kSortItems ? wide_sort_blocks_per_sm(capacity >= kLateSortKeys) : 4;
    const uint32_t cap = (uint32_t)std::min(kMaxSortBlocks, per_sm * device_sm_count());
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

// ---------------------------------------------------------------- radix

template <int ITEMS>
__global__ void __launch_bounds__(kSortThreads) k_radix_upsweep(const uint32_t *keys, const uint32_t *d_n,
                                                                uint32_t cap, int shift, uint32_t mask,
                                                                uint32_t *hist) {
    pdl_enter();
    __shared__ uint32_t sh[kRadix];
    for (int d = threadIdx.x; d < kRadix; d += kSortThreads) sh[d] = 0;
    __syncthreads();
    uint32_t b0, b1;
    segment_of(min(*d_n, cap), gridDim.x, kSortThreads * ITEMS, &b0, &b1);
    for (uint32_t i = b0 + threadIdx.x; i < b1; i += kSortThreads) atomicAdd(&sh[(keys[i] >> shift) & mask], 1u);
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += kSortThreads) hist[d * gridDim.x + blockIdx.x] = sh[d];
}

// Row scan of the digit-major histogram hist[d * G + b], one block per
// digit d: exclusive prefix over the G blocks in place, row total to
// totals[d].  The downsweep adds the exclusive prefix of the totals over
// the digits.  G <= 1024.
__global__ void __launch_bounds__(1024) k_radix_scan(uint32_t *hist, uint32_t *totals, int G) {
    pdl_enter();
    __shared__ uint32_t smem[33];
    uint32_t *row = hist + (size_t)blockIdx.x * G;
    const uint32_t v = (int)threadIdx.x < G ? row[threadIdx.x] : 0u;
    uint32_t tot;
    const uint32_t ex = block_excl_scan(v, smem, &tot);
    if ((int)threadIdx.x < G) row[threadIdx.x] = ex;
    if (threadIdx.x == 0) totals[blockIdx.x] = tot;
}

// Expansion of the sorted visible items into (tile id, depth position)
// pairs, one chunk of kEmitChunk outputs at a time.  The item of every
// output comes from a block max-scan of start markers (each item whose
// first output falls in the chunk marks that slot with its m; the scan
// carries the last mark forward).  Its r-th pair is the r-th tile, row by
// row, of the rectangle tiles that its footprint ellipse meets: read from
// the item's packed row table when it has one (at most kTabRows rows),
// else recomputed from the stored ellipse, 32 rows at a time by the whole
// warp, for one such item after another.  The kernel also counts the
// first digit pass of the tile sort that follows (hist, zeroed by the
// scan before it): each chunk's outputs are contiguous, so their counts
// are summed in shared memory per sort block and added with atomics.
__global__ void __launch_bounds__(kEmitThreads) k_expand_pairs(const uint32_t *__restrict__ vis_off,
                                                              const uint32_t *__restrict__ vis_cnt,
                                                              const uint32_t *__restrict__ chunk_start,
                                                              const uint2 *__restrict__ rect,
                                                              const uint4 *__restrict__ rowtab,
                                                              const float4 *__restrict__ ell, int tile_w,
                                                              int tile_h, const uint32_t *__restrict__ sgid,
                                                              const ViewDesc *views, int nv, const uint32_t *d_m,
                                                              const uint32_t *d_k, uint32_t capacity,
                                                              uint32_t *__restrict__ keys, uint32_t *__restrict__ vals,
                                                              uint32_t *__restrict__ hist, int sort_G,
                                                              uint32_t sort_tile) {
    pdl_enter();
    constexpr int kPer = kEmitChunk / kEmitThreads;  // slots per thread in the scan
    __shared__ uint32_t s_item[kEmitChunk];
    __shared__ uint32_t s_warp[kEmitThreads / 32];
    __shared__ uint32_t s_hist[kCompactSpan][kRadix];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t M = *d_m;
    const uint32_t K = min(*d_k, capacity);
    const uint32_t nchunks = (K + kEmitChunk - 1) / kEmitChunk;
    // the tile sort's partition of the K pairs (its segment of whole tiles)
    const uint32_t seg = max(((K + sort_G - 1) / sort_G + sort_tile - 1) / sort_tile * sort_tile, 1u);
    for (uint32_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const uint32_t j0 = c * kEmitChunk;
        const uint32_t m_lo = chunk_start[c];
        const uint32_t m_hi = (c + 1 < nchunks) ? chunk_start[c + 1] : M - 1;
        // sort blocks of the chunk's outputs: sb0 .. sb0 + nsb - 1 counted in
        // shared memory (any beyond kCompactSpan straight into hist)
        const uint32_t sb0 = j0 / seg;
        const int nsb = (int)min((min(j0 + kEmitChunk, K) - 1) / seg - sb0 + 1, (uint32_t)kCompactSpan);
        __syncthreads();
        for (int q = threadIdx.x; q < (int)kEmitChunk; q += kEmitThreads) s_item[q] = 0u;
        for (int q = threadIdx.x; q < nsb * kRadix; q += kEmitThreads) (&s_hist[0][0])[q] = 0u;
        __syncthreads();
        // marks: slot 0 holds the item containing j0 (chunk_start); a
        // non-empty item starting inside the chunk marks its first slot
        // (distinct slots: non-empty items start at distinct offsets)
        if (threadIdx.x == 0) s_item[0] = m_lo;
        for (uint32_t m = m_lo + threadIdx.x; m <= m_hi; m += kEmitThreads) {
            const uint32_t o = vis_off[m];
            if (o >= j0 && o - j0 < kEmitChunk && vis_cnt[m] > 0u) s_item[o - j0] = m;
        }
        __syncthreads();
        // inclusive max-scan of the marks: kPer consecutive slots per
        // thread, then across the warp, then across the warps
        uint32_t loc[kPer];
        uint32_t run = 0;
#pragma unroll
        for (int i = 0; i < kPer; i++) {
            run = max(run, s_item[threadIdx.x * kPer + i]);
            loc[i] = run;
        }
        uint32_t wrun = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, wrun, o);
            if (lane >= o) wrun = max(wrun, y);
        }
        if (lane == 31) s_warp[warp] = wrun;
        uint32_t before = __shfl_up_sync(kFull, wrun, 1);
        if (lane == 0) before = 0;
        __syncthreads();
        for (int w = 0; w < warp; w++) before = max(before, s_warp[w]);
#pragma unroll
        for (int i = 0; i < kPer; i++) s_item[threadIdx.x * kPer + i] = max(loc[i], before);
        __syncthreads();
        // whole warps iterate together (kEmitChunk is a multiple of the
        // block), so the warp-wide steps below see all 32 lanes
        for (uint32_t q = threadIdx.x; q < kEmitChunk; q += kEmitThreads) {
            const uint32_t j = j0 + q;
            const bool valid = j < K;
            if (!__any_sync(kFull, valid)) break;
            const uint32_t m = valid ? s_item[q] : m_lo;
            uint32_t r = valid ? j - vis_off[m] : 0u;
            const uint2 rc = rect[m];
            const uint32_t tx0 = rc.x & 0xffffu, ty0 = rc.x >> 16, tx1 = rc.y & 0xffffu, ty1 = rc.y >> 16;
            uint32_t tx = tx0, ty = ty0;  // the rows sum to the item's count; first tile otherwise
            const bool tab = has_row_table(tx0, ty0, tx1, ty1);
            if (valid && tab) {
                const uint4 t = rowtab[m];
                const uint32_t w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
                for (int i = 0; i < (int)kTabRows; i++) {
                    if (ty0 + i >= ty1) break;
                    const uint32_t v = (w[i >> 1] >> (16 * (i & 1))) & 0xffffu;
                    const uint32_t sp = v >> 8;
                    if (r < sp) {
                        tx = tx0 + (v & 0xffu) + r;
                        ty = ty0 + i;
                        break;
                    }
                    r -= sp;
                }
            }
            // items without a table, one at a time: the warp evaluates 32
            // rows at once, scans their spans and each of the item's lanes
            // finds its row by binary search over the inclusive sums.  Every
            // lane takes part in every shuffle (none sits behind a branch or
            // a short-circuit).
            const bool coop = valid && !tab;
            uint32_t pending = __ballot_sync(kFull, coop);
            while (pending) {
                const int L = __ffs(pending) - 1;
                const uint32_t mL = __shfl_sync(kFull, m, L);
                const bool mine = coop && m == mL;
                const FootprintEllipse EL = load_ellipse(ell, mL);
                const uint2 rl = rect[mL];
                const uint32_t ltx0 = rl.x & 0xffffu, lty0 = rl.x >> 16, ltx1 = rl.y & 0xffffu, lty1 = rl.y >> 16;
                bool todo = mine;
                uint32_t base = 0;
                for (uint32_t row0 = lty0; row0 < lty1; row0 += 32) {
                    const uint32_t row = row0 + lane;
                    uint32_t cx = 0, sp = 0;
                    if (row < lty1) {
                        const uint2 cc = footprint_cols(EL, row, tile_w, tile_h, ltx0, ltx1);
                        cx = cc.x;
                        sp = cc.y - cc.x;
                    }
                    const uint32_t inc = warp_incl_scan(sp);
                    const uint32_t total = __shfl_sync(kFull, inc, 31);
                    const uint32_t rr = r - base;  // used only while todo (then r >= base)
                    uint32_t k = 0;  // first lane whose inclusive sum exceeds rr
#pragma unroll
                    for (int step = 16; step; step >>= 1) {
                        const uint32_t v = __shfl_sync(kFull, inc, k + step - 1);
                        if (v <= rr) k += step;
                    }
                    const uint32_t inc_k = __shfl_sync(kFull, inc, k), sp_k = __shfl_sync(kFull, sp, k);
                    const uint32_t cx_k = __shfl_sync(kFull, cx, k);
                    if (todo && rr < total) {
                        ty = row0 + k;
                        tx = cx_k + rr - (inc_k - sp_k);
                        todo = false;
                    }
                    base += total;
                    if (!__any_sync(kFull, todo)) break;
                }
                pending &= ~__ballot_sync(kFull, mine);
            }
            if (valid) {
                const int view = nv == 1 ? 0 : view_of_item(views, nv, sgid[m]);
                const uint32_t key = views[view].tile_base + ty * (uint32_t)views[view].tiles_x + tx;
                keys[j] = key;
                vals[j] = m;
                const uint32_t d = key & (kRadix - 1u), sb = j / seg - sb0;
                if (sb < (uint32_t)nsb) atomicAdd(&s_hist[sb][d], 1u);
                else atomicAdd(&hist[(size_t)d * sort_G + sb0 + sb], 1u);
            }
        }
        __syncthreads();
        for (int q = threadIdx.x; q < nsb * kRadix; q += kEmitThreads) {
            const uint32_t cnt = (&s_hist[0][0])[q];
            if (cnt) atomicAdd(&hist[(size_t)(q % kRadix) * sort_G + sb0 + (uint32_t)(q / kRadix)], cnt);
        }
    }
}

static_assert(kSortThreads == kRadix, "one thread per digit in the downsweep");

template <int TILE>
struct SortSmem {
    uint32_t base[kRadix];                // running global offset per digit
    uint32_t warp_hist[kSortWarps][kRadix];
    uint32_t tile_start[kRadix];
    uint32_t keys[TILE];
    uint32_t vals[TILE];
    uint32_t scan[33];
};

// NB: ballots per key in the ranking (the pass's digit width, or 8)
template <int ITEMS, int NB, bool kLateVals>
__device__ __forceinline__ void radix_downsweep(const uint32_t *__restrict__ keys_in,
                                                const uint32_t *__restrict__ vals_in, uint32_t *__restrict__ keys_out,
                                                uint32_t *__restrict__ vals_out, const uint32_t *d_n, uint32_t cap,
                                                int shift, uint32_t mask, const uint32_t *hist,
                                                const uint32_t *totals, uint32_t *__restrict__ inv_out) {
    constexpr int kSortTile = kSortThreads * ITEMS;
    __shared__ SortSmem<kSortTile> S;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    {
        // digit bases: exclusive prefix of the per-digit totals (one thread per digit)
        uint32_t tot;
        const uint32_t dbase = block_excl_scan(totals[tid], S.scan, &tot);
        S.base[tid] = dbase + hist[tid * gridDim.x + blockIdx.x];
    }
    uint32_t b0, b1;
    segment_of(min(*d_n, cap), gridDim.x, kSortTile, &b0, &b1);
    const uint32_t lt = lanemask_lt();
    for (uint32_t t0 = b0; t0 < b1; t0 += kSortTile) {
        for (int k = tid; k < kSortWarps * kRadix; k += kSortThreads) (&S.warp_hist[0][0])[k] = 0;
        __syncthreads();
        // kLateVals: the values are read only when they are placed (below),
        // so that a thread holds its keys and ranks but not its values
        // meanwhile (64 registers: four CTAs per SM)
        uint32_t key[ITEMS], val[kLateVals ? 1 : ITEMS], rank[ITEMS];
        bool valid[ITEMS];
#pragma unroll
        for (int j = 0; j < ITEMS; j++) {
            const uint32_t pos = t0 + warp * (32 * ITEMS) + j * 32 + lane;
            valid[j] = pos < b1;
            key[j] = valid[j] ? keys_in[pos] : 0u;
            if constexpr (!kLateVals) val[j] = valid[j] ? vals_in[pos] : 0u;
        }
#pragma unroll
        for (int j = 0; j < ITEMS; j++) {
            const uint32_t d = (key[j] >> shift) & mask;
            uint32_t peers = __ballot_sync(0xffffffffu, valid[j]);
#pragma unroll
            for (int bit = 0; bit < NB; bit++) {
                const bool on = (d >> bit) & 1u;
                const uint32_t b = __ballot_sync(0xffffffffu, on);
                peers &= on ? b : ~b;
            }
            uint32_t before = 0;
            if (valid[j]) before = S.warp_hist[warp][d];
            __syncwarp();
            if (valid[j] && (peers & lt) == 0) S.warp_hist[warp][d] = before + __popc(peers);
            __syncwarp();
            rank[j] = before + __popc(peers & lt);
        }
        __syncthreads();
        // per digit: exclusive offsets across warps, tile count, tile start
        uint32_t tile_cnt = 0;
        {
            const int d = tid;  // kSortThreads == kRadix
#pragma unroll
            for (int w = 0; w < kSortWarps; w++) {
                const uint32_t c = S.warp_hist[w][d];
                S.warp_hist[w][d] = tile_cnt;
                tile_cnt += c;
            }
            uint32_t tot;
            S.tile_start[d] = block_excl_scan(tile_cnt, S.scan, &tot);
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < ITEMS; j++) {
            if (!valid[j]) continue;
            const uint32_t d = (key[j] >> shift) & mask;
            const uint32_t p = S.tile_start[d] + S.warp_hist[warp][d] + rank[j];
            S.keys[p] = key[j];
            if constexpr (kLateVals) S.vals[p] = vals_in[t0 + warp * (32 * ITEMS) + j * 32 + lane];
            else S.vals[p] = val[j];
        }
        __syncthreads();
        const uint32_t nvalid = (b1 - t0) < (uint32_t)kSortTile ? (b1 - t0) : (uint32_t)kSortTile;
        for (uint32_t p = tid; p < nvalid; p += kSortThreads) {
            const uint32_t k = S.keys[p];
            const uint32_t d = (k >> shift) & mask;
            const uint32_t dst = S.base[d] + (p - S.tile_start[d]);
            keys_out[dst] = k;
            vals_out[dst] = S.vals[p];
            if (inv_out) inv_out[S.vals[p]] = dst;
        }
        __syncthreads();
        S.base[tid] += tile_cnt;
        __syncthreads();
    }
}

// The downsweep for ITEMS keys per thread, values read with the keys; and
// the wide one for long sorts (kLateSortKeys and more), with late value
// reads, held to 64 registers: four CTAs of 43 KB per SM instead of three.
// A block of a long sort walks tens of tiles, where the extra CTA per SM
// pays (64M random keys: 2.09 vs 2.40 ms); with a few tiles per block the
// late reads' latency shows instead (a 3.3M-pair tile sort: 0.070 vs 0.061
// ms).
template <int ITEMS, int NB>
__global__ void __launch_bounds__(kSortThreads) k_radix_downsweep(const uint32_t *__restrict__ keys_in,
                                                                  const uint32_t *__restrict__ vals_in,
                                                                  uint32_t *__restrict__ keys_out,
                                                                  uint32_t *__restrict__ vals_out,
                                                                  const uint32_t *d_n, uint32_t cap, int shift,
                                                                  uint32_t mask, const uint32_t *hist,
                                                                  const uint32_t *totals,
                                                                  uint32_t *__restrict__ inv_out) {
    pdl_enter();
    radix_downsweep<ITEMS, NB, false>(keys_in, vals_in, keys_out, vals_out, d_n, cap, shift, mask, hist, totals,
                                      inv_out);
}

template <int NB>
__global__ void __launch_bounds__(kSortThreads, 4) k_radix_downsweep_wide(const uint32_t *__restrict__ keys_in,
                                                                           const uint32_t *__restrict__ vals_in,
                                                                           uint32_t *__restrict__ keys_out,
                                                                           uint32_t *__restrict__ vals_out,
                                                                           const uint32_t *d_n, uint32_t cap,
                                                                           int shift, uint32_t mask,
                                                                           const uint32_t *hist,
                                                                           const uint32_t *totals,
                                                                           uint32_t *__restrict__ inv_out) {
    pdl_enter();
    radix_downsweep<kSortItems, NB, true>(keys_in, vals_in, keys_out, vals_out, d_n, cap, shift, mask, hist, totals,
                                          inv_out);
}

// [start, end) of every tile's run in the sorted keys.  Eight keys per
// thread per sweep (two 16-byte loads and the two neighbours), so that
// few dependent sweeps remain.
__global__ void __launch_bounds__(256) k_ranges(const uint32_t *__restrict__ keys, const uint32_t *d_k,
                                                uint32_t capacity, uint2 *__restrict__ ranges) {
    pdl_enter();
    constexpr uint32_t kNone = 0xffffffffu;  // no tile has this id
    const uint32_t K = min(*d_k, capacity);
    const uint32_t stride = gridDim.x * blockDim.x * 8u;
    for (uint32_t j0 = (blockIdx.x * blockDim.x + threadIdx.x) * 8u; j0 < K; j0 += stride) {
        uint32_t k[10];  // keys[j0 - 1 .. j0 + 8]
        k[0] = j0 > 0 ? keys[j0 - 1] : kNone;
        if (j0 + 8 <= K) {
            const uint4 a = reinterpret_cast<const uint4 *>(keys + j0)[0];
            const uint4 b = reinterpret_cast<const uint4 *>(keys + j0)[1];
            k[1] = a.x; k[2] = a.y; k[3] = a.z; k[4] = a.w;
            k[5] = b.x; k[6] = b.y; k[7] = b.z; k[8] = b.w;
        } else {
#pragma unroll
            for (int i = 0; i < 8; i++) k[1 + i] = j0 + i < K ? keys[j0 + i] : kNone;
        }
        k[9] = j0 + 8 < K ? keys[j0 + 8] : kNone;
#pragma unroll
        for (int i = 0; i < 8; i++) {
            const uint32_t t = k[1 + i];
            if (t == kNone) break;
            if (k[i] != t) ranges[t].x = j0 + i;
            if (k[2 + i] != t) ranges[t].y = j0 + i + 1;
        }
    }
}

int wide_sort_blocks_per_sm(bool late) {
    static std::atomic<int> cached[2] = {{0}, {0}};
    int n = cached[late].load(std::memory_order_relaxed);
    if (n > 0) return n;
    int occ = 0;
    const cudaError_t e =
        late ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_radix_downsweep_wide<8>, kSortThreads, 0)
             : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_radix_downsweep<kSortItems, 8>, kSortThreads, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        occ = 3;
    }
    n = std::max(1, std::min(occ, 4));
    cached[late].store(n, std::memory_order_relaxed);
    return n;
}

struct TempLayout {
    uint32_t *hist;      // kRadix * kMaxSortBlocks
    uint32_t *partials;  // kMaxScanBlocks
    uint32_t *totals;    // kRadix (shares the partials' space: never live together)
};

TempLayout temp_layout(void *temp) {
    TempLayout t;
    t.hist = (uint32_t *)temp;
    t.partials = t.hist + kRadix * kMaxSortBlocks;
    t.totals = t.partials;
    return t;
}

}  // namespace

static_assert(kSortTempBytes >= sizeof(uint32_t) * ((size_t)kRadix * kMaxSortBlocks + kMaxScanBlocks),
              "sort scratch layout");
size_t sort_temp_bytes() { return kSortTempBytes; }

void compact_visible(const Params &p, uint32_t *keys_out, uint32_t *vals_out, uint32_t *inv, void *temp,
                     cudaStream_t s) {
    TempLayout t = temp_layout(temp);
    CompactF f{p.item_cnt, p.item_zkey, keys_out, vals_out, inv, p.n_items};
    const int G = scan_blocks(p.n_items);
    // the depth sort's partition (radix_sort_pairs with capacity n_items)
    const int sort_items = p.n_items <= kSmallSort ? kSmallItems : kSortItems;
    const int sort_G = sort_blocks(p.n_items, kSortThreads * sort_items);
    note_launch();
    pdl_launch(k_scan_reduce<CompactF>, G, kScanThreads, 0, s, f, t.partials, t.hist, (uint32_t)(kRadix * sort_G));
    note_launch();
    pdl_launch(k_scan_partials, 1, 1024, 0, s, t.partials, G, &p.counters[0], 0xffffffffu, nullptr);
    note_launch();
    pdl_launch(k_compact_apply, G, kScanThreads, 0, s, f, (const uint32_t *)t.partials,
               (const uint32_t *)&p.counters[0], t.hist, sort_G, (uint32_t)(kSortThreads * sort_items));
}

template <int ITEMS>
void radix_passes(uint32_t *keys, uint32_t *vals, uint32_t *keys_alt, uint32_t *vals_alt, const uint32_t *d_count,
                  uint32_t capacity, int begin_bit, int end_bit, void *temp, cudaStream_t s, bool *result_in_alt,
                  uint32_t *inv_out, bool first_hist);

void radix_sort_pairs(uint32_t *keys, uint32_t *vals, uint32_t *keys_alt, uint32_t *vals_alt,
                      const uint32_t *d_count, uint32_t capacity, int begin_bit, int end_bit, void *temp,
                      cudaStream_t s, bool *result_in_alt, uint32_t *inv_out, bool first_hist) {
    if (capacity <= kSmallSort)
        radix_passes<kSmallItems>(keys, vals, keys_alt, vals_alt, d_count, capacity, begin_bit, end_bit, temp, s,
                                  result_in_alt, inv_out, first_hist);
    else
        radix_passes<kSortItems>(keys, vals, keys_alt, vals_alt, d_count, capacity, begin_bit, end_bit, temp, s,
                                 result_in_alt, inv_out, first_hist);
}

template <int ITEMS>
void radix_passes(uint32_t *keys, uint32_t *vals, uint32_t *keys_alt, uint32_t *vals_alt, const uint32_t *d_count,
                  uint32_t capacity, int begin_bit, int end_bit, void *temp, cudaStream_t s, bool *result_in_alt,
                  uint32_t *inv_out, bool first_hist) {
    TempLayout t = temp_layout(temp);
    const int G = sort_blocks(capacity, kSortThreads * ITEMS);
    bool alt = false;
    for (int b = begin_bit; b < end_bit;) {
        const int nb = (end_bit - b) >= 8 ? 8 : (end_bit - b);
        const uint32_t mask = (1u << nb) - 1u;
        const uint32_t *ki = alt ? keys_alt : keys;
        const uint32_t *vi = alt ? vals_alt : vals;
        uint32_t *ko = alt ? keys : keys_alt;
        uint32_t *vo = alt ? vals : vals_alt;
        if (!(first_hist && b == begin_bit)) {  // else counted by the producer of the keys
            note_launch();
            pdl_launch(k_radix_upsweep<ITEMS>, G, kSortThreads, 0, s, ki, d_count, capacity, b, mask, t.hist);
        }
        note_launch();
        pdl_launch(k_radix_scan, kRadix, 1024, 0, s, t.hist, t.totals, G);
        note_launch();
        uint32_t *inv_pass = b + nb >= end_bit ? inv_out : nullptr;  // the last pass only
        // one ballot per digit bit: the last pass of a sort by fewer than a
        // multiple of 8 bits ranks with fewer ballots
#define PVG_DOWNSWEEP(NBITS)                                                                                    \
    case NBITS:                                                                                                 \
        if (ITEMS == kSortItems && capacity >= kLateSortKeys)                                                  \
            pdl_launch(k_radix_downsweep_wide<NBITS>, G, kSortThreads, 0, s, ki, vi, ko, vo, d_count, capacity, b, \
                       mask, t.hist, t.totals, inv_pass);                                                       \
        else                                                                                                    \
            pdl_launch(k_radix_downsweep<ITEMS, NBITS>, G, kSortThreads, 0, s, ki, vi, ko, vo, d_count, capacity, b, \
                       mask, t.hist, t.totals, inv_pass);                                                       \
        break;
        switch (nb) {
            PVG_DOWNSWEEP(1) PVG_DOWNSWEEP(2) PVG_DOWNSWEEP(3) PVG_DOWNSWEEP(4)
            PVG_DOWNSWEEP(5) PVG_DOWNSWEEP(6) PVG_DOWNSWEEP(7)
            default: PVG_DOWNSWEEP(8)
        }
#undef PVG_DOWNSWEEP
        alt = !alt;
        b += nb;
    }
    *result_in_alt = alt;
}

// scan of the per-visible tile counts: K -> counters[1], overflow flag ->
// counters[2]; then emission of the (tile, m) pairs in depth order.
void scan_count_pairs(const Params &p, void *temp, cudaStream_t s) {
    TempLayout t = temp_layout(temp);
    EmitF f{&p.counters[0], p.vis_cnt, p.vis_off, p.chunk_start, p.pair_capacity};
    const int G = scan_blocks(p.n_items);
    // the tile ranges are zeroed here for k_ranges, which writes only the
    // non-empty tiles' (no memset node in the launch sequence)
    note_launch();
    pdl_launch(k_scan_reduce<EmitF>, G, kScanThreads, 0, s, f, t.partials, reinterpret_cast<uint32_t *>(p.ranges),
               (uint32_t)(2 * p.total_tiles));
    note_launch();
    pdl_launch(k_scan_partials, 1, 1024, 0, s, t.partials, G, &p.counters[1], p.pair_capacity, &p.counters[2]);
}

size_t emit_chunks(uint32_t capacity) { return (capacity + kEmitChunk - 1) / kEmitChunk + 1; }

void scan_emit_pairs(const Params &p, void *temp, cudaStream_t s) {
    TempLayout t = temp_layout(temp);
    EmitF f{&p.counters[0], p.vis_cnt, p.vis_off, p.chunk_start, p.pair_capacity};
    const int G = scan_blocks(p.n_items);
    // the tile sort's partition (radix_sort_pairs with capacity pair_capacity);
    // its first histogram is zeroed here and counted by the expansion
    const int sort_items = p.pair_capacity <= kSmallSort ? kSmallItems : kSortItems;
    const int sort_G = sort_blocks(p.pair_capacity, kSortThreads * sort_items);
    note_launch();
    pdl_launch(k_scan_apply<EmitF>, G, kScanThreads, 0, s, f, (const uint32_t *)t.partials, t.hist,
               (uint32_t)(kRadix * sort_G));
    uint32_t grid = (uint32_t)((p.pair_capacity + kEmitChunk - 1) / kEmitChunk);
    if (grid < 1) grid = 1;
    if (grid > (uint32_t)(8 * device_sm_count())) grid = 8 * device_sm_count();
    note_launch();
    pdl_launch(k_expand_pairs, grid, kEmitThreads, 0, s, p.vis_off, p.vis_cnt, p.chunk_start, p.rect, p.rowtab, p.ell,
                                                 p.tile_w, p.tile_h,
                                                 p.sgid, p.views, p.n_views,
                                                 &p.counters[0], &p.counters[1], p.pair_capacity, p.pair_keys,
                                                 p.pair_vals, t.hist, sort_G, (uint32_t)(kSortThreads * sort_items));
}

// Tile order for the compositor: heaviest lists first (64 log-spaced
// length buckets, longest bucket first), so the long tiles start at once
// and the short ones fill in behind them.  Order within a bucket is left
// to the atomics (each tile's result does not depend on when it runs).
// walk (optional): order by the tiles' walk lengths instead (the adjoint:
// each tile's largest last-blend position, which the forward recorded).
// One block, any multiple of 64 threads.
__device__ __forceinline__ void tile_order_block(const uint2 *__restrict__ ranges, const uint32_t *walk,
                                                 uint32_t n_tiles, uint32_t *__restrict__ order) {
    __shared__ uint32_t cnt[64];
    __shared__ uint32_t smem[33];
    if (threadIdx.x < 64) cnt[threadIdx.x] = 0;
    __syncthreads();
    auto bucket = [&](uint32_t t) {
        const uint32_t len = walk ? walk[t] : ranges[t].y - ranges[t].x;
        const int b = min(63, (int)(log2f((float)len + 1.0f) * 3.0f));
        return 63 - b;  // longest first
    };
    for (uint32_t t = threadIdx.x; t < n_tiles; t += blockDim.x) atomicAdd(&cnt[bucket(t)], 1u);
    __syncthreads();
    uint32_t tot;
    const uint32_t v = threadIdx.x < 64 ? cnt[threadIdx.x] : 0u;
    const uint32_t ex = block_excl_scan(v, smem, &tot);
    if (threadIdx.x < 64) cnt[threadIdx.x] = ex;
    __syncthreads();
    for (uint32_t t = threadIdx.x; t < n_tiles; t += blockDim.x) order[atomicAdd(&cnt[bucket(t)], 1u)] = t;
}

__global__ void __launch_bounds__(1024) k_tile_order(const uint2 *__restrict__ ranges, uint32_t n_tiles,
                                                     uint32_t *__restrict__ order) {
    pdl_enter();
    tile_order_block(ranges, nullptr, n_tiles, order);
}

// The adjoint's first kernel: rows [0, *d_m) of a [*, per] array zeroed
// (the visible items' image-space gradients, which the adjoint accumulates)
// by all blocks but the last, which orders the tiles by their walk lengths
// and resets the per-item adjoint's chunk ticket (counters[3]).
__global__ void __launch_bounds__(1024) k_bwd_prep(float *__restrict__ a, const uint32_t *d_m, int per,
                                                  const uint32_t *walk, uint32_t n_tiles,
                                                  uint32_t *__restrict__ order, uint32_t *ticket) {
    pdl_enter();
    if (blockIdx.x == gridDim.x - 1) {
        if (threadIdx.x == 0) *ticket = 0u;  // the per-item adjoint's chunk ticket
        tile_order_block(nullptr, walk, n_tiles, order);
        return;
    }
    const size_t n = (size_t)per * *d_m;
    const size_t stride = (size_t)(gridDim.x - 1) * blockDim.x;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += stride) a[k] = 0.f;
}

void launch_tile_order(const Params &p, cudaStream_t s) {
    if (p.total_tiles == 0) return;
    note_launch();
    pdl_launch(k_tile_order, 1, 1024, 0, s, p.ranges, p.total_tiles, p.tile_order);
}

void launch_bwd_prep(const Params &p, const uint32_t *walk, uint32_t *order, cudaStream_t s) {
    note_launch();
    pdl_launch(k_bwd_prep, device_sm_count() + 1, 1024, 0, s, p.g2d, (const uint32_t *)&p.counters[0], 10, walk,
               p.total_tiles, order, &p.counters[3]);
}

// ranges: zeroed by the pair count scan (scan_count_pairs)
void launch_ranges(const Params &p, cudaStream_t s) {
    note_launch();
    pdl_launch(k_ranges, 8 * device_sm_count(), 256, 0, s, p.pair_keys, &p.counters[1], p.pair_capacity, p.ranges);
}

}  // namespace pvg
