// Tile binning and key sort (the tile pipeline of Section 3.2).
//
// The order required is that of the 64-bit key (view, tile, depth bits) with
// ties by Gaussian index.  Instead of radix-sorting 64-bit keys of every
// (Gaussian, tile) pair, the sort is split in two stable stages:
//   1. the V*N (view, Gaussian) entries are sorted by depth bits -- 4
//      byte-digit passes on the FP32 depth bits, stable, so equal depths keep
//      the index order (the views interleave; stage 2's key holds the view).
//      The keys kernel also writes the first pass's block counts and the OR
//      of the keys and of their complements; before the counting sort, a
//      pass on a byte that is the same in every key is skipped whole and the
//      kernels of each pass find the buffer holding the keys from the parity
//      of the passes before it that ran (elsewhere such a pass is a copy);
//   2. the pairs of every entry's bins are ordered on the (view * bins + bin)
//      key alone, stably, so each list keeps its entries' depth order.  When
//      the per-warp key tables fit in shared memory (V * bins <= CS_MAX_KEYS)
//      this is a counting sort that writes each pair once, straight to its
//      place; otherwise the pairs are emitted in entry order and radix-sorted
//      on the key, ceil(log2(V * bins) / 8) byte passes.
// A bin is bin x bin tiles.  With bin = 1 the lists are the per-tile lists;
// with larger bins every tile of a bin shares the bin's depth-ordered list and
// the compositing kernels keep, on the fly, the entries whose footprint
// rectangle holds their tile -- the same records in the same order as the
// per-tile list, for far fewer pairs to sort.
// All passes are of reduce-then-scan form (counts, one-block scans, ranked
// scatter): no inter-block waits, deterministic output.  Equal digits or
// keys within a warp are found with one ballot per bit (ballot_match), which
// measured faster here than __match_any_sync.
#include <algorithm>

#include "common.cuh"
#include "sort.cuh"

namespace gs3 {

constexpr int RADIX = 256;
constexpr int SORT_THREADS = 256;
constexpr int SORT_WARPS = SORT_THREADS / 32;
constexpr int SORT_ITEMS = 8;
constexpr int SORT_TILE = SORT_THREADS * SORT_ITEMS;  // 2048 keys per block step
constexpr int SORT_BLOCKS_MAX = kMaxSMs * 4;          // bound of the fixed sort grid (workspace)
// the sort grid: fixed (n may live on the device), 4 blocks per SM
inline int sort_blocks() { return num_sms() * 4; }
constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

struct SortPass {
    const uint32_t *kin, *vin;
    uint32_t *kout, *vout;
    const int64_t *d_n;  // device count (NULL: use n_host)
    int64_t n_host;
    int shift;
    uint32_t *hist;      // [RADIX][G]
    int G;
    // optional: OR of the keys and OR of their complements.  A byte set in
    // both differs between keys; a pass on any other byte keeps the order
    // and is skipped whole.  Each pass then reads buffer kb/vb[f & 1], f the
    // passes before it that are not skipped, and writes the other (kin,
    // vin, kout, vout are set from them on the device).
    const uint32_t *kor;
    uint32_t *kb[2], *vb[2];
};

__device__ __forceinline__ int64_t pass_n(const SortPass &s) { return s.d_n ? *s.d_n : s.n_host; }

__device__ __forceinline__ void block_range(int64_t n, int G, int b, int64_t &beg, int64_t &end)
{
    int64_t tiles = (n + SORT_TILE - 1) / SORT_TILE;
    int64_t per = (tiles + G - 1) / G;
    beg = (int64_t)b * per * SORT_TILE;
    end = min(n, beg + per * SORT_TILE);
}

__device__ __forceinline__ bool byte_constant(const uint32_t *kor, int shift)
{
    return kor && (((kor[0] & kor[1]) >> shift) & (RADIX - 1)) == 0u;
}

// Passes on the bytes below `shift` that are not skipped (kor as in SortPass).
__device__ __forceinline__ int passes_below(const uint32_t *kor, int shift)
{
    const uint32_t diff = kor[0] & kor[1];
    int f = 0;
    for (int sh = 0; sh < shift; sh += 8) f += ((diff >> sh) & (RADIX - 1)) != 0u;
    return f;
}

__device__ __forceinline__ void pass_buffers(SortPass &s)
{
    if (!s.kor) return;
    const bool odd = passes_below(s.kor, s.shift) & 1;  // selects, not an indexed (local) copy
    s.kin = odd ? s.kb[1] : s.kb[0];
    s.vin = odd ? s.vb[1] : s.vb[0];
    s.kout = odd ? s.kb[0] : s.kb[1];
    s.vout = odd ? s.vb[0] : s.vb[1];
}


// Lanes whose value v (below 2^BITS) equals this lane's, among the lanes with
// ok set (an empty set for a lane without): one ballot per bit.
template <int BITS>
__device__ __forceinline__ unsigned ballot_match(uint32_t v, bool ok)
{
    const unsigned okm = __ballot_sync(0xffffffffu, ok);
    unsigned m = ok ? okm : 0u;
#pragma unroll
    for (int b = 0; b < BITS; ++b) {
        const bool bit = (v >> b) & 1u;
        const unsigned bb = __ballot_sync(0xffffffffu, bit);
        m &= bit ? bb : ~bb;
    }
    return m;
}

__device__ __forceinline__ uint32_t digit_of(const SortPass &s, uint32_t k, uint32_t v)
{
    return (k >> s.shift) & (RADIX - 1);
}

__global__ void __launch_bounds__(SORT_THREADS) radix_hist_kernel(SortPass s)
{
    if (byte_constant(s.kor, s.shift)) return;
    pass_buffers(s);
    __shared__ uint32_t h[RADIX];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t beg, end;
    block_range(pass_n(s), s.G, blockIdx.x, beg, end);
    // a tile's loads in flight before its counts
    for (int64_t t0 = beg; t0 < end; t0 += SORT_TILE) {
        uint32_t d[SORT_ITEMS];
#pragma unroll
        for (int j = 0; j < SORT_ITEMS; ++j) {
            const int64_t i = t0 + j * SORT_THREADS + threadIdx.x;
            d[j] = i < end ? (s.kin[i] >> s.shift) & (RADIX - 1) : (uint32_t)RADIX;
        }
#pragma unroll
        for (int j = 0; j < SORT_ITEMS; ++j)
            if (d[j] < RADIX) atomicAdd(&h[d[j]], 1u);
    }
    __syncthreads();
    s.hist[threadIdx.x * s.G + blockIdx.x] = h[threadIdx.x];
}

// Key bases of the counting sort (exclusive scan, in place, of the key
// totals tot[0..nkeys)), the range of every key (empty for an empty key, and
// for all keys over capacity), the total and the capacity check; by one block.
struct KeyBases {
    uint32_t *done;      // rows finished (zeroed before); NULL: no key bases
    int64_t capacity;
    int64_t *d_count, *n_eff;
    int32_t *d_err;
    uint32_t *ranges;
};

__device__ __forceinline__ int64_t block_scan_i64(int64_t x, int64_t *s_warp, int64_t &total);

__device__ __forceinline__ void key_bases(uint32_t *tot, int nkeys, KeyBases kb)
{
    __shared__ int64_t s_warp[32];
    const int nt = (int)blockDim.x;
    const int per = (nkeys + nt - 1) / nt;
    const int beg = min(nkeys, (int)threadIdx.x * per), end = min(nkeys, beg + per);
    int64_t sum = 0;
    for (int k = beg; k < end; ++k) sum += __ldcg(tot + k);
    int64_t total;
    int64_t run = block_scan_i64(sum, s_warp, total);
    const bool fits = total <= kb.capacity;
    for (int k = beg; k < end; ++k) {
        const uint32_t c = __ldcg(tot + k);
        const bool some = fits && c > 0;
        kb.ranges[2 * (int64_t)k] = some ? (uint32_t)run : 0u;
        kb.ranges[2 * (int64_t)k + 1] = some ? (uint32_t)(run + c) : 0u;
        tot[k] = (uint32_t)run;
        run += c;
    }
    if (threadIdx.x == 0) {
        *kb.d_count = total;
        *kb.n_eff = fits ? total : 0;
        if (!fits && kb.d_err) atomicCAS(kb.d_err, 0, (int32_t)GS_ERR_CAPACITY);
    }
}

constexpr int ROW_ITEMS = 4;  // a row of up to SORT_THREADS x ROW_ITEMS counts is scanned in one step

// Per row d (one block each; a digit of a radix pass or a key of the
// counting sort): exclusive scan, in place, of the G block counts
// hist[d][0..G), and the row's total in hist[rows * G + d].  Nothing for a
// radix pass whose byte is constant (kor, shift as in SortPass).  With
// kb.done, the block that finishes last also takes the key bases of the
// totals (the others' rows and totals are fenced before they count).
__global__ void __launch_bounds__(SORT_THREADS, 1) scan_digit_rows_kernel(uint32_t *hist, int G, int rows,
                                                                      const uint32_t *kor, int shift,
                                                                      KeyBases kb)
{
    if (byte_constant(kor, shift)) return;  // a radix pass that is skipped
    __shared__ uint32_t s_w[SORT_WARPS];
    __shared__ uint32_t s_carry;
    __shared__ int s_last;
    const int d = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t *row = hist + (int64_t)d * G;
    uint32_t total;
    if (G <= SORT_THREADS * ROW_ITEMS) {
        // each thread a run of up to ROW_ITEMS consecutive counts, all loaded at once
        const int per = (G + SORT_THREADS - 1) / SORT_THREADS;
        const int b0 = threadIdx.x * per;
        uint32_t x[ROW_ITEMS];
        uint32_t sum = 0u;
#pragma unroll
        for (int k = 0; k < ROW_ITEMS; ++k) {
            x[k] = k < per && b0 + k < G ? row[b0 + k] : 0u;
            sum += x[k];
        }
        uint32_t inc = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) s_w[warp] = inc;
        __syncthreads();
        uint32_t before = 0u;
        total = 0u;
#pragma unroll
        for (int w = 0; w < SORT_WARPS; ++w) {
            const uint32_t c = s_w[w];
            before += w < warp ? c : 0u;
            total += c;
        }
        uint32_t run = before + inc - sum;
#pragma unroll
        for (int k = 0; k < ROW_ITEMS; ++k) {
            if (k < per && b0 + k < G) row[b0 + k] = run;
            run += x[k];
        }
    } else {
        if (threadIdx.x == 0) s_carry = 0;
        __syncthreads();
        for (int base = 0; base < G; base += SORT_THREADS) {
            int i = base + threadIdx.x;
            uint32_t x = i < G ? row[i] : 0u;
            uint32_t inc = x;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            if (lane == 31) s_w[warp] = inc;
            __syncthreads();
            uint32_t before = s_carry;
            for (int w = 0; w < warp; ++w) before += s_w[w];
            if (i < G) row[i] = before + inc - x;
            __syncthreads();
            if (threadIdx.x == SORT_THREADS - 1) s_carry = before + inc;
            __syncthreads();
        }
        total = s_carry;
    }
    if (threadIdx.x == 0) hist[(int64_t)rows * G + d] = total;
    if (kb.done == nullptr) return;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(kb.done, 1u) == (uint32_t)(rows - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    key_bases(hist + (int64_t)rows * G, rows, kb);
}

// Ranked scatter of one pass.  Each tile of SORT_TILE items is first put in
// digit order in shared memory (stable), then written out so consecutive
// threads store consecutive positions of each digit's run (coalesced).
__global__ void __launch_bounds__(SORT_THREADS, 4) radix_scatter_kernel(SortPass s)
{
    __shared__ uint32_t s_off[RADIX];
    __shared__ uint32_t s_tot[RADIX];
    __shared__ uint32_t s_lst[RADIX];
    __shared__ uint32_t s_ws[SORT_WARPS];
    __shared__ uint32_t s_wh[SORT_WARPS][RADIX];
    __shared__ uint32_t s_k[SORT_TILE], s_v[SORT_TILE];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned lt = (1u << lane) - 1u;
    if (byte_constant(s.kor, s.shift)) return;
    pass_buffers(s);
    const int64_t n = pass_n(s);
    int64_t beg, end;
    block_range(n, s.G, blockIdx.x, beg, end);
    // the block's counts and the first tile's items are loaded before
    // anything waits; each later tile's while the one before is written out
    const uint32_t tot = s.hist[(int64_t)RADIX * s.G + tid];
    const uint32_t mine = s.hist[(int64_t)tid * s.G + blockIdx.x];
    uint32_t key[SORT_ITEMS], val[SORT_ITEMS];
    auto load_tile = [&](int64_t t0) {
#pragma unroll
        for (int j = 0; j < SORT_ITEMS; ++j) {
            const int64_t idx = t0 + (int64_t)warp * 32 * SORT_ITEMS + j * 32 + lane;
            const bool ok = idx < end;
            key[j] = ok ? s.kin[idx] : 0u;
            val[j] = ok ? s.vin[idx] : 0u;
        }
    };
    if (beg < end) load_tile(beg);
    {
        // digit base = exclusive scan of the digit totals (RADIX == threads)
        // one digit holds every item: the pass keeps the order, a copy
        if (!s.kor && __syncthreads_or((int64_t)tot == n)) {
            // 16 bytes a load where the buffers allow it (beg is a multiple
            // of SORT_TILE; a caller's vals may be only 4-byte aligned), all
            // of a thread's loads before its stores
            const bool vec = ((reinterpret_cast<uintptr_t>(s.kin) | reinterpret_cast<uintptr_t>(s.vin) |
                               reinterpret_cast<uintptr_t>(s.kout) | reinterpret_cast<uintptr_t>(s.vout)) &
                              15) == 0;
            const int64_t n4 = vec ? max((int64_t)0, end - beg) >> 2 : 0;
            const uint4 *k4 = reinterpret_cast<const uint4 *>(s.kin + beg);
            const uint4 *v4 = reinterpret_cast<const uint4 *>(s.vin + beg);
            uint4 *ko = reinterpret_cast<uint4 *>(s.kout + beg);
            uint4 *vo = reinterpret_cast<uint4 *>(s.vout + beg);
            for (int64_t i0 = 0; i0 < n4; i0 += 2 * SORT_THREADS) {
                const int64_t i = i0 + tid, j = i + SORT_THREADS;
                uint4 a = {}, b = {}, c = {}, d = {};
                if (i < n4) { a = k4[i]; b = v4[i]; }
                if (j < n4) { c = k4[j]; d = v4[j]; }
                if (i < n4) { ko[i] = a; vo[i] = b; }
                if (j < n4) { ko[j] = c; vo[j] = d; }
            }
            for (int64_t i = beg + 4 * n4 + tid; i < end; i += SORT_THREADS) {
                s.kout[i] = s.kin[i];
                s.vout[i] = s.vin[i];
            }
            return;
        }
        uint32_t inc = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) s_tot[warp] = inc;
        __syncthreads();
        uint32_t before = 0;
        for (int w = 0; w < warp; ++w) before += s_tot[w];
        s_off[tid] = before + inc - tot + mine;
    }
    for (int64_t t0 = beg; t0 < end; t0 += SORT_TILE) {
        for (int k = tid; k < SORT_WARPS * RADIX; k += SORT_THREADS) (&s_wh[0][0])[k] = 0u;
        __syncthreads();
        uint32_t rank[SORT_ITEMS], dig[SORT_ITEMS];
#pragma unroll
        for (int j = 0; j < SORT_ITEMS; ++j) {
            const int64_t idx = t0 + (int64_t)warp * 32 * SORT_ITEMS + j * 32 + lane;
            dig[j] = idx < end ? digit_of(s, key[j], val[j]) : (uint32_t)RADIX;
        }
#pragma unroll
        for (int j = 0; j < SORT_ITEMS; ++j) {
            const uint32_t d = dig[j];
            const bool ok = d < RADIX;
            unsigned peers = ballot_match<8>(d, ok);
            uint32_t before = 0;
            if (ok) before = s_wh[warp][d];
            __syncwarp();
            if (ok && lane == __ffs(peers) - 1) s_wh[warp][d] = before + __popc(peers);
            __syncwarp();
            rank[j] = before + __popc(peers & lt);
        }
        __syncthreads();
        {
            uint32_t run = 0;
#pragma unroll
            for (int w = 0; w < SORT_WARPS; ++w) {
                uint32_t c = s_wh[w][tid];
                s_wh[w][tid] = run;
                run += c;
            }
            s_tot[tid] = run;
            // block-local start of digit tid: exclusive scan of the totals
            uint32_t inc = run;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            if (lane == 31) s_ws[warp] = inc;
            __syncthreads();
            uint32_t before = 0;
            for (int w = 0; w < warp; ++w) before += s_ws[w];
            s_lst[tid] = before + inc - run;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < SORT_ITEMS; ++j) {
            uint32_t d = dig[j];
            if (d < RADIX) {
                uint32_t lp = s_lst[d] + s_wh[warp][d] + rank[j];
                s_k[lp] = key[j];
                s_v[lp] = val[j];
            }
        }
        __syncthreads();
        if (t0 + SORT_TILE < end) load_tile(t0 + SORT_TILE);
        const int cnt = (int)min((int64_t)SORT_TILE, end - t0);
        for (int i = tid; i < cnt; i += SORT_THREADS) {
            const uint32_t k = s_k[i], v = s_v[i];
            const uint32_t d = digit_of(s, k, v);
            const uint32_t pos = s_off[d] + ((uint32_t)i - s_lst[d]);
            s.kout[pos] = k;
            s.vout[pos] = v;
        }
        __syncthreads();
        s_off[tid] += s_tot[tid];
    }
}

// ---------------------------------------------------------------- stage 1
// Keys (IEEE bits of the positive depths, which are monotone; culled entries
// last) and values (the entry index) of the depth sort, with the first
// pass's block counts hist[d][G] (the blocks of block_range) and the keys'
// OR and complements' OR in kor[0..1] (zeroed before).
__global__ void __launch_bounds__(SORT_THREADS) depth_keys_kernel(const float *depth, const int32_t *radius,
                                                                  int64_t NV, int G, uint32_t *k, uint32_t *v,
                                                                  uint32_t *hist, uint32_t *kor)
{
    __shared__ uint32_t h[RADIX];
    __shared__ uint32_t s_or[2];
    h[threadIdx.x] = 0u;
    if (threadIdx.x < 2) s_or[threadIdx.x] = 0u;
    __syncthreads();
    int64_t beg, end;
    block_range(NV, G, blockIdx.x, beg, end);
    uint32_t o1 = 0u, o0 = 0u;
    for (int64_t t0 = beg; t0 < end; t0 += SORT_TILE) {
        uint32_t key[SORT_ITEMS];
#pragma unroll
        for (int j = 0; j < SORT_ITEMS; ++j) {
            const int64_t i = t0 + j * SORT_THREADS + threadIdx.x;
            key[j] = 0u;
            if (i < end) key[j] = radius[i] > 0 ? __float_as_uint(depth[i]) : 0xffffffffu;
        }
#pragma unroll
        for (int j = 0; j < SORT_ITEMS; ++j) {
            const int64_t i = t0 + j * SORT_THREADS + threadIdx.x;
            if (i < end) {
                k[i] = key[j];
                v[i] = (uint32_t)i;
                o1 |= key[j];
                o0 |= ~key[j];
                atomicAdd(&h[key[j] & (RADIX - 1)], 1u);
            }
        }
    }
    o1 = __reduce_or_sync(0xffffffffu, o1);
    o0 = __reduce_or_sync(0xffffffffu, o0);
    if ((threadIdx.x & 31) == 0) {
        atomicOr(&s_or[0], o1);
        atomicOr(&s_or[1], o0);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * G + blockIdx.x] = h[threadIdx.x];
    if (threadIdx.x == 0) {
        if (s_or[0]) atomicOr(kor, s_or[0]);
        if (s_or[1]) atomicOr(kor + 1, s_or[1]);
    }
}

// Number of bins of every entry, in the sorted order (same rectangle rule as
// the emission below and as gs_project's tiles_touched).
__global__ void sorted_counts_kernel(const uint32_t *svals, const float2 *mean2d,
                                     const int32_t *radius, int64_t NV, int tx, int ty, int bin,
                                     int32_t *cnt)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NV) return;
    uint32_t sv = svals[i];
    int r = radius[sv];
    int c = 0;
    if (r > 0) {
        float2 m = mean2d[sv];
        int x0, y0, x1, y1;
        bin_rect(m.x, m.y, r, tx, ty, bin, x0, y0, x1, y1);
        c = (x1 - x0) * (y1 - y0);
    }
    cnt[i] = c;
}

// ------------------------------------------------- scan of tile counts
__device__ __forceinline__ int64_t block_scan_i64(int64_t x, int64_t *s_warp, int64_t &total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int64_t w = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        s_warp[lane] = w;
    }
    __syncthreads();
    int64_t before = warp > 0 ? s_warp[warp - 1] : 0;
    total = s_warp[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before + inc - x;
}

__global__ void __launch_bounds__(SCAN_THREADS) count_reduce_kernel(const int32_t *cnt, int64_t NV,
                                                                    int64_t *bsum)
{
    __shared__ int64_t s_warp[32];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
    int64_t sum = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k)
        if (base + k < NV) sum += cnt[base + k];
    int64_t total;
    block_scan_i64(sum, s_warp, total);
    if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

// Exclusive scan of the block sums; total count, capacity check, n_eff.
__global__ void __launch_bounds__(SCAN_THREADS) count_top_kernel(int64_t *bsum, int nb,
                                                                 int64_t capacity, int64_t *d_count,
                                                                 int64_t *n_eff, int32_t *d_err)
{
    __shared__ int64_t s_warp[32];
    int per = (nb + SCAN_THREADS - 1) / SCAN_THREADS;
    int beg = threadIdx.x * per, end = min(nb, beg + per);
    int64_t sum = 0;
    for (int i = beg; i < end; ++i) sum += bsum[i];
    int64_t total;
    int64_t run = block_scan_i64(sum, s_warp, total);
    for (int i = beg; i < end; ++i) {
        int64_t x = bsum[i];
        bsum[i] = run;
        run += x;
    }
    if (threadIdx.x == 0) {
        *d_count = total;
        bool fits = total <= capacity;
        *n_eff = fits ? total : 0;
        if (!fits && d_err) atomicCAS(d_err, 0, (int32_t)GS_ERR_CAPACITY);
    }
}

__global__ void __launch_bounds__(SCAN_THREADS) count_down_kernel(const int32_t *cnt, int64_t NV,
                                                                  const int64_t *bsum,
                                                                  int64_t *offsets)
{
    __shared__ int64_t s_warp[32];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
    int64_t c[SCAN_ITEMS];
    int64_t sum = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        c[k] = (base + k < NV) ? cnt[base + k] : 0;
        sum += c[k];
    }
    int64_t total;
    int64_t run = block_scan_i64(sum, s_warp, total) + bsum[blockIdx.x];
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        if (base + k < NV) offsets[base + k] = run;
        run += c[k];
    }
}

// ------------------------------------------------------------- emission
struct EmitParams {
    const uint32_t *svals;  // sorted (view, Gaussian) entries: view * n + g
    const int64_t *offsets;
    const int64_t *n_eff;
    const float2 *mean2d;
    const int32_t *radius;
    int64_t NV, n;
    int tx, ty, bin, bins_x, bins;
    uint32_t *tkeys, *tvals;
};

// A warp's 32 consecutive entries own one contiguous output range; lanes
// stride over it so the key/value stores are coalesced.
__global__ void __launch_bounds__(256) emit_kernel(EmitParams e)
{
    if (*e.n_eff == 0) return;  // nothing to emit, or over capacity
    const int lane = threadIdx.x & 31;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool ok = i < e.NV;
    uint32_t sv = ok ? e.svals[i] : 0u;
    int64_t off = ok ? e.offsets[i] : 0;
    int x0 = 0, y0 = 0, x1 = 0, y1 = 0;
    if (ok) {
        int r = e.radius[sv];
        if (r > 0) {
            float2 m = e.mean2d[sv];
            bin_rect(m.x, m.y, r, e.tx, e.ty, e.bin, x0, y0, x1, y1);
        }
    }
    int w = x1 - x0;
    int64_t cnt = (int64_t)w * (y1 - y0);
    unsigned okmask = __ballot_sync(0xffffffffu, ok);
    if (okmask == 0u) return;  // warp-uniform: the whole warp is past the end
    int lastl = 31 - __clz(okmask);
    // lanes past the end take the warp's end offset so offsets stay monotone
    int64_t wend = __shfl_sync(0xffffffffu, off + cnt, lastl);
    if (!ok) off = wend;
    int64_t wbeg = __shfl_sync(0xffffffffu, off, 0);
    uint32_t view = sv / (uint32_t)e.n;
    uint32_t g = sv - view * (uint32_t)e.n;
    uint32_t kbase = view * (uint32_t)e.bins;
    int64_t span = wend - wbeg;
    for (int64_t k0 = 0; k0 < span; k0 += 32) {
        int64_t o = wbeg + k0 + lane;
        int src = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            int cand = src + step;
            int64_t oc = __shfl_sync(0xffffffffu, off, cand);
            if (oc <= o) src = cand;
        }
        int64_t so = __shfl_sync(0xffffffffu, off, src);
        int sw = __shfl_sync(0xffffffffu, w, src);
        int sx = __shfl_sync(0xffffffffu, x0, src);
        int sy = __shfl_sync(0xffffffffu, y0, src);
        uint32_t sk = __shfl_sync(0xffffffffu, kbase, src);
        uint32_t sg = __shfl_sync(0xffffffffu, g, src);
        if (o < wend) {
            int local = (int)(o - so);
            int ty = sy + local / sw;
            int tx = sx + local - (local / sw) * sw;
            e.tkeys[o] = sk + (uint32_t)(ty * e.bins_x + tx);
            e.tvals[o] = sg;
        }
    }
}

__global__ void ranges_kernel(const uint32_t *tk, const int64_t *n_eff, uint32_t *ranges)
{
    int64_t n = *n_eff;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t k = tk[i];
        if (i == 0 || tk[i - 1] != k) ranges[2 * (int64_t)k] = (uint32_t)i;
        if (i == n - 1 || tk[i + 1] != k) ranges[2 * (int64_t)k + 1] = (uint32_t)(i + 1);
    }
}

__global__ void keys64_kernel(const uint32_t *tk, const uint32_t *vals, const int64_t *n_eff,
                              const float *depth, int64_t n, int tiles, uint64_t *keys)
{
    int64_t cnt = *n_eff;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t k = tk[i];
        int64_t view = k / (uint32_t)tiles;
        uint32_t db = __float_as_uint(depth[view * n + vals[i]]);
        keys[i] = ((uint64_t)k << 32) | db;
    }
}

// ------------------------------------------- stage 2 as a counting sort
// When the per-warp key tables fit in shared memory, stage 2 sorts the pairs
// by key without materialising them.  Every warp owns a contiguous segment of
// the depth-ordered entries and walks their pairs in order, 32 pair slots per
// step (an entry's pairs are its bin rectangle, row by row):
//  - count: each slot adds one to its key's 16-bit counter in the warp's
//    table (two counters per 32-bit word; a warp's count of one key is at
//    most its CS_MAX_ENTRIES entries).  The block then writes, per key, each
//    warp's exclusive prefix over the block's warps to wpre[warp][key] and
//    the block's total to hist[key][block], and every entry's bin rectangle
//    and view, packed, to rect[entry].
//  - scan: per key, exclusive over the blocks (scan_digit_rows_kernel), then
//    over the keys (by the scan's last block), giving each (block, key) its first
//    position, each key its range, the total and the capacity check.
//  - place: each block keeps per key its first position (32 bits) and per
//    (warp, key) a running offset from it (16 bits: a block's count of one
//    key is below 2^16), and each warp walks its pairs again, each placed at
//    its key's running position; within a step the slots of one key are
//    ranked by lane (ballot_match: one ballot per key bit), which a step whose
//    slots all belong to one entry (distinct keys) skips.
// Every list then holds its pairs in the entries' depth order: the same
// result as the stable key sort, bit for bit.
constexpr int CS_WARPS = 16;
constexpr int CS_THREADS = CS_WARPS * 32;
constexpr int CS_MAX_KEYS = 2048;        // keys V * bins at most (16-bit tables: 64 KB per block)
constexpr int CS_MIN_ENTRIES = 64;       // entries per warp at least (bounds the count tables)
constexpr int CS_MAX_ENTRIES = 4095;     // entries per warp at most: CS_WARPS x 4095 < 2^16 per block and key
constexpr int CS_BLOCKS_PER_SM = 4;
constexpr int CS_COUNT_MIN_BLOCKS = 3;   // count kernel: 42 registers, room for its loads run ahead

// Keys padded to a multiple of 8, so a warp's 16-bit row is whole 16-byte words.
inline int cs_pad_keys(int64_t nkeys) { return (int)((nkeys + 7) & ~int64_t(7)); }

// Warps of the counting sort for NV entries on this device (a multiple of
// CS_WARPS), and the bound of that number used to size the workspace
// without a device.
inline int64_t cs_warps(int64_t NV, int sms)
{
    const int64_t want = std::max<int64_t>(1, ceil_div(NV, CS_MIN_ENTRIES));
    const int64_t cap = std::max<int64_t>((int64_t)sms * CS_BLOCKS_PER_SM * CS_WARPS,
                                          ceil_div(NV, CS_MAX_ENTRIES));
    return ceil_div(std::min(want, cap), CS_WARPS) * CS_WARPS;
}
inline int64_t cs_warps_bound(int64_t NV)
{
    return ceil_div(std::max<int64_t>(1, ceil_div(NV, CS_MIN_ENTRIES)), CS_WARPS) * CS_WARPS;
}

struct CsParams {
    const uint32_t *svals;   // sorted (view, Gaussian) entries: view * n + g
    const uint32_t *kor;     // with it, svals is sv[f & 1], f the depth passes not skipped
    const uint32_t *sv[2];
    const float2 *mean2d;
    const int32_t *radius;
    const float *depth;
    int64_t NV, n;
    float inv_n, inv_bin;    // 1/n and 1/bin, rounded to FP32
    int tx, ty, bin, bins_x, bins, V;
    int nkeys, kp;           // V * bins, and padded to a multiple of 8
    int64_t NW;              // warps, G = NW / CS_WARPS blocks
    uint32_t *hist;          // [nkeys][G] block counts -> prefixes, then per key [nkeys] totals -> bases
    uint16_t *wpre;          // [NW][kp] warp offsets within the block
    uint64_t *rect;          // [NV] packed bin rectangle and view of every entry
    uint32_t *done;          // zeroed by the count kernel for the scan after it
    const int64_t *n_eff;
    uint32_t *vals;
    uint64_t *keys;          // optional
};

__device__ __forceinline__ const uint32_t *cs_svals(const CsParams &p)
{
    if (!p.kor) return p.svals;
    return (passes_below(p.kor, 32) & 1) ? p.sv[1] : p.sv[0];
}

__device__ __forceinline__ void cs_segment(const CsParams &p, int64_t &beg, int64_t &end)
{
    const int64_t gw = (int64_t)blockIdx.x * CS_WARPS + (threadIdx.x >> 5);
    const int64_t per = (p.NV + p.NW - 1) / p.NW;
    beg = min(p.NV, gw * per);
    end = min(p.NV, beg + per);
}

// floor(x / d) for 0 <= x, d < 2^12 from r = fl(1/d): q = (x + 1/2) / d is
// at least 1/(2d) from every integer, and the FP32 product (x + 1/2) r is
// within q 2^-23 < 2^-11 / d of q, so it truncates to floor(q) = floor(x / d).
__device__ __forceinline__ int cs_div(int x, float r)
{
    return (int)__fmul_rn(__fadd_rn((float)x, 0.5f), r);
}

// View of entry sv = view * n + g: the FP32 estimate is within 1 of it
// (sv / n < 64, relative error about 2^-22), one correction makes it exact.
__device__ __forceinline__ uint32_t cs_view(const CsParams &p, uint32_t sv)
{
    uint32_t v = min((uint32_t)(p.V - 1), (uint32_t)__fmul_rn((float)sv, p.inv_n));
    if (v * (uint32_t)p.n > sv) --v;
    else if ((v + 1u) * (uint32_t)p.n <= sv) ++v;
    return v;
}

// Packed bin rectangle and view of entry sv (an empty rectangle for a culled
// entry): bin_rect() with the divisions by bin taken by cs_div (tiles < 2^12);
// x0, x1, y0, y1 in 12 bits each (bins <= 1024 a side), the view above them.
__device__ __forceinline__ uint64_t cs_rect(const CsParams &p, uint32_t sv, int r, float2 m)
{
    int x0 = 0, y0 = 0, x1 = 0, y1 = 0;
    if (r > 0) {
        int a0, b0, a1, b1;
        tile_rect(m.x, m.y, r, p.tx, p.ty, a0, b0, a1, b1);
        if (a1 > a0 && b1 > b0) {
            x0 = cs_div(a0, p.inv_bin);
            y0 = cs_div(b0, p.inv_bin);
            x1 = cs_div(a1 - 1, p.inv_bin) + 1;
            y1 = cs_div(b1 - 1, p.inv_bin) + 1;
        }
    }
    return (uint64_t)x0 | ((uint64_t)x1 << 12) | ((uint64_t)y0 << 24) | ((uint64_t)y1 << 36) |
           ((uint64_t)cs_view(p, sv) << 48);
}

// 32 entries of a warp's segment (one per lane), compacted: lane j < nent
// holds the j-th entry with pairs: its first slot, first key | width << 16,
// Gaussian index and 1/width.
struct CsChunk {
    int total, nent, off, kw;
    uint32_t gi;
    float rw;
};

__device__ __forceinline__ CsChunk cs_chunk(const CsParams &p, uint32_t sv, uint64_t rc, uint8_t *idx)
{
    const int lane = threadIdx.x & 31;
    const int x0 = (int)(rc & 0xfff), x1 = (int)((rc >> 12) & 0xfff);
    const int y0 = (int)((rc >> 24) & 0xfff), y1 = (int)((rc >> 36) & 0xfff);
    const uint32_t view = (uint32_t)(rc >> 48);
    const int w = x1 - x0, cnt = w * (y1 - y0);
    int inc = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    CsChunk c;
    c.total = __shfl_sync(0xffffffffu, inc, 31);
    const unsigned nz = __ballot_sync(0xffffffffu, cnt > 0);
    c.nent = __popc(nz);
    if (cnt > 0) idx[__popc(nz & ((1u << lane) - 1u))] = (uint8_t)lane;
    __syncwarp();
    const int src = lane < c.nent ? idx[lane] : 0;
    __syncwarp();
    c.off = __shfl_sync(0xffffffffu, inc - cnt, src);
    c.kw = __shfl_sync(0xffffffffu, ((int)view * p.bins + y0 * p.bins_x + x0) | (w << 16), src);
    c.gi = __shfl_sync(0xffffffffu, sv - view * (uint32_t)p.n, src);
    c.rw = __shfl_sync(0xffffffffu, cnt > 0 ? __frcp_rn((float)w) : 0.f, src);
    return c;
}

// Key of pair slot s0 + lane of a chunk (-1 past its end) and the slot's
// entry j (compacted; `before` counts the entries that start before s0 and
// is advanced past this step).  single: every slot of the step belongs to one
// entry.
__device__ __forceinline__ int cs_slot(const CsParams &p, const CsChunk &c, int s0, int &before, int &j,
                                       bool &single)
{
    const int lane = threadIdx.x & 31;
    // the entry of slot o: the last one whose first slot is <= o
    const bool starts = lane < c.nent && c.off >= s0 && c.off < s0 + 32;
    const unsigned B = __reduce_or_sync(0xffffffffu, starts ? 1u << (c.off - s0) : 0u);
    j = max(0, before + __popc(B & ((2u << lane) - 1u)) - 1);
    before += __popc(B);
    single = (B & ~1u) == 0u;
    const int so = __shfl_sync(0xffffffffu, c.off, j);
    const int skw = __shfl_sync(0xffffffffu, c.kw, j);
    const float srw = __shfl_sync(0xffffffffu, c.rw, j);
    const int o = s0 + lane;
    if (o >= c.total) return -1;
    const int local = o - so, sw = skw >> 16;
    const int dy = cs_div(local, srw);  // local < bins <= CS_MAX_KEYS, sw <= bins_x
    return (skw & 0xffff) + dy * p.bins_x + (local - dy * sw);
}

__global__ void __launch_bounds__(CS_THREADS, CS_COUNT_MIN_BLOCKS) cs_count_kernel(CsParams p)
{
    extern __shared__ uint32_t s_cnt[];      // [CS_WARPS][kp / 2]: two 16-bit counters a word
    __shared__ uint8_t s_idx[CS_WARPS][32];  // lanes of the entries with pairs
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int kw2 = p.kp >> 1;
    if (blockIdx.x == 0 && threadIdx.x == 0) *p.done = 0u;
    uint32_t *cnt = s_cnt + warp * kw2;
    for (int k = lane; k < kw2; k += 32) cnt[k] = 0u;
    __syncwarp();
    int64_t beg, end;
    cs_segment(p, beg, end);
    // loads run ahead of the counting: the entries two chunks ahead, the
    // radii and means of the next chunk's entries
    const uint32_t *svals = cs_svals(p);
    uint32_t sv_a = beg + lane < end ? svals[beg + lane] : 0u;
    uint32_t sv_b = beg + 32 + lane < end ? svals[beg + 32 + lane] : 0u;
    int r_a = beg + lane < end ? p.radius[sv_a] : 0;
    float2 m_a = r_a > 0 ? p.mean2d[sv_a] : make_float2(0.f, 0.f);
    for (int64_t e0 = beg; e0 < end; e0 += 32) {
        const int64_t i = e0 + lane;
        const uint32_t sv = sv_a;
        const int r = r_a;
        const float2 m = m_a;
        sv_a = sv_b;
        r_a = e0 + 32 + lane < end ? p.radius[sv_a] : 0;
        m_a = r_a > 0 ? p.mean2d[sv_a] : make_float2(0.f, 0.f);
        sv_b = e0 + 64 + lane < end ? svals[e0 + 64 + lane] : 0u;
        uint64_t rc = 0;
        if (i < end) {
            rc = cs_rect(p, sv, r, m);
            p.rect[i] = rc;
        }
        const CsChunk c = cs_chunk(p, i < end ? sv : 0u, rc, s_idx[warp]);
        int before = 0;
        for (int s0 = 0; s0 < c.total; s0 += 32) {
            int j;
            bool single;
            const int key = cs_slot(p, c, s0, before, j, single);
            if (key >= 0) atomicAdd(&cnt[key >> 1], 1u << ((key & 1) << 4));
        }
    }
    __syncthreads();
    // per pair of keys: each warp's offset within the block (exclusive over
    // the warps, both halves at once: no half exceeds 2^16 - 1) and the
    // block's counts
    const int G = (int)(p.NW / CS_WARPS);
    uint32_t *pre = reinterpret_cast<uint32_t *>(p.wpre) + (int64_t)blockIdx.x * CS_WARPS * kw2;
    for (int k2 = threadIdx.x; k2 < kw2; k2 += CS_THREADS) {
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < CS_WARPS; ++w) {
            const uint32_t x = s_cnt[w * kw2 + k2];
            pre[(int64_t)w * kw2 + k2] = run;
            run += x;
        }
        const int key = 2 * k2;
        if (key < p.nkeys) p.hist[(int64_t)key * G + blockIdx.x] = run & 0xffffu;
        if (key + 1 < p.nkeys) p.hist[(int64_t)(key + 1) * G + blockIdx.x] = run >> 16;
    }
}

__global__ void __launch_bounds__(CS_THREADS) cs_place_kernel(CsParams p)
{
    // per key the block's first position, then per (warp, key) the running
    // offset from it
    extern __shared__ __align__(16) uint32_t s_base[];
    uint16_t *s_off = reinterpret_cast<uint16_t *>(s_base + p.kp);
    __shared__ uint8_t s_idx[CS_WARPS][32];  // lanes of the entries with pairs
    if (*p.n_eff == 0) return;               // nothing to place, or over capacity
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    int64_t beg, end;
    cs_segment(p, beg, end);
    // the next 32 entries are loaded while the present ones are placed
    const uint32_t *svals = cs_svals(p);
    uint32_t sv_next = 0;
    uint64_t rc_next = 0;
    if (beg + lane < end) {
        sv_next = svals[beg + lane];
        rc_next = p.rect[beg + lane];
    }
    {
        const int G = (int)(p.NW / CS_WARPS);
        const uint32_t *base = p.hist + (int64_t)p.nkeys * G;
        for (int key = threadIdx.x; key < p.nkeys; key += CS_THREADS)
            s_base[key] = base[key] + p.hist[(int64_t)key * G + blockIdx.x];
        // the warp's own row of offsets, 16 bytes a lane
        const uint4 *src = reinterpret_cast<const uint4 *>(p.wpre + ((int64_t)blockIdx.x * CS_WARPS + warp) * p.kp);
        uint4 *dst = reinterpret_cast<uint4 *>(s_off + warp * p.kp);
        for (int k = lane; k < (p.kp >> 3); k += 32) dst[k] = src[k];
    }
    __syncthreads();
    uint16_t *g = s_off + warp * p.kp;
    for (int64_t e0 = beg; e0 < end; e0 += 32) {
        const uint32_t sv = sv_next;
        const uint64_t rc = rc_next;
        sv_next = 0;
        rc_next = 0;
        if (e0 + 32 + lane < end) {
            sv_next = svals[e0 + 32 + lane];
            rc_next = p.rect[e0 + 32 + lane];
        }
        const CsChunk c = cs_chunk(p, sv, rc, s_idx[warp]);
        int before = 0;
        for (int s0 = 0; s0 < c.total; s0 += 32) {
            int j;
            bool single;
            const int key = cs_slot(p, c, s0, before, j, single);
            const uint32_t sgi = __shfl_sync(0xffffffffu, c.gi, j);
            const bool valid = key >= 0;
            // slots of one key in this step, ranked by lane
            const unsigned peers = single ? 1u << lane : ballot_match<11>((uint32_t)key, valid);
            uint32_t pos = 0;
            if (valid) pos = s_base[key] + g[key] + __popc(peers & lt);
            __syncwarp();
            if (valid && lane == __ffs(peers) - 1) g[key] = (uint16_t)(g[key] + __popc(peers));
            __syncwarp();
            if (valid) {
                p.vals[pos] = sgi;
                if (p.keys)
                    p.keys[pos] = ((uint64_t)(uint32_t)key << 32) |
                                  __float_as_uint(p.depth[(int64_t)(key / p.bins) * p.n + sgi]);
            }
        }
    }
}

// ------------------------------------------------------------- workspace
struct BinWs {
    uint32_t *dk[2], *dv[2];
    int64_t *offsets, *bsum;
    int32_t *cnt;
    uint32_t *hist;
    int64_t *n_eff;
    uint32_t *kor;     // the depth keys' OR and their complements' OR
    uint32_t *done;    // rows of the counting sort's scan finished
    uint32_t *tk[2], *tv;
    uint64_t *rect;    // counting sort; shares its space with the emit path's buffers
    uint16_t *wpre;
    size_t bytes;
};

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

static BinWs carve(void *base, int64_t NV, int64_t cap)
{
    BinWs w{};
    char *p = reinterpret_cast<char *>(base);
    size_t o = 0;
    auto take = [&](size_t bytes) {
        char *r = p ? p + o : nullptr;
        o += align256(bytes);
        return r;
    };
    for (int k = 0; k < 2; ++k) w.dk[k] = reinterpret_cast<uint32_t *>(take(4 * NV));
    for (int k = 0; k < 2; ++k) w.dv[k] = reinterpret_cast<uint32_t *>(take(4 * NV));
    // the radix passes' digit counts, or the counting sort's per-block key counts
    const int64_t cw = cs_warps_bound(NV);
    const size_t hist_words = std::max<size_t>((size_t)RADIX * SORT_BLOCKS_MAX + RADIX,
                                               (size_t)CS_MAX_KEYS * (cw / CS_WARPS + 1));
    w.hist = reinterpret_cast<uint32_t *>(take(4 * hist_words));
    w.n_eff = reinterpret_cast<int64_t *>(take(64));
    w.kor = reinterpret_cast<uint32_t *>(take(8));
    w.done = reinterpret_cast<uint32_t *>(take(4));
    // stage 2 takes one of two paths: their buffers share one region
    const size_t region = o;
    w.offsets = reinterpret_cast<int64_t *>(take(8 * (NV + 1)));
    w.cnt = reinterpret_cast<int32_t *>(take(4 * NV));
    w.bsum = reinterpret_cast<int64_t *>(take(8 * (ceil_div(NV, SCAN_TILE) + 1)));
    for (int k = 0; k < 2; ++k) w.tk[k] = reinterpret_cast<uint32_t *>(take(4 * cap));
    w.tv = reinterpret_cast<uint32_t *>(take(4 * cap));
    const size_t emit_end = o;
    o = region;
    w.rect = reinterpret_cast<uint64_t *>(take(8 * NV));
    w.wpre = reinterpret_cast<uint16_t *>(take(2 * (size_t)CS_MAX_KEYS * cw));
    w.bytes = std::max(emit_end, o);
    return w;
}

// One radix pass; with counts false the block counts are already in s.hist.
static gs_status run_pass(SortPass s, cudaStream_t st, bool counts = true)
{
    if (counts) {
        note_launch();
        radix_hist_kernel<<<s.G, SORT_THREADS, 0, st>>>(s);
    }
    note_launch();
    scan_digit_rows_kernel<<<RADIX, SORT_THREADS, 0, st>>>(s.hist, s.G, RADIX, s.kor, s.shift, KeyBases{});
    note_launch();
    radix_scatter_kernel<<<s.G, SORT_THREADS, 0, st>>>(s);
    return launch_status("radix pass");
}

size_t radix_sort_hist_words() { return (size_t)RADIX * SORT_BLOCKS_MAX + RADIX; }

gs_status radix_sort_pairs(uint32_t *k[2], uint32_t *v[2], int64_t n, int bits, uint32_t *hist, int &cur,
                           cudaStream_t st)
{
    cur = 0;
    const int G = (int)std::min<int64_t>(sort_blocks(), std::max<int64_t>(1, ceil_div(n, SORT_TILE)));
    for (int shift = 0; shift < bits; shift += 8) {
        SortPass s{};
        s.kin = k[cur];
        s.vin = v[cur];
        s.kout = k[cur ^ 1];
        s.vout = v[cur ^ 1];
        s.d_n = nullptr;
        s.n_host = n;
        s.shift = shift;
        s.hist = hist;
        s.G = G;
        gs_status e = run_pass(s, st);
        if (e != GS_OK) return e;
        cur ^= 1;
    }
    return GS_OK;
}

}  // namespace gs3

using namespace gs3;

extern "C" size_t gs_bin_sort_workspace_size(int64_t n, int V, int W, int H, int64_t capacity)
{
    (void)W;
    (void)H;
    // n is bounded before n * V is formed (a wrapped product would pass)
    if (n < 0 || V < 1 || capacity < 0 || n > ((int64_t(1) << 32) - 2) / V) return 0;
    return carve(nullptr, n * V, capacity).bytes;
}

extern "C" gs_status gs_bin_sort(const gs_projected *proj, int64_t n, int V, int W, int H, int bin,
                                 int64_t capacity, uint32_t *vals, uint32_t *ranges, uint64_t *keys,
                                 int64_t *d_count, int32_t *d_err, void *ws, size_t ws_bytes,
                                 gs_stream stream)
{
    GS_REQUIRE(bin >= 1 && bin <= 64, "gs_bin_sort: bin must be 1..64 tiles");
    GS_REQUIRE(proj && vals && ranges && d_count && ws, "gs_bin_sort: null argument");
    GS_REQUIRE(n >= 0 && V >= 1 && V <= GS_MAX_VIEWS, "gs_bin_sort: bad n or V");
    GS_REQUIRE(W > 0 && H > 0 && W <= 16384 && H <= 16384, "gs_bin_sort: bad image size");
    GS_REQUIRE(n <= ((int64_t(1) << 32) - 2) / V, "gs_bin_sort: n * V must fit in 32 bits");
    GS_REQUIRE(capacity >= 0 && capacity < (int64_t(1) << 32) - 1,
               "gs_bin_sort: capacity must fit in 32 bits");
    GS_REQUIRE(aligned(ws, 256), "gs_bin_sort: workspace must be 256-byte aligned");
    const int64_t NV = n * V;
    BinWs w = carve(ws, NV, capacity);
    GS_REQUIRE(ws_bytes >= w.bytes, "gs_bin_sort: workspace too small (%zu < %zu)", ws_bytes,
               w.bytes);
    cudaStream_t st = as_stream(stream);
    const int tx = tiles_x_of(W), ty = tiles_y_of(H);
    const int bins_x = bins_x_of(W, bin);
    const int bins = bins_x * bins_y_of(H, bin);
    const int64_t nkeys = (int64_t)V * bins;
    // the counting sort writes every key's range; the other paths only the
    // non-empty ones
    if (NV == 0 || nkeys > CS_MAX_KEYS) cudaMemsetAsync(ranges, 0, sizeof(uint32_t) * 2 * nkeys, st);
    if (NV == 0) {
        cudaMemsetAsync(d_count, 0, sizeof(int64_t), st);
        return launch_status("gs_bin_sort");
    }
    // ---- stage 1: (view, depth) order of the V*N entries; before the
    // counting sort, the passes whose byte is the same in every key are
    // skipped and the kernels find their buffers on the device
    const bool cs = nkeys <= CS_MAX_KEYS;
    int cur = 0;
    const int Gd = (int)std::min<int64_t>(sort_blocks(), ceil_div(NV, SORT_TILE));
    cudaMemsetAsync(w.kor, 0, 2 * sizeof(uint32_t), st);
    note_launch();
    depth_keys_kernel<<<Gd, SORT_THREADS, 0, st>>>(proj->depth, proj->radius, NV, Gd, w.dk[0], w.dv[0], w.hist,
                                                   w.kor);
    // depth order only: stage 2 sorts stably on a key that holds the view,
    // so each (view, bin) list needs its view's entries in (depth, index)
    // order, not the views grouped
    for (int pass = 0; pass < 4; ++pass) {
        SortPass s{};
        s.kin = w.dk[cur];
        s.vin = w.dv[cur];
        s.kout = w.dk[cur ^ 1];
        s.vout = w.dv[cur ^ 1];
        s.d_n = nullptr;
        s.n_host = NV;
        s.shift = 8 * pass;
        s.hist = w.hist;
        s.G = Gd;
        if (cs) {
            s.kor = w.kor;
            for (int b = 0; b < 2; ++b) {
                s.kb[b] = w.dk[b];
                s.vb[b] = w.dv[b];
            }
        }
        gs_status e = run_pass(s, st, pass > 0);  // the keys kernel counted the first pass
        if (e != GS_OK) return e;
        cur ^= 1;
    }
    const uint32_t *svals = w.dv[cur];
    // ---- stage 2 as a counting sort when the per-warp key tables fit in shared memory
    if (cs) {
        CsParams cp{};
        cp.svals = svals;
        cp.kor = w.kor;
        cp.sv[0] = w.dv[0];
        cp.sv[1] = w.dv[1];
        cp.mean2d = reinterpret_cast<const float2 *>(proj->mean2d);
        cp.radius = proj->radius;
        cp.depth = proj->depth;
        cp.NV = NV;
        cp.n = n;
        cp.inv_n = 1.0f / (float)n;
        cp.inv_bin = 1.0f / (float)bin;
        cp.tx = tx;
        cp.ty = ty;
        cp.bin = bin;
        cp.bins_x = bins_x;
        cp.bins = bins;
        cp.V = V;
        cp.nkeys = (int)nkeys;
        cp.kp = cs_pad_keys(nkeys);
        cp.NW = cs_warps(NV, num_sms());
        const int G = (int)(cp.NW / CS_WARPS);
        cp.hist = w.hist;
        cp.wpre = w.wpre;
        cp.rect = w.rect;
        cp.done = w.done;
        cp.n_eff = w.n_eff;
        cp.vals = vals;
        cp.keys = keys;
        const int smem_count = CS_WARPS * (cp.kp / 2) * (int)sizeof(uint32_t);
        const int smem_place = cp.kp * (int)(sizeof(uint32_t) + CS_WARPS * sizeof(uint16_t));
        set_smem_limit((const void *)cs_count_kernel, smem_count, st);
        set_smem_limit((const void *)cs_place_kernel, smem_place, st);
        note_launch();
        cs_count_kernel<<<G, CS_THREADS, smem_count, st>>>(cp);
        note_launch();
        const KeyBases kb{w.done, capacity, d_count, w.n_eff, d_err, ranges};
        scan_digit_rows_kernel<<<(int)nkeys, SORT_THREADS, 0, st>>>(w.hist, G, (int)nkeys, nullptr, 0, kb);
        note_launch();
        cs_place_kernel<<<G, CS_THREADS, smem_place, st>>>(cp);
        return launch_status("gs_bin_sort");
    }
    // ---- otherwise: offsets of every entry's pairs in that order
    int nb = (int)ceil_div(NV, SCAN_TILE);
    note_launch();
    sorted_counts_kernel<<<(int)ceil_div(NV, 256), 256, 0, st>>>(
        svals, reinterpret_cast<const float2 *>(proj->mean2d), proj->radius, NV, tx, ty, bin, w.cnt);
    note_launch();
    count_reduce_kernel<<<nb, SCAN_THREADS, 0, st>>>(w.cnt, NV, w.bsum);
    note_launch();
    count_top_kernel<<<1, SCAN_THREADS, 0, st>>>(w.bsum, nb, capacity, d_count, w.n_eff, d_err);
    note_launch();
    count_down_kernel<<<nb, SCAN_THREADS, 0, st>>>(w.cnt, NV, w.bsum, w.offsets);
    // ---- stage 2: emit pairs, stable sort on the tile key
    int bits = 0;
    while ((int64_t(1) << bits) < nkeys) ++bits;
    int passes = (bits + 7) / 8;
    EmitParams ep{};
    ep.svals = svals;
    ep.offsets = w.offsets;
    ep.n_eff = w.n_eff;
    ep.mean2d = reinterpret_cast<const float2 *>(proj->mean2d);
    ep.radius = proj->radius;
    ep.NV = NV;
    ep.n = n;
    ep.tx = tx;
    ep.ty = ty;
    ep.bin = bin;
    ep.bins_x = bins_x;
    ep.bins = bins;
    ep.tkeys = w.tk[0];
    ep.tvals = (passes % 2 == 0) ? vals : w.tv;
    note_launch();
    emit_kernel<<<(int)ceil_div(NV, 256), 256, 0, st>>>(ep);
    gs_status e = launch_status("gs_bin_sort emit");
    if (e != GS_OK) return e;
    int kc = 0;
    uint32_t *vcur = ep.tvals;
    for (int pass = 0; pass < passes; ++pass) {
        SortPass s{};
        s.kin = w.tk[kc];
        s.vin = vcur;
        s.kout = w.tk[kc ^ 1];
        s.vout = (vcur == vals) ? w.tv : vals;
        s.d_n = w.n_eff;
        s.n_host = 0;
        s.shift = 8 * pass;
        s.hist = w.hist;
        s.G = sort_blocks();
        e = run_pass(s, st);
        if (e != GS_OK) return e;
        kc ^= 1;
        vcur = s.vout;
    }
    note_launch();
    ranges_kernel<<<num_sms() * 8, 256, 0, st>>>(w.tk[kc], w.n_eff, ranges);
    if (keys) {
        note_launch();
        keys64_kernel<<<num_sms() * 8, 256, 0, st>>>(w.tk[kc], vals, w.n_eff, proj->depth, n, bins,
                                                   keys);
    }
    return launch_status("gs_bin_sort");
}
