// Tile binning: the stable sort of (tile << 32 | depth bits, Gaussian) pairs
// that the tile-based rasterizer needs (Sec. 4 builds on the 3D-GS
// rasterizer), computed as an LSD radix sort whose low 32-bit digits are
// sorted before the pairs are expanded:
//   1. radix-sort the visible Gaussians by the 32 bits of their depth
//      (4 stable 8-bit passes over n keys, not over P pairs);
//   2. one stable counting pass on the tile digit over the P pairs: Gaussians
//      are cut, in depth order, into chunks of 256; per chunk and tile the
//      number of members comes from per-warp row/column bitmasks, a prefix
//      over (tile, chunk) gives each chunk's slot in every tile's range, and
//      each chunk writes its members tile by tile in depth order.
// Every pair of one Gaussian shares its depth bits, so sorting the depth
// digits on the Gaussians first and then the tile digit stably on the pairs is
// exactly the LSD order of the 64-bit key; the output equals the stable sort.
// qn_bin_sort_partial stops before writing the lists longer than list_max
// (with list_max 0, every list): the compositing forward forms them from the
// chunk masks, walking only the chunks that hold a member of its tile (a
// per-tile occupancy bitmap over the chunks, built with the tile totals).
#include <algorithm>
#include <mutex>

#include "bins.cuh"
#include "common.cuh"

namespace qn {
namespace {

constexpr int SORT_THREADS = 256;
constexpr int SORT_ITEMS = 8;
constexpr int SORT_TILE = SORT_THREADS * SORT_ITEMS;   // keys per block per pass
constexpr int RADIX = 256;
constexpr int CHUNK = BIN_CHUNK;                       // Gaussians per binning chunk
constexpr int CHUNK_WARPS = BIN_CHUNK_WARPS;
// Rects above this many tiles are listed by the binning and summed by a whole
// block in the gather (0.2% of the visible Gaussians of a 300k-Gaussian
// 1352x1014 view, 2% at 1M and 1920x1080, where the largest covers ~4300
// tiles): walked by one warp, 32 tiles a pass, they would take up to ~140
// passes in a row and set the gather's time on their own.  Measured against
// 512 and 1024, 384 gives the shortest gather at both sizes.
constexpr int GATHER_BIG_AREA = 384;
constexpr uint32_t KEY_CULLED = 0xffffffffu;

struct Header {
    uint32_t n_vis;
    uint32_t overflow;
    unsigned long long pairs;
    uint32_t n_big;                                     // entries of the large-rect list
    uint32_t prefix_done;                               // blocks of k_chunk_prefix finished
    uint32_t list_max;                                  // lists of at most this many pairs are written
    uint32_t key_or, key_nor;                           // OR of the sort keys, OR of their complements
};

// Whether every sort key has the same 8-bit digit at `shift` (a stable pass on
// it is then the identity): no bit of the digit is 1 in one key and 0 in another.
__device__ __forceinline__ bool digit_constant(const Header *hdr, int shift) {
    return (((hdr->key_or & hdr->key_nor) >> shift) & (RADIX - 1)) == 0;
}

struct Layout {
    size_t hdr, dtot, keys0, vals0, keys1, vals1, hist, counts, tile_total, tile_off, masks, big, visited, hit, occ,
        wext, total;
};

// 32-chunk words of the per-tile chunk occupancy (bit c % 32 of word c / 32:
// chunk c has a member in the tile)
int occ_words(int n) { return div_up(div_up(n > 0 ? n : 1, CHUNK), 32); }

size_t align_up(size_t v) { return (v + 255) & ~size_t(255); }

// masks: per chunk, the column words mx[TX][CHUNK_WARPS] then the row words
// my[TY][CHUNK_WARPS], tile-major so that a tile's words are contiguous
// (built once by k_chunk_counts, read by the scatter and the gather).
Layout layout_of(int n, int TX, int TY) {
    const int n_tiles = TX * TY;
    Layout L;
    const size_t nb = (size_t)div_up(n > 0 ? n : 1, SORT_TILE);
    const size_t chunks = (size_t)div_up(n > 0 ? n : 1, CHUNK);
    size_t o = 0;
    L.hdr = o; o = align_up(o + sizeof(Header));
    L.dtot = o; o = align_up(o + 4 * 4 * (size_t)RADIX);      // digit totals of the 4 passes
    L.keys0 = o; o = align_up(o + 4 * (size_t)(n > 0 ? n : 1));
    L.vals0 = o; o = align_up(o + 4 * (size_t)(n > 0 ? n : 1));
    L.keys1 = o; o = align_up(o + 4 * (size_t)(n > 0 ? n : 1));
    L.vals1 = o; o = align_up(o + 4 * (size_t)(n > 0 ? n : 1));
    L.hist = o; o = align_up(o + 4 * (size_t)RADIX * nb);
    L.counts = o; o = align_up(o + 4 * chunks * (size_t)n_tiles);
    L.tile_total = o; o = align_up(o + 4 * (size_t)n_tiles);
    L.tile_off = o; o = align_up(o + 4 * (size_t)(n_tiles + 1));
    L.masks = o; o = align_up(o + 4 * chunks * CHUNK_WARPS * (size_t)(TX + TY));
    L.big = o; o = align_up(o + 4 * (size_t)(n > 0 ? n : 1));  // depth-sorted indices of large rects
    // written by the compositing adjoint's first pass, read by its gather
    L.visited = o; o = align_up(o + 4 * (size_t)n_tiles);       // visited prefix of each tile's list
    L.hit = o; o = align_up(o + (size_t)(n > 0 ? n : 1));        // Gaussians with a contributing record
    L.occ = o; o = align_up(o + 4 * (size_t)occ_words(n) * n_tiles);   // [word][tile]
    // lists formed in the forward: per tile, the chunks below this one had
    // their first list position (the counts' prefix) written by the forward
    L.wext = o; o = align_up(o + 4 * (size_t)n_tiles);
    L.total = o;
    return L;
}

// ---------------------------------------------------------------- step 0
// Keys (depth bits, culled last) and values of one sort block of SORT_TILE
// Gaussians, and that block's histogram of the first pass's digit (what
// k_radix_hist gives for it, without reading the keys again).
__global__ void __launch_bounds__(SORT_THREADS) k_bin_prep(int n, const float *__restrict__ depth, int dstride,
                                                           const int4 *__restrict__ rects,
                                                           uint32_t *__restrict__ keys, uint32_t *__restrict__ vals,
                                                           uint32_t *__restrict__ hist, uint32_t *__restrict__ dtot,
                                                           Header *hdr) {
    pdl_enter();
    __shared__ uint32_t h[RADIX];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int base = blockIdx.x * SORT_TILE;
    uint32_t nvis = 0, kor = 0, knor = 0;
#pragma unroll
    for (int r = 0; r < SORT_ITEMS; ++r) {
        const int i = base + r * SORT_THREADS + threadIdx.x;
        if (i < n) {
            const int4 rc = rects[i];
            const bool vis = rc.z > rc.x && rc.w > rc.y;
            const uint32_t key = vis ? __float_as_uint(depth[(size_t)i * dstride]) : KEY_CULLED;
            keys[i] = key;
            vals[i] = (uint32_t)i;
            nvis += vis ? 1u : 0u;
            kor |= key;
            knor |= ~key;
            atomicAdd(&h[key & (RADIX - 1)], 1u);
        }
    }
    nvis = __reduce_add_sync(FULL, nvis);
    kor = __reduce_or_sync(FULL, kor);
    knor = __reduce_or_sync(FULL, knor);
    if ((threadIdx.x & 31) == 0) {
        if (nvis) atomicAdd(&hdr->n_vis, nvis);
        atomicOr(&hdr->key_or, kor);
        atomicOr(&hdr->key_nor, knor);
    }
    __syncthreads();
    const uint32_t c = h[threadIdx.x];
    hist[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = c;
    if (c) atomicAdd(&dtot[threadIdx.x], c);              // integer: the total is order-independent
}

// ---------------------------------------------------------------- step 1: radix sort of depth keys
__global__ void __launch_bounds__(SORT_THREADS) k_radix_hist(int n, int shift, const uint32_t *__restrict__ keys,
                                                             uint32_t *__restrict__ hist,
                                                             uint32_t *__restrict__ dtot, const Header *hdr) {
    pdl_enter();
    if (digit_constant(hdr, shift)) return;             // the pass is a copy
    __shared__ uint32_t h[RADIX];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int base = blockIdx.x * SORT_TILE;
#pragma unroll
    for (int r = 0; r < SORT_ITEMS; ++r) {
        const int i = base + r * SORT_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & (RADIX - 1)], 1u);
    }
    __syncthreads();
    const uint32_t c = h[threadIdx.x];
    hist[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = c;
    if (c) atomicAdd(&dtot[threadIdx.x], c);              // integer: the total is order-independent
}

// Exclusive scan, in place and in digit-major order, of the [RADIX][nb]
// per-block digit histogram: one warp per digit (RADIX / 32 blocks of 32
// warps).  Warp d starts from the count of all smaller digits (from the digit
// totals) and walks its digit's blocks 256 at a time.
__global__ void __launch_bounds__(1024) k_radix_scan(uint32_t *__restrict__ hist, int nb,
                                                     const uint32_t *__restrict__ dtot, const Header *hdr,
                                                     int shift) {
    pdl_enter();
    if (digit_constant(hdr, shift)) return;             // the pass is a copy
    const int lane = threadIdx.x & 31;
    const int d = blockIdx.x * 32 + (threadIdx.x >> 5);
    constexpr int PER = RADIX / 32;
    uint32_t below = 0;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int e = lane * PER + q;
        below += e < d ? dtot[e] : 0u;
    }
    uint32_t run = __reduce_add_sync(FULL, below);
    // SCAN_PER consecutive blocks per lane, SCAN_PER * 32 blocks per round,
    // all of a round's loads in flight together
    constexpr int SCAN_PER = 8;
    uint32_t *row = hist + (size_t)d * nb;
    for (int b0 = 0; b0 < nb; b0 += 32 * SCAN_PER) {
        const int bl = b0 + lane * SCAN_PER;
        uint32_t v[SCAN_PER];
#pragma unroll
        for (int q = 0; q < SCAN_PER; ++q) v[q] = bl + q < nb ? row[bl + q] : 0u;
        uint32_t mine = 0;
#pragma unroll
        for (int q = 0; q < SCAN_PER; ++q) mine += v[q];
        uint32_t incl = mine;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t x = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += x;
        }
        uint32_t at = run + incl - mine;
#pragma unroll
        for (int q = 0; q < SCAN_PER; ++q) {
            if (bl + q < nb) row[bl + q] = at;
            at += v[q];
        }
        run += __shfl_sync(FULL, incl, 31);
    }
}

// Stable scatter: within a block items are ranked in their original order
// (round by round, warp by warp, lane by lane).  A pass whose digit is the
// same in every key is the identity: the block copies its items.
__global__ void __launch_bounds__(SORT_THREADS) k_radix_scatter(int n, int shift,
                                                                const uint32_t *__restrict__ kin,
                                                                const uint32_t *__restrict__ vin,
                                                                const uint32_t *__restrict__ offs,
                                                                uint32_t *__restrict__ kout,
                                                                uint32_t *__restrict__ vout, const Header *hdr) {
    pdl_enter();
    constexpr int W = SORT_THREADS / 32;
    __shared__ uint32_t base[RADIX];          // running count of each digit in this block
    __shared__ uint32_t wcnt[W][RADIX];
    const int warp = threadIdx.x >> 5;
    const int blk = blockIdx.x * SORT_TILE;
    uint32_t keys[SORT_ITEMS], vals[SORT_ITEMS];      // all of the block's loads in flight at once
#pragma unroll
    for (int r = 0; r < SORT_ITEMS; ++r) {
        const int i = blk + r * SORT_THREADS + threadIdx.x;
        keys[r] = i < n ? kin[i] : 0u;
        vals[r] = i < n ? vin[i] : 0u;
    }
    if (digit_constant(hdr, shift)) {
#pragma unroll
        for (int r = 0; r < SORT_ITEMS; ++r) {
            const int i = blk + r * SORT_THREADS + threadIdx.x;
            if (i < n) {
                kout[i] = keys[r];
                vout[i] = vals[r];
            }
        }
        return;
    }
    base[threadIdx.x] = offs[(size_t)threadIdx.x * gridDim.x + blockIdx.x];
#pragma unroll
    for (int r = 0; r < SORT_ITEMS; ++r) {
        for (int w = 0; w < W; ++w) wcnt[w][threadIdx.x] = 0;
        __syncthreads();
        const int i = blk + r * SORT_THREADS + threadIdx.x;
        const bool ok = i < n;
        const uint32_t key = keys[r];
        const uint32_t d = (key >> shift) & (RADIX - 1);
        const unsigned act = __ballot_sync(FULL, ok);
        const unsigned peers = __match_any_sync(FULL, ok ? d : 0xffffffffu) & act;
        const uint32_t rank = __popc(peers & lanemask_lt());
        if (ok && rank == 0) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        // per digit: exclusive prefix over warps, then advance the running base
        {
            const uint32_t dd = threadIdx.x;
            uint32_t run = base[dd];
            for (int w = 0; w < W; ++w) {
                const uint32_t c = wcnt[w][dd];
                wcnt[w][dd] = run;
                run += c;
            }
            base[dd] = run;
        }
        __syncthreads();
        if (ok) {
            const uint32_t pos = wcnt[warp][d] + rank;
            kout[pos] = key;
            vout[pos] = vals[r];
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- step 2: counting pass on the tile digit
// A chunk's masks in shared memory, tile-major like their workspace slot: a
// tile column's (row's) CHUNK_WARPS words are 32 contiguous bytes.
struct ChunkSmem {
    __align__(16) uint32_t mx[QN_MAX_TILES_X][CHUNK_WARPS];
    __align__(16) uint32_t my[QN_MAX_TILES_Y][CHUNK_WARPS];
    int4 rect[CHUNK];
    uint32_t id[CHUNK];
    int ux0, uy0, ux1, uy1;
};

// Loads chunk c of the depth-sorted visible Gaussians (ids, rects, union
// bounding box of the rects).
__device__ void load_chunk_rects(int c, int TX, int TY, const uint32_t *__restrict__ sorted,
                                 const int4 *__restrict__ rects, uint32_t n_vis, ChunkSmem &s) {
    const int j = threadIdx.x;
    const uint32_t g = (uint32_t)c * CHUNK + j;
    int4 r = make_int4(0, 0, 0, 0);
    uint32_t id = 0;
    if (g < n_vis) {
        id = sorted[g];
        r = rects[id];
    }
    s.rect[j] = r;
    s.id[j] = id;
    if (j == 0) {
        s.ux0 = TX; s.uy0 = TY; s.ux1 = 0; s.uy1 = 0;
    }
    __syncthreads();
    const bool has = r.z > r.x;
    int x0 = has ? r.x : TX, y0 = has ? r.y : TY, x1 = has ? r.z : 0, y1 = has ? r.w : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        x0 = min(x0, __shfl_xor_sync(FULL, x0, o));
        y0 = min(y0, __shfl_xor_sync(FULL, y0, o));
        x1 = max(x1, __shfl_xor_sync(FULL, x1, o));
        y1 = max(y1, __shfl_xor_sync(FULL, y1, o));
    }
    if ((j & 31) == 0) {
        atomicMin(&s.ux0, x0); atomicMin(&s.uy0, y0);
        atomicMax(&s.ux1, x1); atomicMax(&s.uy1, y1);
    }
    __syncthreads();
}

// Builds, per warp, the bitmask of the chunk's members covering each tile
// column and each tile row (after load_chunk_rects).
__device__ void build_masks(int TX, int TY, ChunkSmem &s) {
    const int j = threadIdx.x, warp = j >> 5;
    const int4 r = s.rect[j];
    for (int tx = 0; tx < TX; ++tx) {
        const unsigned b = __ballot_sync(FULL, r.x <= tx && tx < r.z);
        if ((j & 31) == 0) s.mx[tx][warp] = b;
    }
    for (int ty = 0; ty < TY; ++ty) {
        const unsigned b = __ballot_sync(FULL, r.y <= ty && ty < r.w);
        if ((j & 31) == 0) s.my[ty][warp] = b;
    }
    __syncthreads();
}

// Copies the chunk's masks between shared memory and their workspace slot
// (both tile-major: word i = tile i / 8, warp i % 8).
__device__ void store_masks(int TX, int TY, const ChunkSmem &s, uint32_t *__restrict__ gm) {
    const uint32_t *sx = &s.mx[0][0], *sy = &s.my[0][0];
    for (int i = threadIdx.x; i < CHUNK_WARPS * TX; i += blockDim.x) gm[i] = sx[i];
    uint32_t *gy = gm + CHUNK_WARPS * TX;
    for (int i = threadIdx.x; i < CHUNK_WARPS * TY; i += blockDim.x) gy[i] = sy[i];
}

__device__ void fetch_masks(int TX, int TY, const uint32_t *__restrict__ gm, ChunkSmem &s) {
    uint32_t *sx = &s.mx[0][0], *sy = &s.my[0][0];
    for (int i = threadIdx.x; i < CHUNK_WARPS * TX; i += blockDim.x) sx[i] = gm[i];
    const uint32_t *gy = gm + CHUNK_WARPS * TX;
    for (int i = threadIdx.x; i < CHUNK_WARPS * TY; i += blockDim.x) sy[i] = gy[i];
    __syncthreads();
}

// The chunk's members in a tile: column words x0, x1 against the row's words.
__device__ __forceinline__ uint32_t tile_members(uint4 x0, uint4 x1, const ChunkSmem &s, int ty) {
    const uint4 y0 = *reinterpret_cast<const uint4 *>(&s.my[ty][0]);
    const uint4 y1 = *reinterpret_cast<const uint4 *>(&s.my[ty][4]);
    return __popc(x0.x & y0.x) + __popc(x0.y & y0.y) + __popc(x0.z & y0.z) + __popc(x0.w & y0.w) +
           __popc(x1.x & y1.x) + __popc(x1.y & y1.y) + __popc(x1.z & y1.z) + __popc(x1.w & y1.w);
}

__device__ void load_chunk(int c, int TX, int TY, const uint32_t *__restrict__ sorted,
                           const int4 *__restrict__ rects, uint32_t n_vis, ChunkSmem &s) {
    load_chunk_rects(c, TX, TY, sorted, rects, n_vis, s);
    build_masks(TX, TY, s);
}


__global__ void __launch_bounds__(CHUNK) k_chunk_counts(int TX, int TY, const uint32_t *__restrict__ sorted,
                                                        const int4 *__restrict__ rects, Header *hdr,
                                                        uint32_t *__restrict__ counts,
                                                        uint32_t *__restrict__ masks,
                                                        uint32_t *__restrict__ big_list) {
    pdl_enter();
    __shared__ ChunkSmem s;
    const int c = blockIdx.x;
    const uint32_t n_vis = hdr->n_vis;
    const int n_tiles = TX * TY;
    uint32_t *row = counts + (size_t)c * n_tiles;
    if ((uint32_t)c * CHUNK >= n_vis) {
        for (int t = threadIdx.x; t < n_tiles; t += CHUNK) row[t] = 0;
        return;
    }
    load_chunk(c, TX, TY, sorted, rects, n_vis, s);
    store_masks(TX, TY, s, masks + (size_t)c * CHUNK_WARPS * (TX + TY));
    {
        // list the chunk's rects above GATHER_BIG_AREA tiles (in any order:
        // the gather sums each on its own); slots past n_vis hold empty rects
        const int j = threadIdx.x, lane = j & 31;
        const int4 r = s.rect[j];
        const bool big = (r.z - r.x) * (r.w - r.y) > GATHER_BIG_AREA;
        const unsigned b = __ballot_sync(FULL, big);
        uint32_t at = 0;
        if (lane == 0 && b) at = atomicAdd(&hdr->n_big, (uint32_t)__popc(b));
        at = __shfl_sync(FULL, at, 0);
        if (big) big_list[at + __popc(b & ((1u << lane) - 1u))] = (uint32_t)c * CHUNK + j;
    }
    // thread (column tx, row phase g): its column's words in registers, the
    // rows g, g + k, ... (k = CHUNK / TX row phases; a row's stores coalesce)
    const int k = CHUNK / TX, tx = threadIdx.x % TX, g = threadIdx.x / TX;
    if (g < k) {
        const uint4 x0 = *reinterpret_cast<const uint4 *>(&s.mx[tx][0]);
        const uint4 x1 = *reinterpret_cast<const uint4 *>(&s.mx[tx][4]);
        const bool colin = tx >= s.ux0 && tx < s.ux1;
        for (int ty = g; ty < TY; ty += k)
            row[ty * TX + tx] = colin && ty >= s.uy0 && ty < s.uy1 ? tile_members(x0, x1, s, ty) : 0u;
    }
}

// Exclusive scan of tile totals -> tile offsets, ranges and P, by one block of
// 1024 threads: thread i takes a run of consecutive tiles (loads in batches
// of 8), then a shuffle scan of the 64-bit run sums within each warp and over
// the warps.  total is read through L2: other blocks of the same launch wrote it.
__device__ void tile_offsets(int n_tiles, const uint32_t *__restrict__ total, uint32_t *__restrict__ off,
                             uint32_t *__restrict__ ranges, Header *hdr, unsigned long long capacity,
                             long long *n_pairs, uint32_t list_max) {
    __shared__ unsigned long long wsum[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int per = div_up_dev(n_tiles, 1024);
    const int b = threadIdx.x * per, e = min(n_tiles, b + per);
    unsigned long long s = 0;
    for (int t0 = b; t0 < e; t0 += 8) {
        uint32_t v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = t0 + k < e ? __ldcg(total + t0 + k) : 0u;
#pragma unroll
        for (int k = 0; k < 8; ++k) s += v[k];
    }
    unsigned long long incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long x = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += x;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const unsigned long long w = wsum[lane];
        unsigned long long wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long x = __shfl_up_sync(FULL, wi, o);
            if (lane >= o) wi += x;
        }
        wsum[lane] = wi - w;                            // exclusive over warps
    }
    __syncthreads();
    unsigned long long run = wsum[warp] + incl - s;
    __shared__ unsigned long long total_pairs;
    if (threadIdx.x == 1023) total_pairs = wsum[31] + incl;
    __syncthreads();
    const unsigned long long PT = total_pairs;
    const bool over = PT > capacity || PT > 0xffffffffull;
    for (int t = b; t < e; ++t) {
        const uint32_t v = __ldcg(total + t);
        off[t] = (uint32_t)run;
        ranges[2 * (size_t)t] = over ? 0u : (uint32_t)run;
        ranges[2 * (size_t)t + 1] = over ? 0u : (uint32_t)(run + v);
        run += v;
    }
    if (threadIdx.x == 0) {
        hdr->pairs = PT;
        hdr->overflow = over ? 1u : 0u;
        hdr->list_max = list_max;
        if (n_pairs) *n_pairs = (long long)PT;
    }
}

// In place: counts[c][t] <- sum_{c' < c} counts[c'][t] (unless list_max is
// 0); tile_total[t] = sum_c.  Block = 32 tiles (lanes) x 32 chunk segments
// (warps).  Each warp walks its segment PREFIX_BATCH chunks at a time with
// the loads issued together (the walk is otherwise one dependent memory
// round trip per chunk).  With occ,
// the occupancy bits (count > 0) of the block's tiles are gathered in shared
// memory ([word][tile], occ_w words) and written to occ[word][tile].  The
// block that finishes last (a ticket counter; nothing waits) then scans the
// tile totals into the tile offsets, the ranges and P.
constexpr int PREFIX_BATCH = 8;

__global__ void __launch_bounds__(1024) k_chunk_prefix(int n_chunks, int n_tiles, uint32_t *__restrict__ counts,
                                                       uint32_t *__restrict__ tile_total,
                                                       uint32_t *__restrict__ tile_off, uint32_t *__restrict__ ranges,
                                                       Header *hdr, unsigned long long capacity,
                                                       long long *n_pairs, uint32_t list_max,
                                                       uint32_t *__restrict__ occ, int occ_w) {
    pdl_enter();
    __shared__ uint32_t seg[32][33];
    extern __shared__ uint32_t socc[];                  // [occ_w][32] when occ is given
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int t = blockIdx.x * 32 + lane;
    const int per = div_up_dev(n_chunks, 32);
    const int c0 = warp * per, c1 = min(n_chunks, c0 + per);
    if (occ)
        for (int i = threadIdx.x; i < occ_w * 32; i += blockDim.x) socc[i] = 0;
    __syncthreads();
    uint32_t s = 0;
    if (t < n_tiles) {
        int c = c0;
        for (; c + PREFIX_BATCH <= c1; c += PREFIX_BATCH) {
            uint32_t v[PREFIX_BATCH];
#pragma unroll
            for (int k = 0; k < PREFIX_BATCH; ++k) v[k] = counts[(size_t)(c + k) * n_tiles + t];
#pragma unroll
            for (int k = 0; k < PREFIX_BATCH; ++k) {
                s += v[k];
                if (occ && v[k]) atomicOr(&socc[((c + k) >> 5) * 32 + lane], 1u << ((c + k) & 31));
            }
        }
        for (; c < c1; ++c) {
            const uint32_t v = counts[(size_t)c * n_tiles + t];
            s += v;
            if (occ && v) atomicOr(&socc[(c >> 5) * 32 + lane], 1u << (c & 31));
        }
    }
    seg[warp][lane] = s;
    __syncthreads();
    if (occ && t < n_tiles)
        for (int w = warp; w < occ_w; w += 32) occ[(size_t)w * n_tiles + t] = socc[w * 32 + lane];
    if (warp == 0) {
        uint32_t run = 0;
        for (int w = 0; w < 32; ++w) {
            const uint32_t v = seg[w][lane];
            seg[w][lane] = run;
            run += v;
        }
        if (t < n_tiles) tile_total[t] = run;
    }
    __syncthreads();
    // the per-chunk list positions: the chunk scatter of written lists reads
    // them; with no list written (list_max 0) the forward writes those of
    // the chunks it walks instead
    if (t < n_tiles && list_max != 0u) {
        uint32_t run = seg[warp][lane];
        int c = c0;
        for (; c + PREFIX_BATCH <= c1; c += PREFIX_BATCH) {
            uint32_t v[PREFIX_BATCH];
#pragma unroll
            for (int k = 0; k < PREFIX_BATCH; ++k) v[k] = counts[(size_t)(c + k) * n_tiles + t];
#pragma unroll
            for (int k = 0; k < PREFIX_BATCH; ++k) {
                counts[(size_t)(c + k) * n_tiles + t] = run;
                run += v[k];
            }
        }
        for (; c < c1; ++c) {
            const size_t o = (size_t)c * n_tiles + t;
            const uint32_t v = counts[o];
            counts[o] = run;
            run += v;
        }
    }
    __shared__ bool last;
    if (warp == 0) __threadfence();                     // this block's tile totals (warp 0's) before its ticket
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&hdr->prefix_done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    tile_offsets(n_tiles, tile_total, tile_off, ranges, hdr, capacity, n_pairs, list_max);
}

// The chunk prefix's shared occupancy bits above the 48 KB default: set once
// per process (before any graph capture that the first call precedes).
constexpr size_t PREFIX_MAX_OCC_SMEM = 192 * 1024;
cudaError_t prefix_attributes() {
    static std::once_flag once;
    static cudaError_t err = cudaSuccess;
    std::call_once(once, [] {
        err = cudaFuncSetAttribute(k_chunk_prefix, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)PREFIX_MAX_OCC_SMEM);
    });
    return err;
}

// Writes chunk c's members tile by tile: one thread per tile of the chunk's
// bounding box writes the tile's members in depth order (the set bits of the
// per-warp words, warp by warp) to consecutive slots from the chunk's first
// slot in that tile.  Tiles holding more than list_max pairs are left out
// (the compositing forward forms their lists).
__global__ void __launch_bounds__(CHUNK) k_chunk_scatter(int TX, int TY, const uint32_t *__restrict__ sorted,
                                                         const int4 *__restrict__ rects,
                                                         const float *__restrict__ depth, int dstride,
                                                         const Header *hdr, const uint32_t *__restrict__ gbase,
                                                         const uint32_t *__restrict__ tile_off,
                                                         const uint32_t *__restrict__ masks,
                                                         uint32_t *__restrict__ vals,
                                                         unsigned long long *__restrict__ keys, int vec,
                                                         const uint32_t *__restrict__ tile_total,
                                                         uint32_t list_max) {
    __shared__ ChunkSmem s;
    __shared__ uint32_t dbits[CHUNK];                   // depth bits of the members (for keys)
    const int c = blockIdx.x;
    const uint32_t n_vis = hdr->n_vis;
    if (hdr->overflow || (uint32_t)c * CHUNK >= n_vis) return;
    load_chunk_rects(c, TX, TY, sorted, rects, n_vis, s);
    if (keys) dbits[threadIdx.x] = __float_as_uint(depth[(size_t)s.id[threadIdx.x] * dstride]);
    fetch_masks(TX, TY, masks + (size_t)c * CHUNK_WARPS * (TX + TY), s);
    const int n_tiles = TX * TY;
    const int uw = s.ux1 - s.ux0, uh = s.uy1 - s.uy0;
    if (uw <= 0 || uh <= 0) return;
    const uint32_t *grow = gbase + (size_t)c * n_tiles;
    for (int q = threadIdx.x; q < uw * uh; q += CHUNK) {
        const int tx = s.ux0 + q % uw, ty = s.uy0 + q / uw;
        uint32_t m[CHUNK_WARPS];
        bool any = false;
#pragma unroll
        for (int w = 0; w < CHUNK_WARPS; ++w) {
            m[w] = s.mx[tx][w] & s.my[ty][w];
            any |= m[w] != 0;
        }
        if (!any) continue;
        const int t = ty * TX + tx;
        if (list_max != 0xffffffffu && tile_total[t] > list_max) continue;
        uint32_t pos = tile_off[t] + grow[t];
        if (keys || !vec) {
#pragma unroll
            for (int w = 0; w < CHUNK_WARPS; ++w) {
                uint32_t b = m[w];
                while (b) {
                    const int jj = w * 32 + __ffs(b) - 1;
                    b &= b - 1;
                    vals[pos] = s.id[jj];
                    if (keys) keys[pos] = ((unsigned long long)(uint32_t)t << 32) | (unsigned long long)dbits[jj];
                    ++pos;
                }
            }
            continue;
        }
        // the run's slots are consecutive: single stores up to a 16-byte
        // boundary, then four members per 16-byte store (one memory
        // transaction instead of four), then the tail
        uint32_t q0 = 0, q1 = 0, q2 = 0;
        int nq = 0;
#pragma unroll
        for (int w = 0; w < CHUNK_WARPS; ++w) {
            uint32_t b = m[w];
            while (b) {
                const int jj = w * 32 + __ffs(b) - 1;
                b &= b - 1;
                const uint32_t id = s.id[jj];
                if (nq == 0 && (pos & 3u)) {
                    vals[pos++] = id;
                } else if (nq == 0) {
                    q0 = id; nq = 1;
                } else if (nq == 1) {
                    q1 = id; nq = 2;
                } else if (nq == 2) {
                    q2 = id; nq = 3;
                } else {
                    *reinterpret_cast<uint4 *>(vals + pos) = make_uint4(q0, q1, q2, id);
                    pos += 4;
                    nq = 0;
                }
            }
        }
        if (nq > 0) vals[pos] = q0;
        if (nq > 1) vals[pos + 1] = q1;
        if (nq > 2) vals[pos + 2] = q2;
    }
}

// Adjoint of the pair scatter: each visible Gaussian sums the per-pair
// gradient records of the visited positions of its tiles, walking its rect in
// row-major order with a fixed thread assignment and a fixed reduction order
// -- so the sums are reproducible.  A Gaussian's rank in a tile's list comes
// from its chunk's row/column bitmasks (stored by k_chunk_counts); a tile is
// skipped when the Gaussian lies beyond the tile's visited prefix.  Every load
// of a tile (the chunk's count-row entry, the visited length, the tile's
// offset and its 16 mask words, four 16-byte loads) depends on the tile alone
// and is issued before the first is used, so a tile costs two dependent memory
// round trips: those loads, then the record.
constexpr int GATHER_THREADS = 256;
constexpr int GATHER_WARPS = GATHER_THREADS / 32;

// Where depth-sorted Gaussian g's chunk keeps its masks and count row.
struct GatherChunk {
    const uint4 *mx, *my;                               // a tile column's / row's CHUNK_WARPS words
    const uint32_t *grow;                               // the chunk's first slot in each tile
    const uint32_t *wext;                               // nullable: the forward's walked chunk extent per tile
    uint32_t c;                                         // the chunk
    int wj;                                             // g's warp in the chunk
    unsigned below;                                     // g's lower lanes in that warp
};

__device__ __forceinline__ GatherChunk gather_chunk(int TX, int TY, uint32_t g, const uint32_t *__restrict__ gbase,
                                                    const uint32_t *__restrict__ masks,
                                                    const uint32_t *__restrict__ wext) {
    // 16-byte aligned: the workspace slot is, a chunk's masks take 32 (TX + TY)
    // bytes and a tile's words 32
    static_assert(CHUNK_WARPS == 8, "a tile's mask words are two uint4");
    const int c = (int)(g / CHUNK), j = (int)(g % CHUNK);
    GatherChunk k;
    k.mx = reinterpret_cast<const uint4 *>(masks + (size_t)c * CHUNK_WARPS * (TX + TY));
    k.my = k.mx + 2 * TX;
    k.grow = gbase + (size_t)c * TX * TY;
    k.wext = wext;
    k.c = (uint32_t)c;
    k.wj = j >> 5;
    k.below = (1u << (j & 31)) - 1u;
    return k;
}

// The pair slot of the Gaussian in tile (tx, ty), or -1 when it lies past the
// tile's visited prefix (no record there).  With wext (lists formed in the
// forward) a chunk at or past the tile's walked extent has no written list
// position and lies past the visited prefix.
__device__ __forceinline__ long long gather_slot(int TX, int tx, int ty, const GatherChunk &k,
                                                 const uint32_t *__restrict__ tile_off,
                                                 const uint32_t *__restrict__ visited) {
    const int t = ty * TX + tx;
    const uint32_t base = k.grow[t], vis = visited[t], off = tile_off[t];
    const uint32_t ext = k.wext ? k.wext[t] : 0xffffffffu;
    const uint4 x0 = k.mx[2 * tx], x1 = k.mx[2 * tx + 1], y0 = k.my[2 * ty], y1 = k.my[2 * ty + 1];
    const uint32_t m[CHUNK_WARPS] = {x0.x & y0.x, x0.y & y0.y, x0.z & y0.z, x0.w & y0.w,
                                     x1.x & y1.x, x1.y & y1.y, x1.z & y1.z, x1.w & y1.w};
    // members of the earlier warps, then those below g in its own warp
    uint32_t rank = 0;
#pragma unroll
    for (int w = 0; w < CHUNK_WARPS; ++w) rank += __popc(m[w] & (w < k.wj ? ~0u : w == k.wj ? k.below : 0u));
    return k.c < ext && base + rank < vis ? (long long)off + base + rank : -1ll;
}

__device__ __forceinline__ void add_record(const float4 *__restrict__ pair_grads, long long slot, float acc[9]) {
    const float4 *p = pair_grads + 3 * (size_t)slot;
    const float4 b0 = p[0], b1 = p[1], b2 = p[2];
    acc[0] += b0.x; acc[1] += b0.y; acc[2] += b0.z;
    acc[3] += b1.x; acc[4] += b1.y; acc[5] += b1.z;
    acc[6] += b2.x; acc[7] += b2.y; acc[8] += b2.z;
}

// Thread i of `threads` walks tiles i, i + threads, ... of rect r in row-major
// order, stepping its (column, row) without a division per tile, two tiles at
// a time: both tiles' slot loads are in flight together, then both records,
// added in walk order (the sums do not depend on the unrolling).
__device__ __forceinline__ bool gather_walk(int TX, int4 r, int i, int threads, const GatherChunk &k,
                                            const uint32_t *__restrict__ tile_off,
                                            const uint32_t *__restrict__ visited,
                                            const float4 *__restrict__ pair_grads, float acc[9]) {
    const int rw = r.z - r.x, area = rw * (r.w - r.y);
    bool found = false;
    int cx = rw > 0 ? i % rw : 0, cy = rw > 0 ? i / rw : 0;
    const int dq = rw > 0 ? threads / rw : 0, dr = rw > 0 ? threads % rw : 0;
    for (int q = i; q < area; q += 2 * threads) {
        const int ax = cx, ay = cy;
        cx += dr;
        cy += dq;
        if (cx >= rw) {
            cx -= rw;
            ++cy;
        }
        const bool second = q + threads < area;
        const int bx = cx, by = cy;
        if (second) {
            cx += dr;
            cy += dq;
            if (cx >= rw) {
                cx -= rw;
                ++cy;
            }
        }
        const long long sa = gather_slot(TX, r.x + ax, r.y + ay, k, tile_off, visited);
        const long long sb = second ? gather_slot(TX, r.x + bx, r.y + by, k, tile_off, visited) : -1ll;
        if (sa >= 0) add_record(pair_grads, sa, acc);
        if (sb >= 0) add_record(pair_grads, sb, acc);
        found |= (sa >= 0) | (sb >= 0);
    }
    return found;
}

// The nine sums of a Gaussian's record (d mean2d x, y, d opacity, d conic
// a, b, c, d rgb) to their places in its 48-byte gradient record.
__device__ __forceinline__ void put_record(float *o, int q, float v) { o[(q / 3) * 4 + q % 3] = v; }

struct GatherSmem {
    uint32_t g[GATHER_THREADS], id[GATHER_THREADS];
    int4 rect[GATHER_THREADS];
    int wcount[GATHER_WARPS];
    float part[GATHER_WARPS][9];
};

// The large rects: block b of G takes the listed entries b, b + G, ...
// (GATHER_THREADS at a time, loaded together), keeps the wanted ones, and
// sums each with all its threads: per-warp sums, then the warps' sums in warp
// order.
__device__ void gather_big(int TX, int TY, uint32_t n_big, const uint32_t *__restrict__ big_list,
                           const uint32_t *__restrict__ sorted, const int4 *__restrict__ rects,
                           const uint32_t *__restrict__ gbase, const uint32_t *__restrict__ tile_off,
                           const uint32_t *__restrict__ visited, const float4 *__restrict__ pair_grads,
                           const uint8_t *__restrict__ skip, const uint8_t *__restrict__ ghit,
                           const uint32_t *__restrict__ masks, const uint32_t *__restrict__ wext,
                           float4 *__restrict__ out, GatherSmem &sm) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const size_t G = gridDim.x;
    for (size_t e0 = blockIdx.x; e0 < n_big; e0 += G * GATHER_THREADS) {
        const size_t e = e0 + (size_t)tid * G;
        uint32_t g = 0, id = 0;
        int4 r = make_int4(0, 0, 0, 0);
        bool wanted = false;
        if (e < n_big) {
            g = big_list[e];
            id = sorted[g];
            wanted = !(skip && skip[id]) && !(ghit && !ghit[id]);
            if (wanted) r = rects[id];
        }
        const unsigned m = __ballot_sync(FULL, wanted);
        if (lane == 0) sm.wcount[warp] = __popc(m);
        __syncthreads();
        int at = 0, total = 0;
#pragma unroll
        for (int w = 0; w < GATHER_WARPS; ++w) {
            at += w < warp ? sm.wcount[w] : 0;
            total += sm.wcount[w];
        }
        if (wanted) {
            const int q = at + __popc(m & ((1u << lane) - 1u));
            sm.g[q] = g;
            sm.id[q] = id;
            sm.rect[q] = r;
        }
        __syncthreads();
        for (int i = 0; i < total; ++i) {
            const GatherChunk k = gather_chunk(TX, TY, sm.g[i], gbase, masks, wext);
            float acc[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            gather_walk(TX, sm.rect[i], tid, GATHER_THREADS, k, tile_off, visited, pair_grads, acc);
            const float red = reduce_scatter8(acc, lane);  // lane 4q holds the sum of value q
            const float red8 = warp_sum(acc[8]);
            if ((lane & 3) == 0) sm.part[warp][lane >> 2] = red;
            if (lane == 0) sm.part[warp][8] = red8;
            __syncthreads();
            if (tid < 9) {
                float v = 0.f;
#pragma unroll
                for (int w = 0; w < GATHER_WARPS; ++w) v += sm.part[w][tid];
                put_record(reinterpret_cast<float *>(out + 3 * (size_t)sm.id[i]), tid, v);
            }
            __syncthreads();                            // part and the list are reused
        }
    }
}

// One Gaussian by one warp (g its depth-sorted index, id its index in the
// scene).
__device__ __forceinline__ void gather_warp(int TX, int TY, uint32_t g, uint32_t id, int4 r, int lane,
                                            const uint32_t *__restrict__ gbase,
                                            const uint32_t *__restrict__ tile_off,
                                            const uint32_t *__restrict__ visited,
                                            const float4 *__restrict__ pair_grads,
                                            const uint32_t *__restrict__ masks,
                                            const uint32_t *__restrict__ wext, float4 *__restrict__ out) {
    const GatherChunk k = gather_chunk(TX, TY, g, gbase, masks, wext);
    float acc[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const bool found = gather_walk(TX, r, lane, 32, k, tile_off, visited, pair_grads, acc);
    if (!__any_sync(FULL, found)) return;               // no visited pair: stays 0
    float *o = reinterpret_cast<float *>(out + 3 * (size_t)id);
    const float red = reduce_scatter8(acc, lane);       // lane 4q holds the sum of value q
    const float red8 = warp_sum(acc[8]);
    if ((lane & 3) == 0) put_record(o, lane >> 2, red);
    if (lane == 0) {
        put_record(o, 8, red8);
        o[3] = o[7] = o[11] = 0.f;
    }
}

// Every block first takes its share of the large rects (gather_big); then
// warp w of W takes the depth-sorted Gaussians w, w + W, w + 2W, ...: its
// lanes test 32 of them at once (skipped, without a composited record, or a
// large rect -> not its work) and load the rects of the wanted ones, then the
// warp sums the wanted ones one after another.  The stride spreads the
// front-most Gaussians, which own nearly all visited pairs, over every warp.
// The grid is one wave of resident blocks.
__global__ void __launch_bounds__(GATHER_THREADS, 3) k_bin_gather(int TX, int TY,
                                                               const uint32_t *__restrict__ sorted,
                                                               const int4 *__restrict__ rects, const Header *hdr,
                                                               const uint32_t *__restrict__ big_list,
                                                               const uint32_t *__restrict__ gbase,
                                                               const uint32_t *__restrict__ tile_off,
                                                               const uint32_t *__restrict__ visited,
                                                               const float4 *__restrict__ pair_grads,
                                                               const uint8_t *__restrict__ skip,
                                                               const uint8_t *__restrict__ ghit,
                                                               const uint32_t *__restrict__ masks,
                                                               const uint32_t *__restrict__ wext_ws,
                                                               float4 *__restrict__ out) {
    __shared__ GatherSmem sm;
    if (hdr->overflow) return;
    const uint32_t n_vis = hdr->n_vis;
    // with no list written the list positions are those the forward wrote
    const uint32_t *wext = hdr->list_max == 0u ? wext_ws : nullptr;
    gather_big(TX, TY, hdr->n_big, big_list, sorted, rects, gbase, tile_off, visited, pair_grads, skip, ghit,
               masks, wext, out, sm);
    const uint32_t W = (uint32_t)((gridDim.x * (size_t)blockDim.x) >> 5);
    const uint32_t w = (uint32_t)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    for (uint32_t k0 = 0; w + (size_t)k0 * W < n_vis; k0 += 32) {
        const size_t gl = w + (size_t)(k0 + lane) * W;
        uint32_t id = 0;
        bool wanted = false;
        if (gl < n_vis) {
            id = sorted[gl];
            wanted = !(skip && skip[id]) && !(ghit && !ghit[id]);
        }
        const int4 rr = wanted ? rects[id] : make_int4(0, 0, 0, 0);
        wanted = wanted && (rr.z - rr.x) * (rr.w - rr.y) <= GATHER_BIG_AREA;
        unsigned m = __ballot_sync(FULL, wanted);
        while (m) {
            const int l = __ffs(m) - 1;
            m &= m - 1;
            const uint32_t gid = __shfl_sync(FULL, id, l);
            const int4 r = make_int4(__shfl_sync(FULL, rr.x, l), __shfl_sync(FULL, rr.y, l),
                                     __shfl_sync(FULL, rr.z, l), __shfl_sync(FULL, rr.w, l));
            gather_warp(TX, TY, (uint32_t)(w + (size_t)(k0 + l) * W), gid, r, lane, gbase, tile_off, visited,
                        pair_grads, masks, wext, out);
        }
    }
}

}  // namespace
}  // namespace qn

namespace qn {
int bin_view(int32_t n, int32_t tiles_x, int32_t tiles_y, void *workspace, size_t workspace_bytes, BinView &v) {
    QN_REQUIRE(n >= 0 && tiles_x > 0 && tiles_y > 0 && tiles_x <= QN_MAX_TILES_X && tiles_y <= QN_MAX_TILES_Y,
               "bad n or tile grid");
    QN_REQUIRE(workspace && ((uintptr_t)workspace & 255) == 0, "binning workspace is required, 256-byte aligned");
    const Layout L = layout_of(n, tiles_x, tiles_y);
    QN_REQUIRE(workspace_bytes >= L.total, "binning workspace too small (%zu < %zu)", workspace_bytes, L.total);
    char *ws = static_cast<char *>(workspace);
    v.masks = reinterpret_cast<const uint32_t *>(ws + L.masks);
    v.sorted = reinterpret_cast<const uint32_t *>(ws + L.vals0);   // after the 4 passes, back in vals0
    v.n_vis = reinterpret_cast<const uint32_t *>(ws + L.hdr + offsetof(Header, n_vis));
    v.list_max = reinterpret_cast<const uint32_t *>(ws + L.hdr + offsetof(Header, list_max));
    v.occ = reinterpret_cast<const uint32_t *>(ws + L.occ);
    v.occ_w = occ_words(n);
    v.gbase = reinterpret_cast<uint32_t *>(ws + L.counts);
    v.wext = reinterpret_cast<uint32_t *>(ws + L.wext);
    return QN_OK;
}
}  // namespace qn

extern "C" size_t qn_bin_sort_workspace_size(int32_t n, int32_t tiles_x, int32_t tiles_y) {
    if (n < 0 || tiles_x <= 0 || tiles_y <= 0) return 0;
    return qn::layout_of(n, tiles_x, tiles_y).total;
}

namespace qn {
namespace {
// Both binning entry points: the lists of the tiles holding at most list_max
// pairs are written (all of them for list_max = 0xffffffff).
int bin_sort_impl(int32_t n, const float *depth, int32_t depth_stride, const int32_t *rects, int32_t tiles_x,
                  int32_t tiles_y, void *workspace, size_t workspace_bytes, int64_t pair_capacity,
                  uint32_t list_max, uint32_t *vals, uint64_t *keys, uint32_t *ranges, int64_t *n_pairs,
                  int64_t *n_pairs_host, qn_stream_t stream) {
    QN_REQUIRE(n >= 0, "n must be >= 0");
    QN_REQUIRE(tiles_x > 0 && tiles_y > 0 && tiles_x <= QN_MAX_TILES_X && tiles_y <= QN_MAX_TILES_Y,
               "tile grid %dx%d out of range", tiles_x, tiles_y);
    QN_REQUIRE(depth_stride >= 1, "depth_stride must be >= 1");
    QN_REQUIRE(pair_capacity >= 0, "pair_capacity must be >= 0");
    QN_REQUIRE(ranges && n_pairs, "ranges and n_pairs are required");
    QN_REQUIRE(n == 0 || (depth && rects && workspace), "null pointer argument");
    QN_REQUIRE(pair_capacity == 0 || vals, "vals is required when pair_capacity > 0");
    QN_REQUIRE(((uintptr_t)rects & 15) == 0 && ((uintptr_t)workspace & 255) == 0,
               "rects must be 16-byte and workspace 256-byte aligned");
    const int n_tiles = tiles_x * tiles_y;
    const Layout L = layout_of(n, tiles_x, tiles_y);
    QN_REQUIRE(n == 0 || workspace_bytes >= L.total, "workspace too small (%zu < %zu)", workspace_bytes, L.total);
    QN_REQUIRE(list_max == 0xffffffffu || 32 * 4 * (size_t)occ_words(n) <= PREFIX_MAX_OCC_SMEM,
               "%d Gaussians are too many for lists formed in the compositing forward (at most %d)", n,
               (int)(PREFIX_MAX_OCC_SMEM / 128 * 32 * CHUNK));
    const int64_t capacity = std::min<int64_t>(pair_capacity, 0xffffffffll);   // pair positions are 32-bit
    cudaStream_t s = as_stream(stream);
    if (n == 0) {
        if (cudaMemsetAsync(ranges, 0, sizeof(uint32_t) * 2 * n_tiles, s) != cudaSuccess ||
            cudaMemsetAsync(n_pairs, 0, sizeof(int64_t), s) != cudaSuccess)
            return check_launch("qn_bin_sort memset");
        if (n_pairs_host) {
            if (cudaStreamSynchronize(s) != cudaSuccess) return check_launch("qn_bin_sort sync");
            *n_pairs_host = 0;
        }
        return QN_OK;
    }
    char *ws = static_cast<char *>(workspace);
    Header *hdr = reinterpret_cast<Header *>(ws + L.hdr);
    uint32_t *k0 = reinterpret_cast<uint32_t *>(ws + L.keys0), *v0 = reinterpret_cast<uint32_t *>(ws + L.vals0);
    uint32_t *k1 = reinterpret_cast<uint32_t *>(ws + L.keys1), *v1 = reinterpret_cast<uint32_t *>(ws + L.vals1);
    uint32_t *hist = reinterpret_cast<uint32_t *>(ws + L.hist);
    uint32_t *counts = reinterpret_cast<uint32_t *>(ws + L.counts);
    uint32_t *tile_total = reinterpret_cast<uint32_t *>(ws + L.tile_total);
    uint32_t *tile_off = reinterpret_cast<uint32_t *>(ws + L.tile_off);
    const int4 *r4 = reinterpret_cast<const int4 *>(rects);

    uint32_t *dtot = reinterpret_cast<uint32_t *>(ws + L.dtot);
    if (cudaMemsetAsync(hdr, 0, L.keys0 - L.hdr, s) != cudaSuccess)      // header and digit totals
        return check_launch("qn_bin_sort memset");
    const int nb = div_up(n, SORT_TILE);
    pdl_launch(k_bin_prep, nb, SORT_THREADS, 0, s, n, depth, depth_stride, r4, k0, v0, hist, dtot, hdr);
    for (int pass = 0; pass < 4; ++pass) {
        const int shift = 8 * pass;
        uint32_t *ki = (pass & 1) ? k1 : k0, *vi = (pass & 1) ? v1 : v0;
        uint32_t *ko = (pass & 1) ? k0 : k1, *vo = (pass & 1) ? v0 : v1;
        if (pass > 0)                                   // the first pass's histogram came with the keys
            pdl_launch(k_radix_hist, nb, SORT_THREADS, 0, s, n, shift, (const uint32_t *)ki, hist,
                       dtot + pass * RADIX, (const Header *)hdr);
        pdl_launch(k_radix_scan, RADIX / 32, 1024, 0, s, hist, nb, (const uint32_t *)(dtot + pass * RADIX),
                   (const Header *)hdr, shift);
        pdl_launch(k_radix_scatter, nb, SORT_THREADS, 0, s, n, shift, (const uint32_t *)ki, (const uint32_t *)vi,
                   (const uint32_t *)hist, ko, vo, (const Header *)hdr);
    }
    // after 4 passes the sorted (depth, index) order is back in k0 / v0
    const int n_chunks = div_up(n, CHUNK);
    uint32_t *masks = reinterpret_cast<uint32_t *>(ws + L.masks);
    pdl_launch(k_chunk_counts, n_chunks, CHUNK, 0, s, tiles_x, tiles_y, (const uint32_t *)v0, r4, hdr, counts, masks,
               reinterpret_cast<uint32_t *>(ws + L.big));
    // the occupancy bits only for lists the compositing forward forms
    uint32_t *occ = list_max != 0xffffffffu ? reinterpret_cast<uint32_t *>(ws + L.occ) : nullptr;
    const int occ_w = occ_words(n);
    const size_t occ_smem = occ ? sizeof(uint32_t) * 32 * (size_t)occ_w : 0;
    if (occ_smem > 48 * 1024 && prefix_attributes() != cudaSuccess) return check_launch("k_chunk_prefix attributes");
    pdl_launch(k_chunk_prefix, div_up(n_tiles, 32), 1024, occ_smem, s, n_chunks, n_tiles, counts, tile_total,
               tile_off, ranges, hdr, (unsigned long long)capacity, reinterpret_cast<long long *>(n_pairs),
               list_max, occ, occ_w);
    if (list_max > 0 && vals) {                         // the other lists: the compositing forward
        const int vec = ((uintptr_t)vals & 15) == 0;   // 16-byte stores need a 16-byte aligned vals
        k_chunk_scatter<<<n_chunks, CHUNK, 0, s>>>(tiles_x, tiles_y, v0, r4, depth, depth_stride, hdr, counts,
                                                   tile_off, masks, vals,
                                                   reinterpret_cast<unsigned long long *>(keys), vec, tile_total,
                                                   list_max);
    }
    int st = check_launch("qn_bin_sort");
    if (st) return st;
    if (n_pairs_host) {
        if (cudaMemcpyAsync(n_pairs_host, n_pairs, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return check_launch("qn_bin_sort readback");
        if (*n_pairs_host > capacity) {
            set_error("pair count %lld exceeds capacity %lld", (long long)*n_pairs_host, (long long)capacity);
            return QN_ERR_CAPACITY;
        }
    }
    return QN_OK;
}
}  // namespace
}  // namespace qn

extern "C" int qn_bin_sort(int32_t n, const float *depth, int32_t depth_stride, const int32_t *rects,
                           int32_t tiles_x, int32_t tiles_y, void *workspace, size_t workspace_bytes,
                           int64_t pair_capacity, uint32_t *vals, uint64_t *keys, uint32_t *ranges,
                           int64_t *n_pairs, int64_t *n_pairs_host, qn_stream_t stream) {
    return qn::bin_sort_impl(n, depth, depth_stride, rects, tiles_x, tiles_y, workspace, workspace_bytes,
                             pair_capacity, 0xffffffffu, vals, keys, ranges, n_pairs, n_pairs_host, stream);
}

extern "C" int qn_bin_sort_partial(int32_t n, const float *depth, int32_t depth_stride, const int32_t *rects,
                                   int32_t tiles_x, int32_t tiles_y, void *workspace, size_t workspace_bytes,
                                   int64_t pair_capacity, uint32_t list_max, uint32_t *vals, uint32_t *ranges,
                                   int64_t *n_pairs, int64_t *n_pairs_host, qn_stream_t stream) {
    return qn::bin_sort_impl(n, depth, depth_stride, rects, tiles_x, tiles_y, workspace, workspace_bytes,
                             pair_capacity, list_max, vals, nullptr, ranges, n_pairs, n_pairs_host, stream);
}

namespace {

// The camera's tile grid and the workspace checks shared by both passes of
// the compositing adjoint.
int adjoint_setup(const qn_camera *cam, int32_t n, const void *workspace, size_t workspace_bytes, int &TX, int &TY,
                  qn::Layout &L) {
    using namespace qn;
    QN_REQUIRE(cam, "camera is required");
    QN_REQUIRE(cam->width > 0 && cam->height > 0 && cam->width <= QN_TILE * QN_MAX_TILES_X &&
                   cam->height <= QN_TILE * QN_MAX_TILES_Y,
               "image size %dx%d out of range", cam->width, cam->height);
    QN_REQUIRE(n >= 0, "n must be >= 0");
    QN_REQUIRE(workspace && ((uintptr_t)workspace & 255) == 0, "workspace is required, 256-byte aligned");
    TX = (cam->width + QN_TILE - 1) / QN_TILE;
    TY = (cam->height + QN_TILE - 1) / QN_TILE;
    L = layout_of(n, TX, TY);
    QN_REQUIRE(workspace_bytes >= L.total, "workspace too small (%zu < %zu)", workspace_bytes, L.total);
    return QN_OK;
}

}  // namespace

extern "C" int qn_render_bwd_pairs(const qn_camera *cam_host, int32_t n, const uint32_t *ranges,
                                   const uint32_t *vals, const qn_splat *splats, const float *bg_host,
                                   const float *T_final, const uint32_t *last, const float *d_img,
                                   const uint8_t *skip, const uint8_t *composited, const uint32_t *tile_order,
                                   void *workspace, size_t workspace_bytes, qn_splat *pair_scratch,
                                   qn_stream_t stream) {
    using namespace qn;
    int TX, TY;
    Layout L;
    int st = adjoint_setup(cam_host, n, workspace, workspace_bytes, TX, TY, L);
    if (st) return st;
    char *ws = static_cast<char *>(workspace);
    cudaStream_t s = as_stream(stream);
    if (cudaMemsetAsync(ws + L.hit, 0, (size_t)(n > 0 ? n : 1), s) != cudaSuccess)
        return check_launch("qn_render_bwd memset");
    return launch_render_bwd(cam_host, ranges, vals, splats, bg_host, T_final, last, d_img, skip, composited,
                             tile_order, pair_scratch, reinterpret_cast<uint32_t *>(ws + L.visited),
                             reinterpret_cast<uint8_t *>(ws + L.hit), s);
}

extern "C" int qn_render_bwd_gather(const qn_camera *cam_host, int32_t n, const int32_t *rects, const uint8_t *skip,
                                    const void *workspace, size_t workspace_bytes, const qn_splat *pair_scratch,
                                    qn_splat *d_splats, qn_stream_t stream) {
    using namespace qn;
    int TX, TY;
    Layout L;
    int st = adjoint_setup(cam_host, n, workspace, workspace_bytes, TX, TY, L);
    if (st) return st;
    QN_REQUIRE(n == 0 || (rects && pair_scratch && d_splats), "null pointer argument");
    QN_REQUIRE(((uintptr_t)d_splats & 15) == 0 && ((uintptr_t)pair_scratch & 15) == 0 && ((uintptr_t)rects & 15) == 0,
               "misaligned pointer argument");
    cudaStream_t s = as_stream(stream);
    if (n == 0) return QN_OK;
    if (cudaMemsetAsync(d_splats, 0, sizeof(qn_splat) * (size_t)n, s) != cudaSuccess)
        return check_launch("qn_render_bwd memset");
    const char *ws = static_cast<const char *>(workspace);
    int dev = 0, sms = 148, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bin_gather, GATHER_THREADS, 0) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    // one resident wave: a second one would start only as the first's blocks
    // end, doubling the time of equal strided shares
    const int blocks = (int)std::min<int64_t>(div_up((int64_t)n * 32, GATHER_THREADS), (int64_t)sms * per_sm);
    k_bin_gather<<<blocks, GATHER_THREADS, 0, s>>>(
        TX, TY, reinterpret_cast<const uint32_t *>(ws + L.vals0), reinterpret_cast<const int4 *>(rects),
        reinterpret_cast<const Header *>(ws + L.hdr), reinterpret_cast<const uint32_t *>(ws + L.big),
        reinterpret_cast<const uint32_t *>(ws + L.counts), reinterpret_cast<const uint32_t *>(ws + L.tile_off),
        reinterpret_cast<const uint32_t *>(ws + L.visited), reinterpret_cast<const float4 *>(pair_scratch), skip,
        reinterpret_cast<const uint8_t *>(ws + L.hit), reinterpret_cast<const uint32_t *>(ws + L.masks),
        reinterpret_cast<const uint32_t *>(ws + L.wext), reinterpret_cast<float4 *>(d_splats));
    return check_launch("qn_render_bwd gather");
}

extern "C" int qn_render_bwd(const qn_camera *cam_host, int32_t n, const int32_t *rects, const uint32_t *ranges,
                             const uint32_t *vals, const qn_splat *splats, const float *bg_host, const float *T_final,
                             const uint32_t *last, const float *d_img, const uint8_t *skip,
                             const uint8_t *composited, const uint32_t *tile_order, void *workspace,
                             size_t workspace_bytes, qn_splat *pair_scratch, qn_splat *d_splats, qn_stream_t stream) {
    QN_REQUIRE(n == 0 || (rects && d_splats), "null pointer argument");
    int st = qn_render_bwd_pairs(cam_host, n, ranges, vals, splats, bg_host, T_final, last, d_img, skip, composited,
                                 tile_order, workspace, workspace_bytes, pair_scratch, stream);
    if (st) return st;
    return qn_render_bwd_gather(cam_host, n, rects, skip, workspace, workspace_bytes, pair_scratch, d_splats,
                                stream);
}

// ---------------------------------------------------------------- no-allocation variant
// Workspace of qn_bin_sort_noalloc: a fixed device array, so that callers
// which may not allocate can still bin.  Host code only sees a host-side
// stand-in under this name; the device address comes from
// cudaGetSymbolAddress, looked up once per device with that device current.
static __device__ __align__(256) unsigned char g_bin_scratch[QN_BIN_SORT_STATIC_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void *g_scratch_ptr[kMaxDevices] = {};
}  // namespace

extern "C" int qn_bin_sort_noalloc(int32_t n, const float *depth, int32_t depth_stride, const int32_t *rects,
                                   int32_t tiles_x, int32_t tiles_y, int64_t pair_capacity, uint32_t *vals,
                                   uint64_t *keys, uint32_t *ranges, int64_t *n_pairs, int64_t *n_pairs_host,
                                   qn_stream_t stream) {
    QN_REQUIRE(n >= 0 && tiles_x > 0 && tiles_y > 0, "bad n or tile grid");
    const size_t need = qn_bin_sort_workspace_size(n, tiles_x, tiles_y);
    if (need > (size_t)QN_BIN_SORT_STATIC_BYTES) {
        qn::set_error("qn_bin_sort_noalloc: %d Gaussians on a %dx%d tile grid need %zu bytes of workspace, "
                      "more than the static %u bytes; use qn_bin_sort with a caller workspace",
                      n, tiles_x, tiles_y, need, (unsigned)QN_BIN_SORT_STATIC_BYTES);
        return QN_ERR_INVALID_ARG;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return qn::check_launch("qn_bin_sort_noalloc: cudaGetDevice");
    QN_REQUIRE(dev >= 0 && dev < kMaxDevices, "device ordinal %d out of range", dev);
    void *ptr = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_scratch_mu);
        if (!g_scratch_ptr[dev]) {
            void *p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_bin_scratch);
            if (e != cudaSuccess) {
                qn::set_error("qn_bin_sort_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
                return QN_ERR_CUDA;
            }
            g_scratch_ptr[dev] = p;
        }
        ptr = g_scratch_ptr[dev];
    }
    return qn_bin_sort(n, depth, depth_stride, rects, tiles_x, tiles_y, ptr, (size_t)QN_BIN_SORT_STATIC_BYTES,
                       pair_capacity, vals, keys, ranges, n_pairs, n_pairs_host, stream);
}
