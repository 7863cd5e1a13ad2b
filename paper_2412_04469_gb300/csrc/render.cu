// Front-to-back alpha compositing per 16 x 16 tile (Sec. 3.1, Eq. 2) and its
// adjoint.  A tile is split into horizontal bands of 2 PPT rows, one warp per
// band; a lane owns PPT pixels of one column.  A warp walks only the staged
// records that can reach its band (one analytic test per record, lane j
// testing record j).  The forward keeps each pixel as a scalar chain; the
// adjoint works on its pixels in pairs with Blackwell's packed FP32
// instructions (add/sub/mul/fma .f32x2: two lanes of arithmetic per issued
// instruction), its staged records holding every per-Gaussian scalar
// duplicated into a pair, so a 128-bit broadcast load yields operand pairs.
#include "bins.cuh"
#include "common.cuh"
#include "packed.cuh"

namespace qn {
namespace {

constexpr float ALPHA_MIN = 1.f / 255.f;
constexpr float ALPHA_MAX = 0.99f;
constexpr float T_MIN = 1e-4f;
constexpr float LOG2E = 1.4426950408889634f;
// A band whose pixels all have log2(e) power below -log2(255 o) minus this
// margin (far wider than the rounding of ex2 and log2) cannot pass the
// alpha >= 1/255 test anywhere and skips the Gaussian: the cull never changes
// a result.
constexpr float CULL_MARGIN = 1e-3f;
// Below this opacity no pixel's alpha reaches ALPHA_MAX: alpha = o 2^e with
// e <= 0 up to the rounding of the exponent (a positive e stays far below
// 1e-5), so alpha <= o (1 + 1e-5) < 0.99.
constexpr float CAP_FREE_OPACITY = 0.98997f;
template <bool B>
struct CapTag {
    static constexpr bool value = B;
};

// pixels per lane (even): 16 x 16 / (32 PPT) warps per tile
#ifndef QN_FWD_PPT
#define QN_FWD_PPT 4
#endif
#ifndef QN_BWD_PPT
#define QN_BWD_PPT 4
#endif

template <int PPT>
struct Band {
    static_assert(PPT % 2 == 0 && QN_TILE % (2 * PPT) == 0, "pixels per lane");
    static constexpr int NP = PPT / 2;                  // packed pairs per lane
    static constexpr int WARPS = QN_TILE / (2 * PPT);   // warps per tile
    static constexpr int THREADS = 32 * WARPS;
};

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// ---------------------------------------------------------------- band cull
// Whether some pixel centre of the band [x0, x1] x [y0, y1] can reach
// log2(e) power e >= kw, e = A dx^2 + B dx dy + C dy^2 (A, C < 0): the
// maximum of e over the rectangle is 0 when the mean lies inside it, else it
// lies on an edge at the stationary point clamped to that edge.  The margin
// covers the FP32 rounding of this maximum and of the per-pixel exponent
// (both a few ulps of the largest term), so the test never rejects a
// Gaussian some pixel of the band composites.  One lane tests one record, so
// a batch of 32 records costs each lane one test instead of one per record.
__device__ __forceinline__ bool band_reaches(float mx, float my, float A, float B, float C, float kw, float x0,
                                             float x1, float y0, float y1) {
    const float lx = x0 - mx, hx = x1 - mx, ly = y0 - my, hy = y1 - my;
    float em;
    if (lx <= 0.f && hx >= 0.f && ly <= 0.f && hy >= 0.f) {
        em = 0.f;
    } else {
        const float sa = __fdividef(-0.5f, A), sc = __fdividef(-0.5f, C);
        em = -INFINITY;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const float dy = k ? hy : ly;
            const float dx = fminf(fmaxf(B * dy * sa, lx), hx);
            em = fmaxf(em, fmaf(dx, fmaf(A, dx, B * dy), C * dy * dy));
            const float ex = k ? hx : lx;
            const float ey = fminf(fmaxf(B * ex * sc, ly), hy);
            em = fmaxf(em, fmaf(ey, fmaf(C, ey, B * ex), A * ex * ex));
        }
    }
    const float ax = fmaxf(-lx, hx), ay = fmaxf(-ly, hy);
    const float mag = fmaf(-A, ax * ax, fmaf(fabsf(B), ax * ay, -C * ay * ay));
    return em >= kw - fmaf(1e-6f, mag, 1e-3f);
}

// ---------------------------------------------------------------- staged record
// log2(e) power = A dx^2 + B dx dy + C dy^2 with A = -a log2(e) / 2,
// B = -b log2(e), C = -c log2(e) / 2 (conic (a, b, c)), dx = x - mean_x.
struct __align__(16) Rec {
    f2 mx, my;      // mean
    f2 A, B;        // scaled conic
    f2 C, o;        // scaled conic, opacity
    f2 cr, cg;      // colour
    f2 cb;
    float kw;       // cull bound -log2(255 o) - margin
    uint32_t id;    // Gaussian index
};

__device__ __forceinline__ void stage_rec(Rec &r, float4 g0, float4 g1, float4 g2, uint32_t id) {
    const float A = __fmul_rn(-0.5f * LOG2E, g1.x), B = __fmul_rn(-LOG2E, g1.y), C = __fmul_rn(-0.5f * LOG2E, g1.z);
    r.mx = pk(g0.x, g0.x);
    r.my = pk(g0.y, g0.y);
    r.A = pk(A, A);
    r.B = pk(B, B);
    r.C = pk(C, C);
    r.o = pk(g0.z, g0.z);
    r.cr = pk(g2.x, g2.x);
    r.cg = pk(g2.y, g2.y);
    r.cb = pk(g2.z, g2.z);
    r.kw = g0.z > 0.f ? -log2f(255.f * g0.z) - CULL_MARGIN : INFINITY;
    r.id = id;
}

// The exponent at the lane's pixel pairs, with explicit round-to-nearest
// operations so that the forward pass and the adjoint evaluate bit-identical
// alphas and take identical decisions:
//   dx = x - mx, dy = y - my, e = fma(dy, fma(C, dy, B dx), (A dx) dx).
template <int NP>
struct Expo {
    f2 dx;          // (dx, dx)
    f2 dy[NP], e[NP];
};

template <int NP>
__device__ __forceinline__ Expo<NP> exponent(const Rec &r, f2 FX, const f2 (&FY)[NP]) {
    Expo<NP> x;
    x.dx = sub2(FX, r.mx);
    const f2 p0 = mul2(mul2(r.A, x.dx), x.dx);
    const f2 bdx = mul2(r.B, x.dx);
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        x.dy[p] = sub2(FY[p], r.my);
        x.e[p] = fma2(x.dy[p], fma2(r.C, x.dy[p], bdx), p0);
    }
    return x;
}

template <int PPT>
__device__ __forceinline__ void pixel_coords(int tile, int TX, int &px, int &py0) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    px = (tile % TX) * QN_TILE + (lane & 15);
    py0 = (tile / TX) * QN_TILE + warp * (2 * PPT) + (lane >> 4) * PPT;
}

// ---------------------------------------------------------------- unwritten lists
// A warp's walk of its tile's list when the binning did not write it (the
// layout is described with BinView).  The warp lists the tile's members up to
// 32 chunks at a time into a ring of depth-sorted indices in shared memory,
// in list order, and a batch reads its 32 positions from the ring.  The
// chunks come from the tile's occupancy bits (the chunks holding a member of
// the tile, 32 bits a lane, 1024 chunks a warp-wide block), so a sparse tile
// skips its empty chunks: lane l takes the l-th occupied chunk from the
// cursor on, loads that chunk's eight words for the tile, and a scan of their
// member counts places each chunk's members.  Chunks are taken while the ring
// has room (a chunk holds at most 256 members of a tile, and fewer than 32
// listed members are unread when more are listed, so the first always fits).
constexpr int WALK_RING = 512;                          // per warp, a power of two >= 256 + 32

struct ListWalk {
    int cur;                 // the next chunk to consider
    int ob;                  // the occupancy block held (words 32 ob .. 32 ob + 31)
    uint32_t ow;             // lane l: occupancy word 32 ob + l
    uint32_t listed;         // members listed so far (list positions 0 .. listed - 1)
};

// Position of the r-th (from 0) set bit of m (r < popc(m)).
__device__ __forceinline__ int nth_set_bit(uint32_t m, int r) {
    int pos = 0;
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
        const int c = __popc(m & ((1u << s) - 1u));
        if (r >= c) {
            r -= c;
            m >>= s;
            pos += s;
        }
    }
    return pos;
}

__device__ __forceinline__ void walk_window(ListWalk &lw, uint32_t *ring, uint32_t consumed, const BinView &bins,
                                            int TX, int TY, int tx, int ty, int nchunks, int lane) {
    static_assert(BIN_CHUNK_WARPS == 8, "a tile's words of one chunk are two uint4");
    static_assert((WALK_RING & (WALK_RING - 1)) == 0 && WALK_RING >= BIN_CHUNK + 32, "ring size");
    const size_t n_tiles = (size_t)TX * TY, t = (size_t)ty * TX + tx;
    // the occupied chunks from the cursor on, within the block held; an
    // exhausted block gives way to the next
    uint32_t m, mexcl, mtot;
    for (;;) {
        const int wl = 32 * lw.ob + lane, wc = lw.cur >> 5;
        m = wl < wc ? 0u : (wl == wc ? lw.ow & (~0u << (lw.cur & 31)) : lw.ow);
        const uint32_t mc = __popc(m);
        uint32_t incl = mc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t x = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += x;
        }
        mexcl = incl - mc;
        mtot = __shfl_sync(FULL, incl, 31);
        if (mtot > 0) break;
        lw.ob += 1;
        lw.cur = 1024 * lw.ob;
        if (lw.cur >= nchunks) return;                  // no chunk left
        const int w = 32 * lw.ob + lane;
        lw.ow = w < bins.occ_w ? bins.occ[(size_t)w * n_tiles + t] : 0u;
    }
    // lane l: the l-th occupied chunk (the word by a binary search over the
    // words' counts, then the bit)
    int L = 0;
#pragma unroll
    for (int st = 16; st > 0; st >>= 1) {
        const uint32_t e = __shfl_sync(FULL, mexcl, L + st);
        if (e <= (uint32_t)lane) L += st;
    }
    const uint32_t r = (uint32_t)lane - __shfl_sync(FULL, mexcl, L);
    const uint32_t word = __shfl_sync(FULL, m, L);
    const bool valid = (uint32_t)lane < mtot;
    const int c = valid ? 32 * (32 * lw.ob + L) + nth_set_bit(word, (int)r) : 0;
    uint32_t w[BIN_CHUNK_WARPS] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
    if (valid) {
        // 16-byte aligned: the workspace's mask array is, a chunk's words take
        // 32 (TX + TY) bytes and a column's / row's 32
        const uint4 *mx = reinterpret_cast<const uint4 *>(bins.masks + (size_t)c * BIN_CHUNK_WARPS * (TX + TY));
        const uint4 x0 = mx[2 * tx], x1 = mx[2 * tx + 1], y0 = mx[2 * TX + 2 * ty], y1 = mx[2 * TX + 2 * ty + 1];
        w[0] = x0.x & y0.x; w[1] = x0.y & y0.y; w[2] = x0.z & y0.z; w[3] = x0.w & y0.w;
        w[4] = x1.x & y1.x; w[5] = x1.y & y1.y; w[6] = x1.z & y1.z; w[7] = x1.w & y1.w;
    }
    uint32_t cnt = 0;
#pragma unroll
    for (int i = 0; i < BIN_CHUNK_WARPS; ++i) cnt += __popc(w[i]);
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t x = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += x;
    }
    const uint32_t room = (uint32_t)WALK_RING - (lw.listed - consumed);
    const bool take = valid && incl <= room;            // the chunks that fit: a prefix of the lanes
    const int ntake = __popc(__ballot_sync(FULL, take));
    if (take) {
        uint32_t pos = lw.listed + incl - cnt;
        bins.gbase[(size_t)c * n_tiles + t] = pos;      // the chunk's first list position in the tile
        const uint32_t g0 = (uint32_t)c * BIN_CHUNK;
#pragma unroll
        for (int i = 0; i < BIN_CHUNK_WARPS; ++i) {
            for (uint32_t b = w[i]; b; b &= b - 1) ring[pos++ & (WALK_RING - 1)] = g0 + 32 * i + (__ffs(b) - 1);
        }
    }
    lw.listed += __shfl_sync(FULL, incl, ntake - 1);
    const int nfill = (int)min(mtot, 32u);
    lw.cur = ntake < nfill ? __shfl_sync(FULL, c, ntake) : __shfl_sync(FULL, c, ntake - 1) + 1;
    __syncwarp();
}

// ---------------------------------------------------------------- forward
// Every warp composites its band independently: it stages its own copy of
// each batch of records (48 bytes: mean, opacity, scaled conic and cull bound,
// colour) and stops when its pixels have all terminated.  A lane owns
// FWD_PPT pixels of one column as independent scalar chains (packing them
// buys no FP32 throughput here, and the forward's alpha test and update are
// mostly compares and selects).  The per-pixel update is branch-free
// (an effective alpha that is 0 unless the Gaussian is taken).  Per pixel:
//   alpha = min(0.99, o 2^e); skipped if alpha < 1/255 (e <= 0 holds for a
//   positive definite conic, so its sign is not tested: a positive FP32 e
//   only arises from rounding at the footprint's centre);
//   stop before the Gaussian if T (1 - alpha) < 1e-4;
//   C += c alpha T; T -= alpha T.
// comp (nullable): set to 1 for every Gaussian some pixel composites (one
// store per composited record and warp, after each batch).  order
// (nullable): block b composites tile order[b] (heaviest first: the blocks
// start in index order, and a deep tile that starts late sets the kernel's
// end).  cost (nullable): each tile's visited prefix, the largest `last` of
// its pixels, the work measure that orders the next launches.
constexpr int FWD_BATCH = 32;

struct SRec {
    float4 g;   // (mean x, mean y, opacity, cull bound -log2(255 o) - margin)
    float4 k;   // scaled conic (A, B, C, -)
    float4 c;   // colour (r, g, b, -)
};

__device__ __forceinline__ void stage_srec(SRec &r, float4 g0, float4 g1, float4 g2) {
    r.g = make_float4(g0.x, g0.y, g0.z, g0.z > 0.f ? -log2f(255.f * g0.z) - CULL_MARGIN : INFINITY);
    r.k = make_float4(__fmul_rn(-0.5f * LOG2E, g1.x), __fmul_rn(-LOG2E, g1.y), __fmul_rn(-0.5f * LOG2E, g1.z), 0.f);
    r.c = g2;
}

// log2(e) power at the lane's PPT pixels, the same round-to-nearest sequence
// as exponent(): dx = x - mx, dy = y - my, e = fma(dy, fma(C, dy, B dx), (A dx) dx).
template <int PPT>
__device__ __forceinline__ void scalar_exponent(const SRec &r, float fx, float fy0, float (&e)[PPT]) {
    const float dx = __fsub_rn(fx, r.g.x);
    const float p0 = __fmul_rn(__fmul_rn(r.k.x, dx), dx), bdx = __fmul_rn(r.k.y, dx);
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        const float dy = __fsub_rn(fy0 + (float)q, r.g.y);
        e[q] = __fmaf_rn(dy, __fmaf_rn(r.k.z, dy, bdx), p0);
    }
}

// COUNT: write the contributor counts; MARK: set the composited marks.
// LAZY: only the lists of at most list_max pairs were written (to vals); for
// a longer list each warp walks it from the binning's chunk masks (BinView)
// and writes the positions it walks to vals_out (both warps of a tile write
// the same values), so that the list's walked prefix is there for the adjoint.
template <bool COUNT, bool MARK, int PPT, bool LAZY>
__global__ void __launch_bounds__(Band<PPT>::THREADS) k_render_fwd(int W, int H, int TX, int TY,
                                                                  const uint32_t *__restrict__ ranges,
                                                                  const uint32_t *__restrict__ vals,
                                                                  BinView bins, uint32_t *__restrict__ vals_out,
                                                                  const float4 *__restrict__ sp, float bg0, float bg1,
                                                                  float bg2, float *__restrict__ img,
                                                                  float *__restrict__ Tf, uint32_t *__restrict__ last,
                                                                  uint32_t *__restrict__ ncon,
                                                                  uint8_t *__restrict__ comp,
                                                                  const uint32_t *__restrict__ order,
                                                                  uint32_t *__restrict__ cost) {
    constexpr int WARPS = Band<PPT>::WARPS;
    __shared__ SRec sbuf[WARPS][FWD_BATCH];
    __shared__ uint32_t wmax[WARPS];
    __shared__ uint32_t ring[LAZY ? WARPS : 1][LAZY ? WALK_RING : 1];
    SRec *s = sbuf[threadIdx.x >> 5];
    const int tile = order ? (int)order[blockIdx.x] : (int)blockIdx.x;
    const int lane = threadIdx.x & 31;
    int px, py0;
    pixel_coords<PPT>(tile, TX, px, py0);
    const uint32_t beg = ranges[2 * tile], end = ranges[2 * tile + 1];
    const int n = (int)(end - beg);
    const float fx = px + 0.5f, fy0 = py0 + 0.5f;
    // T < 0 marks a pixel that has stopped (its T negated) or lies outside
    // the image: T (1 - alpha) is then negative and fails the 1e-4 test, so
    // the per-pixel update needs no separate liveness test
    float T[PPT], c0[PPT], c1[PPT], c2[PPT];
    uint32_t lastc[PPT], nc[PPT];
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        T[q] = px < W && py0 + q < H ? 1.f : -1.f;
        c0[q] = c1[q] = c2[q] = 0.f;
        lastc[q] = nc[q] = 0;
    }
    // the warp's band of pixel centres, clipped to the image
    const float bx0 = (float)((tile % TX) * QN_TILE) + 0.5f, bx1 = fminf(bx0 + (float)(QN_TILE - 1), W - 0.5f);
    const float by0 = (float)((tile / TX) * QN_TILE + (threadIdx.x >> 5) * (2 * PPT)) + 0.5f;
    const float by1 = fminf(by0 + (float)(2 * PPT - 1), H - 0.5f);
    // LAZY: a list longer than list_max was not written and is walked here
    const bool walk = LAZY && (uint32_t)n > __ldg(bins.list_max);
    const int nchunks = walk ? (int)((__ldg(bins.n_vis) + BIN_CHUNK - 1) / BIN_CHUNK) : 0;
    ListWalk lw{0, 0, 0u, 0u};
    if (walk && lane < bins.occ_w) lw.ow = bins.occ[(size_t)lane * TX * TY + tile];
    for (int b0 = 0; b0 < n; b0 += FWD_BATCH) {
        bool live = false;                              // the warp stops between batches
#pragma unroll
        for (int q = 0; q < PPT; ++q) live |= T[q] > 0.f;
        if (!__any_sync(FULL, live)) break;
        uint32_t my_id = 0;
        bool reach = false;
        bool have = b0 + lane < n;
        if (LAZY && walk) {
            uint32_t *rg = ring[threadIdx.x >> 5];
            const uint32_t need = (uint32_t)min(n, b0 + FWD_BATCH);
            while (lw.listed < need && lw.cur < nchunks)
                walk_window(lw, rg, (uint32_t)b0, bins, TX, TY, tile % TX, tile / TX, nchunks, lane);
            have = have && (uint32_t)(b0 + lane) < lw.listed;   // (always, for a list consistent with the masks)
            if (have) {
                my_id = bins.sorted[rg[(b0 + lane) & (WALK_RING - 1)]];
                vals_out[beg + b0 + lane] = my_id;
            }
        } else if (have) {
            my_id = vals[beg + b0 + lane];
        }
        if (have) {
            SRec rr;
            stage_srec(rr, sp[3 * (size_t)my_id], sp[3 * (size_t)my_id + 1], sp[3 * (size_t)my_id + 2]);
            s[lane] = rr;
            reach = band_reaches(rr.g.x, rr.g.y, rr.k.x, rr.k.y, rr.k.z, rr.g.w, bx0, bx1, by0, by1);
        }
        uint32_t todo = __ballot_sync(FULL, reach);     // the records some pixel of the band can take
        __syncwarp();
        uint32_t batch_added = 0;                       // bit j: record j composited by this warp
        while (todo) {
            const int j = __ffs(todo) - 1;              // front to back
            todo &= todo - 1;
            const SRec &r = s[j];
            float e[PPT];
            scalar_exponent<PPT>(r, fx, fy0, e);
            const float4 c = r.c;
            const uint32_t pos1 = (uint32_t)(b0 + j + 1);
            bool added = false;
            // CAP: the record can reach the 0.99 cap (below CAP_FREE_OPACITY,
            // min(alpha, 0.99) is alpha; the branch is uniform over the warp)
            auto pixels = [&](auto cap_tag) {
                constexpr bool CAP = decltype(cap_tag)::value;
#pragma unroll
                for (int q = 0; q < PPT; ++q) {
                    const float v = __fmul_rn(r.g.z, ex2_approx(e[q]));
                    const float al = CAP ? fminf(v, ALPHA_MAX) : v;
                    const bool ok = al >= ALPHA_MIN;
                    const bool add = ok && __fmul_rn(T[q], __fsub_rn(1.f, al)) >= T_MIN;
                    // the update through the effective alpha ae (0 unless added):
                    // T <- T - ae T, C <- C + c ae T, on the FMA pipe; a pixel
                    // that stops before this Gaussian keeps -|T|
                    const float ae = add ? al : 0.f;
                    const float w = __fmul_rn(ae, T[q]);
                    c0[q] = fmaf(c.x, w, c0[q]);
                    c1[q] = fmaf(c.y, w, c1[q]);
                    c2[q] = fmaf(c.z, w, c2[q]);
                    T[q] = ok && !add ? -fabsf(T[q]) : __fsub_rn(T[q], w);
                    lastc[q] = add ? pos1 : lastc[q];
                    if (COUNT) nc[q] += add ? 1u : 0u;
                    if (MARK) added |= add;
                }
            };
            if (r.g.z > CAP_FREE_OPACITY) pixels(CapTag<true>{});
            else pixels(CapTag<false>{});
            if (MARK && __any_sync(FULL, added)) batch_added |= 1u << j;
        }
        if (MARK && ((batch_added >> lane) & 1u)) comp[my_id] = 1;
        __syncwarp();
    }
    const size_t plane = (size_t)W * H;
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        const int py = py0 + q;
        if (px >= W || py >= H) continue;
        const size_t o = (size_t)py * W + px;
        const float t = fabsf(T[q]);
        img[o] = fmaf(t, bg0, c0[q]);
        img[plane + o] = fmaf(t, bg1, c1[q]);
        img[2 * plane + o] = fmaf(t, bg2, c2[q]);
        Tf[o] = t;
        last[o] = lastc[q];
        if (COUNT) ncon[o] = nc[q];
    }
    if constexpr (LAZY) {
        // the walked chunk extent of the tile (the warps' furthest cursor)
        __shared__ uint32_t wcur[WARPS];
        if (lane == 0) wcur[threadIdx.x >> 5] = walk ? (uint32_t)lw.cur : 0u;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t e = 0;
#pragma unroll
            for (int w = 0; w < WARPS; ++w) e = max(e, wcur[w]);
            bins.wext[tile] = e;
        }
    }
    if (cost) {
        uint32_t m = 0;
#pragma unroll
        for (int q = 0; q < PPT; ++q) m = max(m, lastc[q]);
        m = __reduce_max_sync(FULL, m);
        if (lane == 0) wmax[threadIdx.x >> 5] = m;
        __syncthreads();
        if (threadIdx.x == 0) {
#pragma unroll
            for (int w = 1; w < WARPS; ++w) m = max(m, wmax[w]);
            cost[tile] = m;
        }
    }
}

// ---------------------------------------------------------------- adjoint
// Adjoint of k_render_fwd for one tile, walking its list back to front from
// the last contributor of any of its pixels.  Per pixel the walk rebuilds T in
// front of each Gaussian by division by (1 - alpha) and carries the scalar
// b = B . dL/dC, B the colour behind the Gaussian (B = bg behind the last
// contributor, B <- alpha c + (1 - alpha) B past each one), so that
//   dL/dalpha = T (c . dL/dC - b),   b <- b + alpha (c . dL/dC - b),
//   dL/dc = alpha T dL/dC,           dL/dpower = dL/dalpha alpha (0 if capped).
// Per (lane, Gaussian) the lane accumulates over its pixels s = dL/dpower
// and the moments sum s, sum s dy, sum s dy^2 (dx is shared by the column)
// and the colour sums; each warp sums them with a fixed shuffle pattern, the
// warps' sums are added in warp order, and the record of the pair is formed
// once from the conic (a, b, c):
//   dL/dmean = (a Sx + b Sy, b Sx + c Sy),
//   dL/d(a, b, c) = (-Sxx / 2, -Sxy, -Syy / 2),
//   dL/do = sum s / o   (alpha = o G: dalpha/do = G = alpha / o),
// since power = -(a dx^2 + c dy^2) / 2 - b dx dy and dx = x - mean_x.
// skip (nullable): no record for those Gaussians.  comp (nullable): the
// forward's composited marks; a Gaussian without one changes no pixel, so it
// is dropped from the walk before any arithmetic (skipped or not).  A skipped
// Gaussian that is composited still enters T and b.  hit: set to 1 for every
// Gaussian that gets a record with a contribution.  order (nullable): block b
// walks tile order[b].
template <int PPT>
__global__ void __launch_bounds__(Band<PPT>::THREADS) k_render_bwd(int W, int H, int TX,
                                                                  const uint32_t *__restrict__ ranges,
                                                                  const uint32_t *__restrict__ vals,
                                                                  const float4 *__restrict__ sp, float bg0, float bg1,
                                                                  float bg2, const float *__restrict__ Tf,
                                                                  const uint32_t *__restrict__ last,
                                                                  const float *__restrict__ dimg,
                                                                  const uint8_t *__restrict__ skip,
                                                                  const uint8_t *__restrict__ comp,
                                                                  float4 *__restrict__ pair_grads,
                                                                  uint32_t *__restrict__ visited,
                                                                  uint8_t *__restrict__ hitg,
                                                                  const uint32_t *__restrict__ order) {
    constexpr int NP = Band<PPT>::NP, WARPS = Band<PPT>::WARPS, BATCH = Band<PPT>::THREADS;
    __shared__ Rec s[BATCH];
    __shared__ float rec[WARPS][BATCH][9];
    __shared__ uint8_t hit[WARPS][BATCH];
    __shared__ uint8_t sflag[BATCH];                    // bit 0: skipped, bit 1: composited nowhere
    __shared__ uint32_t wmax[WARPS];
    const int tile = order ? (int)order[blockIdx.x] : (int)blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int px, py0;
    pixel_coords<PPT>(tile, TX, px, py0);
    const uint32_t beg = ranges[2 * tile];
    const float fx = px + 0.5f, fy0 = py0 + 0.5f;
    const f2 FX = pk(fx, fx), ONE = pk(1.f, 1.f);
    f2 FY[NP], T[NP], Bd[NP], D0[NP], D1[NP], D2[NP];
    uint32_t lastp[PPT];
    uint32_t mymax = 0;
    const size_t plane = (size_t)W * H;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        float t[2] = {1.f, 1.f}, d0[2] = {0.f, 0.f}, d1[2] = {0.f, 0.f}, d2[2] = {0.f, 0.f}, b[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int q = 2 * p + h, py = py0 + q;
            lastp[q] = 0;
            if (px < W && py < H) {
                const size_t o = (size_t)py * W + px;
                t[h] = Tf[o];
                lastp[q] = last[o];
                d0[h] = dimg[o];
                d1[h] = dimg[plane + o];
                d2[h] = dimg[2 * plane + o];
            }
            b[h] = fmaf(bg2, d2[h], fmaf(bg1, d1[h], bg0 * d0[h]));      // colour behind = background
            mymax = max(mymax, lastp[q]);
        }
        FY[p] = pk(fy0 + (float)(2 * p), fy0 + (float)(2 * p + 1));
        T[p] = pk(t[0], t[1]);
        Bd[p] = pk(b[0], b[1]);
        D0[p] = pk(d0[0], d0[1]);
        D1[p] = pk(d1[0], d1[1]);
        D2[p] = pk(d2[0], d2[1]);
    }
    const uint32_t wm = __reduce_max_sync(FULL, mymax);
    if (lane == 0) wmax[warp] = wm;
    // the warp's band of pixel centres, clipped to the image
    const float bx0 = (float)((tile % TX) * QN_TILE) + 0.5f, bx1 = fminf(bx0 + (float)(QN_TILE - 1), W - 0.5f);
    const float by0 = (float)((tile / TX) * QN_TILE + warp * (2 * PPT)) + 0.5f;
    const float by1 = fminf(by0 + (float)(2 * PPT - 1), H - 0.5f);
    __syncthreads();
    uint32_t tmax = 0;
#pragma unroll
    for (int w = 0; w < WARPS; ++w) tmax = max(tmax, wmax[w]);
    const int n = (int)tmax;
    if (threadIdx.x == 0) visited[tile] = tmax;
    for (int hi = n; hi > 0; hi -= BATCH) {
        const int lo = max(0, hi - BATCH);
        const int cnt = hi - lo;
        const int t = threadIdx.x;
        float4 conic = make_float4(0.f, 0.f, 0.f, 0.f);   // thread t: raw conic and opacity of record lo + t
        float opac = 0.f;
        bool my_skip = true;
        uint32_t id = 0;
        if (t < cnt) {
            id = vals[beg + lo + t];
            my_skip = skip ? skip[id] != 0 : false;
            const bool inert = comp ? comp[id] == 0 : false;
            sflag[t] = (my_skip ? 1 : 0) | (inert ? 2 : 0);
            if (!inert) {
                const float4 g0 = sp[3 * (size_t)id];
                conic = sp[3 * (size_t)id + 1];
                opac = g0.z;
                stage_rec(s[t], g0, conic, sp[3 * (size_t)id + 2], id);
            }
        }
        __syncthreads();
        for (int k = lane; k < BATCH; k += 32) hit[warp][k] = 0;
        __syncwarp();
        // back to front over chunks of 32 records: lane l tests record
        // 32 c + l against the warp's band (composited somewhere, inside the
        // band's walked prefix, reaching one of its pixel centres)
#pragma unroll 1
        for (int ch = BATCH / 32 - 1; ch >= 0; --ch) {
            const int jt = ch * 32 + lane;
            bool reach = false;
            if (jt < cnt && !(sflag[jt] & 2) && (uint32_t)(lo + jt) < wm) {
                const Rec &q = s[jt];
                float mxs, mys, qa, qb, qc, unused;
                upk(q.mx, mxs, unused);
                upk(q.my, mys, unused);
                upk(q.A, qa, unused);
                upk(q.B, qb, unused);
                upk(q.C, qc, unused);
                reach = band_reaches(mxs, mys, qa, qb, qc, q.kw, bx0, bx1, by0, by1);
            }
            uint32_t todo = __ballot_sync(FULL, reach);
            while (todo) {
                const int jb = 31 - __clz(todo);
                todo &= ~(1u << jb);
                const int j = ch * 32 + jb;
                const uint32_t pos = (uint32_t)(lo + j);
                const Rec r = s[j];
                // no per-pixel cull beyond the band test: it would reject about 5% of
                // the records that pass it, for more instructions than those cost
                const Expo<NP> x = exponent<NP>(r, FX, FY);
                if (sflag[j] & 1) {
                    // skipped (the branch is uniform over the block): it only
                    // enters the transmittance and b of the Gaussians in front
#pragma unroll
                    for (int p = 0; p < NP; ++p) {
                        float e0, e1, v0, v1, m0, m1;
                        upk(x.e[p], e0, e1);
                        upk(mul2(r.o, pk(ex2_approx(e0), ex2_approx(e1))), v0, v1);
                        const float a0 = fminf(v0, ALPHA_MAX), a1 = fminf(v1, ALPHA_MAX);
                        const bool ok0 = pos < lastp[2 * p] && a0 >= ALPHA_MIN;
                        const bool ok1 = pos < lastp[2 * p + 1] && a1 >= ALPHA_MIN;
                        const f2 AE = pk(ok0 ? a0 : 0.f, ok1 ? a1 : 0.f);
                        upk(sub2(ONE, AE), m0, m1);
                        T[p] = mul2(T[p], pk(ok0 ? rcp_approx(m0) : 1.f, ok1 ? rcp_approx(m1) : 1.f));
                        const f2 cd = fma2(r.cr, D0[p], fma2(r.cg, D1[p], mul2(r.cb, D2[p])));
                        Bd[p] = fma2(AE, sub2(cd, Bd[p]), Bd[p]);
                    }
                    continue;
                }
                const f2 Z = pk(0.f, 0.f);
                f2 S0 = Z, S1 = Z, S2 = Z, G0 = Z, G1 = Z, G2 = Z;
                bool any = false;
                // CAP: the record can reach the 0.99 cap.  alpha = o 2^e <= o (1 + 1e-5)
                // (e <= 0 up to rounding), so below CAP_FREE_OPACITY min(alpha, 0.99)
                // is alpha and the cap's zero gradient never applies: the branch
                // without them gives the same bits with fewer instructions
                auto walk = [&](auto cap_tag) {
                    constexpr bool CAP = decltype(cap_tag)::value;
#pragma unroll
                    for (int p = 0; p < NP; ++p) {
                        float e0, e1, v0, v1, m0, m1;
                        upk(x.e[p], e0, e1);
                        upk(mul2(r.o, pk(ex2_approx(e0), ex2_approx(e1))), v0, v1);
                        const float a0 = CAP ? fminf(v0, ALPHA_MAX) : v0, a1 = CAP ? fminf(v1, ALPHA_MAX) : v1;
                        const bool ok0 = pos < lastp[2 * p] && a0 >= ALPHA_MIN;
                        const bool ok1 = pos < lastp[2 * p + 1] && a1 >= ALPHA_MIN;
                        any |= ok0 | ok1;
                        const float ae0 = ok0 ? a0 : 0.f, ae1 = ok1 ? a1 : 0.f;
                        const f2 AE = pk(ae0, ae1);
                        const f2 AG = CAP ? pk(v0 > ALPHA_MAX ? 0.f : ae0, v1 > ALPHA_MAX ? 0.f : ae1)   // the cap passes no gradient
                                          : AE;
                        upk(sub2(ONE, AE), m0, m1);
                        const f2 TQ = mul2(T[p], pk(ok0 ? rcp_approx(m0) : 1.f, ok1 ? rcp_approx(m1) : 1.f));  // in front of j
                        T[p] = TQ;
                        const f2 cd = fma2(r.cr, D0[p], fma2(r.cg, D1[p], mul2(r.cb, D2[p])));
                        const f2 dot = sub2(cd, Bd[p]);
                        Bd[p] = fma2(AE, dot, Bd[p]);
                        const f2 w = mul2(AE, TQ);
                        G0 = fma2(w, D0[p], G0);
                        G1 = fma2(w, D1[p], G1);
                        G2 = fma2(w, D2[p], G2);
                        const f2 sdp = mul2(mul2(TQ, dot), AG);           // dL/dpower
                        const f2 tt = mul2(sdp, x.dy[p]);
                        S0 = add2(S0, sdp);
                        S1 = add2(S1, tt);
                        S2 = fma2(tt, x.dy[p], S2);
                    }
                };
                float o_j, o_unused;
                upk(r.o, o_j, o_unused);
                if (o_j > CAP_FREE_OPACITY) walk(CapTag<true>{});   // uniform over the warp: one record
                else walk(CapTag<false>{});
                const bool any_j = __any_sync(FULL, any);   // the band composites j
                if (lane == 0) hit[warp][j] = any_j;
                if (!any_j) continue;
                float h0, h1, dx, dxx;
                upk(x.dx, dx, dxx);
                upk(S0, h0, h1);
                const float s0 = h0 + h1;
                upk(S1, h0, h1);
                const float s1 = h0 + h1;
                upk(S2, h0, h1);
                const float s2 = h0 + h1;
                upk(G0, h0, h1);
                const float g0 = h0 + h1;
                upk(G1, h0, h1);
                const float g1 = h0 + h1;
                upk(G2, h0, h1);
                const float g2 = h0 + h1;
                const float sx = dx * s0;
                float v[8] = {s0, sx, s1, dx * sx, dx * s1, s2, g0, g1};
                const float red = reduce_scatter8(v, lane);
                const float red8 = warp_sum(g2);
                if ((lane & 3) == 0) rec[warp][j][(lane >> 2) & 7] = red;
                if (lane == 0) rec[warp][j][8] = red8;
            }
        }
        __syncthreads();
        // one record per visited list position: the tile's sum for that Gaussian
        if (t < cnt && !my_skip && !(sflag[t] & 2)) {
            float m[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            bool contributed = false;
#pragma unroll
            for (int w = 0; w < WARPS; ++w) {
                if (!hit[w][t]) continue;
                contributed = true;
#pragma unroll
                for (int q = 0; q < 9; ++q) m[q] += rec[w][t][q];
            }
            if (contributed) hitg[id] = 1;
            // m = (S, Sx, Sy, Sxx, Sxy, Syy, dr, dg, db)
            const float d_o = opac > 0.f ? __fdiv_rn(m[0], opac) : 0.f;
            float4 *d = pair_grads + 3 * (size_t)(beg + lo + t);
            d[0] = make_float4(conic.x * m[1] + conic.y * m[2], conic.y * m[1] + conic.z * m[2], d_o, 0.f);
            d[1] = make_float4(-0.5f * m[3], -m[4], -0.5f * m[5], 0.f);
            d[2] = make_float4(m[6], m[7], m[8], 0.f);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- tile order
// Counting sort of the tiles by descending cost in one block: bucket
// min(cost, ORDER_BUCKETS - 1), heaviest bucket first.  The order inside a
// bucket depends on atomic timing; no result depends on the order.
constexpr int ORDER_BUCKETS = 1024;

__global__ void __launch_bounds__(1024) k_tile_order(int n_tiles, const uint32_t *__restrict__ cost,
                                                     uint32_t *__restrict__ order) {
    __shared__ uint32_t cnt[ORDER_BUCKETS];
    __shared__ uint32_t wsum[32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    cnt[t] = 0;
    __syncthreads();
    for (int i = t; i < n_tiles; i += 1024) atomicAdd(&cnt[ORDER_BUCKETS - 1 - min(cost[i], ORDER_BUCKETS - 1u)], 1u);
    __syncthreads();
    // exclusive scan of the 1024 bucket counts
    const uint32_t c = cnt[t];
    uint32_t x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = wsum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, w, o);
            if (lane >= o) w += y;
        }
        wsum[lane] = w;
    }
    __syncthreads();
    cnt[t] = x - c + (warp ? wsum[warp - 1] : 0u);
    __syncthreads();
    for (int i = t; i < n_tiles; i += 1024)
        order[atomicAdd(&cnt[ORDER_BUCKETS - 1 - min(cost[i], ORDER_BUCKETS - 1u)], 1u)] = (uint32_t)i;
}

}  // namespace

int check_render_args(const qn_camera *cam, const uint32_t *ranges, const uint32_t *vals, const qn_splat *sp) {
    QN_REQUIRE(cam, "camera is required");
    QN_REQUIRE(cam->width > 0 && cam->height > 0 && cam->width <= QN_TILE * QN_MAX_TILES_X &&
                   cam->height <= QN_TILE * QN_MAX_TILES_Y,
               "image size %dx%d out of range", cam->width, cam->height);
    QN_REQUIRE(ranges && vals && sp, "ranges, vals and splats are required");
    QN_REQUIRE(((uintptr_t)sp & 15) == 0, "splats must be 16-byte aligned");
    return QN_OK;
}

int launch_render_bwd(const qn_camera *cam, const uint32_t *ranges, const uint32_t *vals, const qn_splat *splats,
                      const float *bg, const float *T_final, const uint32_t *last, const float *d_img,
                      const uint8_t *skip, const uint8_t *composited, const uint32_t *order,
                      qn_splat *pair_grads, uint32_t *visited, uint8_t *hit, cudaStream_t stream) {
    int st = check_render_args(cam, ranges, vals, splats);
    if (st) return st;
    QN_REQUIRE(T_final && last && d_img && bg && pair_grads, "null pointer argument");
    QN_REQUIRE(((uintptr_t)pair_grads & 15) == 0, "pair records must be 16-byte aligned");
    const int TX = (cam->width + QN_TILE - 1) / QN_TILE, TY = (cam->height + QN_TILE - 1) / QN_TILE;
    constexpr int PPT = QN_BWD_PPT;
    k_render_bwd<PPT><<<TX * TY, Band<PPT>::THREADS, 0, stream>>>(
        cam->width, cam->height, TX, ranges, vals, reinterpret_cast<const float4 *>(splats), bg[0], bg[1], bg[2],
        T_final, last, d_img, skip, composited, reinterpret_cast<float4 *>(pair_grads), visited, hit, order);
    return check_launch("qn_render_bwd");
}

}  // namespace qn

namespace qn {
namespace {
template <bool LAZY>
int launch_render_fwd(const qn_camera *cam_host, const uint32_t *ranges, const uint32_t *vals, const BinView &bins,
                      uint32_t *vals_out, const qn_splat *splats, const float *bg_host, float *img, float *T_final,
                      uint32_t *last, uint32_t *n_contrib, uint8_t *composited, const uint32_t *tile_order,
                      uint32_t *tile_cost, qn_stream_t stream) {
    const int TX = (cam_host->width + QN_TILE - 1) / QN_TILE, TY = (cam_host->height + QN_TILE - 1) / QN_TILE;
    constexpr int PPT = QN_FWD_PPT;
    auto kern = n_contrib ? (composited ? k_render_fwd<true, true, PPT, LAZY> : k_render_fwd<true, false, PPT, LAZY>)
                          : (composited ? k_render_fwd<false, true, PPT, LAZY> : k_render_fwd<false, false, PPT, LAZY>);
    kern<<<TX * TY, Band<PPT>::THREADS, 0, as_stream(stream)>>>(
        cam_host->width, cam_host->height, TX, TY, ranges, vals, bins, vals_out,
        reinterpret_cast<const float4 *>(splats), bg_host[0], bg_host[1], bg_host[2], img, T_final, last, n_contrib,
        composited, tile_order, tile_cost);
    return check_launch(LAZY ? "qn_render_fwd_binned" : "qn_render_fwd");
}
}  // namespace
}  // namespace qn

extern "C" int qn_render_fwd(const qn_camera *cam_host, const uint32_t *ranges, const uint32_t *vals,
                             const qn_splat *splats, const float *bg_host, float *img, float *T_final,
                             uint32_t *last, uint32_t *n_contrib, uint8_t *composited, const uint32_t *tile_order,
                             uint32_t *tile_cost, qn_stream_t stream) {
    int st = qn::check_render_args(cam_host, ranges, vals, splats);
    if (st) return st;
    QN_REQUIRE(img && T_final && last && bg_host, "null pointer argument");
    return qn::launch_render_fwd<false>(cam_host, ranges, vals,
                                        qn::BinView{nullptr, nullptr, nullptr, nullptr, nullptr, 0, nullptr, nullptr},
                                        nullptr,
                                        splats, bg_host, img, T_final, last, n_contrib, composited, tile_order,
                                        tile_cost, stream);
}

extern "C" int qn_render_fwd_binned(const qn_camera *cam_host, int32_t n, void *workspace,
                                    size_t workspace_bytes, const uint32_t *ranges, uint32_t *vals,
                                    const qn_splat *splats, const float *bg_host, float *img, float *T_final,
                                    uint32_t *last, uint32_t *n_contrib, uint8_t *composited,
                                    const uint32_t *tile_order, uint32_t *tile_cost, qn_stream_t stream) {
    int st = qn::check_render_args(cam_host, ranges, vals, splats);
    if (st) return st;
    QN_REQUIRE(img && T_final && last && bg_host, "null pointer argument");
    const int TX = (cam_host->width + QN_TILE - 1) / QN_TILE, TY = (cam_host->height + QN_TILE - 1) / QN_TILE;
    qn::BinView bins;
    st = qn::bin_view(n, TX, TY, workspace, workspace_bytes, bins);
    if (st) return st;
    return qn::launch_render_fwd<true>(cam_host, ranges, vals, bins, vals, splats, bg_host, img, T_final, last,
                                       n_contrib, composited, tile_order, tile_cost, stream);
}

extern "C" int qn_tile_order(int32_t n_tiles, const uint32_t *tile_cost, uint32_t *tile_order, qn_stream_t stream) {
    QN_REQUIRE(n_tiles >= 0 && n_tiles <= QN_MAX_TILES_X * QN_MAX_TILES_Y, "n_tiles out of range");
    QN_REQUIRE(n_tiles == 0 || (tile_cost && tile_order), "null pointer argument");
    if (n_tiles == 0) return QN_OK;
    qn::k_tile_order<<<1, 1024, 0, qn::as_stream(stream)>>>(n_tiles, tile_cost, tile_order);
    return qn::check_launch("qn_tile_order");
}
