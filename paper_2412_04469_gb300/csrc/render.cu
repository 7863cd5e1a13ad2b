// Front-to-back alpha compositing per 16 x 16 tile (Sec. 3.1, Eq. 2) and its
// adjoint.  One warp per tile, eight pixels per lane; Gaussian records are
// staged in shared memory in batches of 32 and read back as broadcasts.
#include "common.cuh"

namespace qn {
namespace {

constexpr float ALPHA_MIN = 1.f / 255.f;
constexpr float ALPHA_MAX = 0.99f;
constexpr float T_MIN = 1e-4f;
constexpr float LOG2E = 1.4426950408889634f;

// A 16 x 16 tile is split into 16 / (2 PPT) horizontal bands of 2 PPT rows,
// one warp per band.  Lane l owns the PPT pixels of column l % 16 in rows
// PPT (l / 16) .. PPT (l / 16) + PPT - 1 of its band, so the horizontal
// offset dx and the dx^2 term of the exponent are shared by all of them, and
// every record read from shared memory and every per-Gaussian reduction
// serves PPT pixels.
template <int PPT>
struct Band {
    static constexpr int WARPS = QN_TILE / (2 * PPT);   // warps per tile
    static constexpr int THREADS = 32 * WARPS;
};
constexpr int FWD_PPT = 2;                      // forward: little work per (lane, Gaussian) besides the pixels
constexpr int BWD_PPT = 2;                      // adjoint: a warp reduction per (warp, Gaussian)
constexpr int BATCH = 32;                       // records staged per round by each forward warp

// Staged record: (mean x, mean y, opacity, -) and the conic scaled for a
// base-2 exponential, log2(e) * power = A dx^2 + B dx dy + C dy^2 with
// A = -a log2(e) / 2, B = -b log2(e), C = -c log2(e) / 2, plus a cull bound:
// alpha >= 1/255 needs o 2^e >= 1/255, i.e. e >= -log2(255 o); a band whose
// pixels all have e below that bound minus a margin (far wider than the
// rounding of ex2 and log2) cannot pass the alpha test anywhere and skips the
// Gaussian, so the cull never changes a result.
constexpr float CULL_MARGIN = 1e-3f;

__device__ __forceinline__ float4 scaled_conic(float4 g1, float opacity) {
    const float bound = opacity > 0.f ? -log2f(255.f * opacity) - CULL_MARGIN : INFINITY;
    return make_float4(__fmul_rn(-0.5f * LOG2E, g1.x), __fmul_rn(-LOG2E, g1.y), __fmul_rn(-0.5f * LOG2E, g1.z),
                       bound);
}

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Per (lane, Gaussian): the dx-only part of the exponent.
struct RowTerms {
    float dx, p0, bdx;
};

__device__ __forceinline__ RowTerms row_terms(const float4 &g0, const float4 &k, float fx) {
    RowTerms r;
    r.dx = __fsub_rn(fx, g0.x);
    r.p0 = __fmul_rn(__fmul_rn(k.x, r.dx), r.dx);
    r.bdx = __fmul_rn(k.y, r.dx);
    return r;
}

struct PixelAlpha {
    float alpha, G, dy;
    bool capped, ok;
};

// log2(e) * power at one pixel of the lane's column; dy = y - mean_y.
__device__ __forceinline__ float pixel_e2(const float4 &g0, const float4 &k, const RowTerms &r, float fy, float &dy) {
    dy = __fsub_rn(fy, g0.y);
    return __fmaf_rn(dy, __fmaf_rn(k.z, dy, r.bdx), r.p0);
}

// alpha = min(0.99, o 2^(log2(e) power)) from the exponent, with explicit
// round-to-nearest operations so that the forward pass and the adjoint
// evaluate bit-identical alphas and take identical skip decisions.
// ok: power <= 0 and alpha >= 1/255.
__device__ __forceinline__ PixelAlpha pixel_alpha(const float4 &g0, float e2, float dy) {
    PixelAlpha p;
    p.dy = dy;
    p.G = ex2_approx(e2);
    const float v = __fmul_rn(g0.z, p.G);
    p.capped = v > ALPHA_MAX;
    p.alpha = fminf(v, ALPHA_MAX);
    p.ok = e2 <= 0.f && p.alpha >= ALPHA_MIN;
    return p;
}

template <int NB>
struct StageBuf {
    float4 g0[NB], k[NB], c[NB];
};

template <int PPT>
__device__ __forceinline__ void pixel_coords(int tile, int TX, int &px, int &py0) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    px = (tile % TX) * QN_TILE + (lane & 15);
    py0 = (tile / TX) * QN_TILE + warp * (2 * PPT) + (lane >> 4) * PPT;
}

// Every warp composites its band independently: it stages its own copy of
// each batch of records and stops when its pixels have all terminated.  The
// per-pixel update is branch-free (selects and zero weights), so the PPT
// pixel chains of a lane interleave.
template <bool COUNT, int PPT = FWD_PPT, int WARPS = Band<PPT>::WARPS>
__global__ void __launch_bounds__(32 * WARPS) k_render_fwd(int W, int H, int TX, const uint32_t *__restrict__ ranges,
                                                        const uint32_t *__restrict__ vals,
                                                        const float4 *__restrict__ sp, float bg0, float bg1,
                                                        float bg2, float *__restrict__ img,
                                                        float *__restrict__ Tf, uint32_t *__restrict__ last,
                                                        uint32_t *__restrict__ ncon) {
    __shared__ StageBuf<BATCH> sbuf[WARPS];
    StageBuf<BATCH> &s = sbuf[threadIdx.x >> 5];
    const int tile = blockIdx.x;
    const int lane = threadIdx.x & 31;
    int px, py0;
    pixel_coords<PPT>(tile, TX, px, py0);
    const uint32_t beg = ranges[2 * tile], end = ranges[2 * tile + 1];
    const int n = (int)(end - beg);
    const float fx = px + 0.5f, fy0 = py0 + 0.5f;
    float T[PPT], c0[PPT], c1[PPT], c2[PPT];
    uint32_t lastc[PPT], nc[PPT];
    uint32_t live = 0;                                  // bit q: pixel q still compositing
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        T[q] = 1.f; c0[q] = c1[q] = c2[q] = 0.f; lastc[q] = nc[q] = 0;
        if (px < W && py0 + q < H) live |= 1u << q;
    }
    for (int b0 = 0; b0 < n; b0 += BATCH) {
        if (!__any_sync(FULL, live)) break;
        if (b0 + lane < n) {
            const size_t id = vals[beg + b0 + lane];
            const float4 g0 = sp[3 * id];
            s.g0[lane] = g0;
            s.k[lane] = scaled_conic(sp[3 * id + 1], g0.z);
            s.c[lane] = sp[3 * id + 2];
        }
        __syncwarp();
        const int cnt = min(BATCH, n - b0);
        for (int j = 0; j < cnt; ++j) {
            if (!__any_sync(FULL, live)) break;
            const float4 g0 = s.g0[j], k = s.k[j], c = s.c[j];
            const RowTerms r = row_terms(g0, k, fx);
            float e2[PPT], dy[PPT];
            bool near = false;
#pragma unroll
            for (int q = 0; q < PPT; ++q) {
                e2[q] = pixel_e2(g0, k, r, fy0 + (float)q, dy[q]);
                near |= e2[q] >= k.w;
            }
            if (!__any_sync(FULL, near)) continue;      // alpha < 1/255 on every pixel of the band
            const uint32_t pos1 = (uint32_t)(b0 + j + 1);
#pragma unroll
            for (int q = 0; q < PPT; ++q) {
                const PixelAlpha p = pixel_alpha(g0, e2[q], dy[q]);
                const bool ok = ((live >> q) & 1u) && p.ok;
                const float Tn = __fmul_rn(T[q], __fsub_rn(1.f, p.alpha));
                const bool stop = Tn < T_MIN;
                const bool add = ok && !stop;
                if (ok && stop) live &= ~(1u << q);
                const float w = add ? p.alpha * T[q] : 0.f;
                c0[q] = fmaf(c.x, w, c0[q]);
                c1[q] = fmaf(c.y, w, c1[q]);
                c2[q] = fmaf(c.z, w, c2[q]);
                T[q] = add ? Tn : T[q];
                lastc[q] = add ? pos1 : lastc[q];
                if (COUNT) nc[q] += add ? 1u : 0u;
            }
        }
        __syncwarp();
    }
    const size_t plane = (size_t)W * H;
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        const int py = py0 + q;
        if (px >= W || py >= H) continue;
        const size_t o = (size_t)py * W + px;
        img[o] = fmaf(T[q], bg0, c0[q]);
        img[plane + o] = fmaf(T[q], bg1, c1[q]);
        img[2 * plane + o] = fmaf(T[q], bg2, c2[q]);
        Tf[o] = T[q];
        last[o] = lastc[q];
        if (COUNT) ncon[o] = nc[q];
    }
}

// Adjoint of k_render_fwd for one tile, walking its list back to front from
// the last contributor of any of its pixels.  Per (lane, Gaussian) the lane
// accumulates, over its pixels, s = dL/dpower and the moments
// sum s dx, sum s dy, sum s dx^2, sum s dx dy, sum s dy^2 (dx shared by the
// column); each warp sums them with a fixed shuffle pattern, the warps'
// sums are added in warp order, and the record of the pair is formed once
// from the conic:
//   dL/dmean = (a Sx + b Sy, b Sx + c Sy),
//   dL/d(a, b, c) = (-Sxx / 2, -Sxy, -Syy / 2),
// since power = -(a dx^2 + c dy^2) / 2 - b dx dy and dx = x - mean_x.
constexpr int PPT = BWD_PPT;
constexpr int WARPS = Band<BWD_PPT>::WARPS;
constexpr int BWD_THREADS = Band<BWD_PPT>::THREADS;
constexpr int BWD_BATCH = BWD_THREADS;          // records staged per round, one per thread

__global__ void __launch_bounds__(BWD_THREADS) k_render_bwd(int W, int H, int TX, const uint32_t *__restrict__ ranges,
                                                        const uint32_t *__restrict__ vals,
                                                        const float4 *__restrict__ sp, float bg0, float bg1,
                                                        float bg2, const float *__restrict__ Tf,
                                                        const uint32_t *__restrict__ last,
                                                        const float *__restrict__ dimg,
                                                        const uint8_t *__restrict__ skip,
                                                        float4 *__restrict__ pair_grads,
                                                        uint32_t *__restrict__ visited,
                                                        uint8_t *__restrict__ ghit) {
    __shared__ StageBuf<BWD_BATCH> s;
    __shared__ float rec[WARPS][BWD_BATCH][9];
    __shared__ int hit[WARPS][BWD_BATCH];
    __shared__ int sskip[BWD_BATCH];
    __shared__ uint32_t wmax[WARPS];
    const int tile = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int px, py0;
    pixel_coords<PPT>(tile, TX, px, py0);
    const uint32_t beg = ranges[2 * tile];
    const float fx = px + 0.5f, fy0 = py0 + 0.5f;
    float T[PPT], dc0[PPT], dc1[PPT], dc2[PPT], B0[PPT], B1[PPT], B2[PPT];
    uint32_t lastp[PPT];
    uint32_t mymax = 0;
    const size_t plane = (size_t)W * H;
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        const int py = py0 + q;
        T[q] = 1.f; dc0[q] = dc1[q] = dc2[q] = 0.f; lastp[q] = 0;
        B0[q] = bg0; B1[q] = bg1; B2[q] = bg2;          // colour behind the current Gaussian
        if (px < W && py < H) {
            const size_t o = (size_t)py * W + px;
            T[q] = Tf[o];
            lastp[q] = last[o];
            dc0[q] = dimg[o];
            dc1[q] = dimg[plane + o];
            dc2[q] = dimg[2 * plane + o];
        }
        mymax = max(mymax, lastp[q]);
    }
    const uint32_t wm = __reduce_max_sync(FULL, mymax);
    if (lane == 0) wmax[warp] = wm;
    __syncthreads();
    uint32_t tmax = 0;
#pragma unroll
    for (int w = 0; w < WARPS; ++w) tmax = max(tmax, wmax[w]);
    const int n = (int)tmax;
    if (threadIdx.x == 0) visited[tile] = tmax;
    for (int hi = n; hi > 0; hi -= BWD_BATCH) {
        const int lo = max(0, hi - BWD_BATCH);
        const int cnt = hi - lo;
        const int t = threadIdx.x;
        float4 conic = make_float4(0.f, 0.f, 0.f, 0.f);   // thread t: raw conic of record lo + t
        bool my_skip = true;
        uint32_t id = 0;
        if (t < cnt) {
            id = vals[beg + lo + t];
            my_skip = skip ? skip[id] != 0 : false;
            const float4 g0 = sp[3 * (size_t)id];
            s.g0[t] = g0;
            conic = sp[3 * (size_t)id + 1];
            s.k[t] = scaled_conic(conic, g0.z);
            s.c[t] = sp[3 * (size_t)id + 2];
            sskip[t] = my_skip;
        }
        __syncthreads();
        for (int j = cnt - 1; j >= 0; --j) {
            const uint32_t pos = (uint32_t)(lo + j);
            if (!__any_sync(FULL, pos < mymax)) {
                if (lane == 0) hit[warp][j] = 0;
                continue;
            }
            const float4 g0 = s.g0[j], k = s.k[j], c = s.c[j];
            const RowTerms r = row_terms(g0, k, fx);
            float e2[PPT], dy[PPT];
            bool near = false;
#pragma unroll
            for (int q = 0; q < PPT; ++q) {
                e2[q] = pixel_e2(g0, k, r, fy0 + (float)q, dy[q]);
                near |= e2[q] >= k.w && pos < lastp[q];
            }
            if (!__any_sync(FULL, near)) {              // no pixel of the band can take j
                if (lane == 0) hit[warp][j] = 0;
                continue;
            }
            float S0 = 0.f, S1 = 0.f, S2 = 0.f, So = 0.f, gc0 = 0.f, gc1 = 0.f, gc2 = 0.f;
            bool any = false;
#pragma unroll
            for (int q = 0; q < PPT; ++q) {
                const PixelAlpha p = pixel_alpha(g0, e2[q], dy[q]);
                const bool valid = pos < lastp[q] && p.ok;
                any |= valid;
                const float Tq = valid ? __fdividef(T[q], 1.f - p.alpha) : T[q];   // in front of j
                T[q] = Tq;
                const float av = valid ? p.alpha : 0.f;
                const float w = av * Tq;
                const float e0 = c.x - B0[q], e1 = c.y - B1[q], e2 = c.z - B2[q];
                const float da = valid ? Tq * (dc0[q] * e0 + dc1[q] * e1 + dc2[q] * e2) : 0.f;
                B0[q] = fmaf(av, e0, B0[q]);
                B1[q] = fmaf(av, e1, B1[q]);
                B2[q] = fmaf(av, e2, B2[q]);
                gc0 = fmaf(w, dc0[q], gc0);
                gc1 = fmaf(w, dc1[q], gc1);
                gc2 = fmaf(w, dc2[q], gc2);
                const float dav = p.capped ? 0.f : da;         // the 0.99 cap passes no gradient
                So = fmaf(dav, p.G, So);                       // d opacity
                const float sdp = dav * p.alpha;               // dL/dpower
                const float tt = sdp * p.dy;
                S0 += sdp;
                S1 += tt;
                S2 = fmaf(tt, p.dy, S2);
            }
            const bool any_j = __any_sync(FULL, any);   // the band composites j (skipped or not)
            if (lane == 0) hit[warp][j] = any_j;
            if (!any_j || sskip[j]) continue;
            const float Sx = r.dx * S0;
            float v[8] = {Sx, S1, r.dx * Sx, r.dx * S1, S2, So, gc0, gc1};
            const float red = reduce_scatter8(v, lane);
            const float red8 = warp_sum(gc2);
            if ((lane & 3) == 0) rec[warp][j][(lane >> 2) & 7] = red;
            if (lane == 0) rec[warp][j][8] = red8;
        }
        __syncthreads();
        // one record per visited list position: the tile's sum for that Gaussian
        if (t < cnt && my_skip && ghit) {
            bool composited = false;
#pragma unroll
            for (int w = 0; w < WARPS; ++w) composited |= hit[w][t] != 0;
            if (composited) ghit[id] = 1;             // a skipped Gaussian some pixel composited
        }
        if (t < cnt && !my_skip) {
            float m[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            bool contributed = false;
#pragma unroll
            for (int w = 0; w < WARPS; ++w) {
                if (!hit[w][t]) continue;
                contributed = true;
#pragma unroll
                for (int q = 0; q < 9; ++q) m[q] += rec[w][t][q];
            }
            if (ghit && contributed) ghit[id] = 1;
            float4 *d = pair_grads + 3 * (size_t)(beg + lo + t);
            d[0] = make_float4(conic.x * m[0] + conic.y * m[1], conic.y * m[0] + conic.z * m[1], m[5], 0.f);
            d[1] = make_float4(-0.5f * m[2], -m[3], -0.5f * m[4], 0.f);
            d[2] = make_float4(m[6], m[7], m[8], 0.f);
        }
        __syncthreads();
    }
}

int check_render_args(const qn_camera *cam, const uint32_t *ranges, const uint32_t *vals, const qn_splat *sp) {
    QN_REQUIRE(cam, "camera is required");
    QN_REQUIRE(cam->width > 0 && cam->height > 0 && cam->width <= QN_TILE * QN_MAX_TILES_X &&
                   cam->height <= QN_TILE * QN_MAX_TILES_Y,
               "image size %dx%d out of range", cam->width, cam->height);
    QN_REQUIRE(ranges && vals && sp, "ranges, vals and splats are required");
    QN_REQUIRE(((uintptr_t)sp & 15) == 0, "splats must be 16-byte aligned");
    return QN_OK;
}

}  // namespace
}  // namespace qn

extern "C" int qn_render_fwd(const qn_camera *cam_host, const uint32_t *ranges, const uint32_t *vals,
                             const qn_splat *splats, const float *bg_host, float *img, float *T_final,
                             uint32_t *last, uint32_t *n_contrib, qn_stream_t stream) {
    int st = qn::check_render_args(cam_host, ranges, vals, splats);
    if (st) return st;
    QN_REQUIRE(img && T_final && last && bg_host, "null pointer argument");
    const int TX = (cam_host->width + QN_TILE - 1) / QN_TILE, TY = (cam_host->height + QN_TILE - 1) / QN_TILE;
    auto kern = n_contrib ? qn::k_render_fwd<true> : qn::k_render_fwd<false>;
    kern<<<TX * TY, qn::Band<qn::FWD_PPT>::THREADS, 0, qn::as_stream(stream)>>>(cam_host->width, cam_host->height, TX, ranges, vals,
                                                   reinterpret_cast<const float4 *>(splats), bg_host[0], bg_host[1],
                                                   bg_host[2], img, T_final, last, n_contrib);
    return qn::check_launch("qn_render_fwd");
}

extern "C" int qn_render_bwd(const qn_camera *cam_host, const uint32_t *ranges, const uint32_t *vals,
                             const qn_splat *splats, const float *bg_host, const float *T_final,
                             const uint32_t *last, const float *d_img, const uint8_t *skip,
                             qn_splat *pair_grads, uint32_t *tile_visited, uint8_t *gauss_hit,
                             qn_stream_t stream) {
    int st = qn::check_render_args(cam_host, ranges, vals, splats);
    if (st) return st;
    QN_REQUIRE(T_final && last && d_img && bg_host && pair_grads && tile_visited, "null pointer argument");
    QN_REQUIRE(((uintptr_t)pair_grads & 15) == 0, "pair_grads must be 16-byte aligned");
    const int TX = (cam_host->width + QN_TILE - 1) / QN_TILE, TY = (cam_host->height + QN_TILE - 1) / QN_TILE;
    qn::k_render_bwd<<<TX * TY, qn::BWD_THREADS, 0, qn::as_stream(stream)>>>(
        cam_host->width, cam_host->height, TX, ranges, vals, reinterpret_cast<const float4 *>(splats), bg_host[0],
        bg_host[1], bg_host[2], T_final, last, d_img, skip, reinterpret_cast<float4 *>(pair_grads), tile_visited,
        gauss_hit);
    return qn::check_launch("qn_render_bwd");
}
