// Front-to-back alpha compositing per 16 x 16 tile (Sec. 3.1, Eq. 2) and its
// adjoint.  One block per tile, four pixels per thread; Gaussian records are
// staged in shared memory in batches and read back as broadcasts.
#include "common.cuh"

namespace qn {
namespace {

constexpr int BLOCK = QN_TILE * QN_TILE;
constexpr int FWD_BATCH = BLOCK;
constexpr float ALPHA_MIN = 1.f / 255.f;
constexpr float ALPHA_MAX = 0.99f;
constexpr float T_MIN = 1e-4f;

struct PixelAlpha {
    float alpha, G, dx, dy;
    bool capped;
};

// alpha = min(0.99, o exp(power)), power = -0.5 (a dx^2 + c dy^2) - b dx dy.
// Written with explicit round-to-nearest intrinsics so the forward and the
// adjoint evaluate bit-identical alphas and take identical skip decisions.
__device__ __forceinline__ bool pixel_alpha(const float4 &g0, const float4 &g1, float fx, float fy,
                                            PixelAlpha &p) {
    p.dx = __fsub_rn(fx, g0.x);
    p.dy = __fsub_rn(fy, g0.y);
    const float q = __fmaf_rn(g1.x, __fmul_rn(p.dx, p.dx), __fmul_rn(g1.z, __fmul_rn(p.dy, p.dy)));
    const float power = __fmaf_rn(-0.5f, q, -__fmul_rn(g1.y, __fmul_rn(p.dx, p.dy)));
    if (power > 0.f) return false;
    p.G = __expf(power);
    const float v = __fmul_rn(g0.z, p.G);
    p.capped = v > ALPHA_MAX;
    p.alpha = p.capped ? ALPHA_MAX : v;
    return p.alpha >= ALPHA_MIN;
}

// Each thread owns PPT vertically adjacent pixels of the tile, so every
// record read from shared memory and every per-Gaussian reduction serves
// PPT pixels.
constexpr int PPT = 4;
constexpr int THREADS = BLOCK / PPT;            // 64 threads per tile
constexpr int FWD_LOAD = FWD_BATCH / THREADS;   // records each thread stages per batch

__global__ void __launch_bounds__(THREADS) k_render_fwd(int W, int H, int TX, const uint32_t *__restrict__ ranges,
                                                        const uint32_t *__restrict__ vals,
                                                        const float4 *__restrict__ sp, float bg0, float bg1,
                                                        float bg2, float *__restrict__ img,
                                                        float *__restrict__ Tf, uint32_t *__restrict__ last,
                                                        uint32_t *__restrict__ ncon) {
    __shared__ float4 s0[FWD_BATCH], s1[FWD_BATCH], s2[FWD_BATCH];
    const int tile = blockIdx.x;
    const int px = (tile % TX) * QN_TILE + (threadIdx.x % QN_TILE);
    const int py0 = (tile / TX) * QN_TILE + (threadIdx.x / QN_TILE) * PPT;
    const uint32_t beg = ranges[2 * tile], end = ranges[2 * tile + 1];
    const int n = (int)(end - beg);
    const float fx = px + 0.5f;
    float T[PPT], c0[PPT], c1[PPT], c2[PPT];
    uint32_t lastc[PPT], nc[PPT];
    bool live[PPT];
    int nlive = 0;
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        T[q] = 1.f; c0[q] = c1[q] = c2[q] = 0.f; lastc[q] = nc[q] = 0;
        live[q] = px < W && py0 + q < H;
        nlive += live[q];
    }
    for (int b0 = 0; b0 < n; b0 += FWD_BATCH) {
        if (__syncthreads_count(nlive == 0) == THREADS) break;
#pragma unroll
        for (int r = 0; r < FWD_LOAD; ++r) {
            const int slot = r * THREADS + threadIdx.x;
            if (b0 + slot < n) {
                const size_t id = vals[beg + b0 + slot];
                s0[slot] = sp[3 * id];
                s1[slot] = sp[3 * id + 1];
                s2[slot] = sp[3 * id + 2];
            }
        }
        __syncthreads();
        const int cnt = min(FWD_BATCH, n - b0);
        for (int j = 0; j < cnt && nlive > 0; ++j) {
            const float4 g0 = s0[j], g1 = s1[j];
#pragma unroll
            for (int q = 0; q < PPT; ++q) {
                if (!live[q]) continue;
                PixelAlpha p;
                if (!pixel_alpha(g0, g1, fx, py0 + q + 0.5f, p)) continue;
                const float Tn = __fmul_rn(T[q], __fsub_rn(1.f, p.alpha));
                if (Tn < T_MIN) {
                    live[q] = false;
                    --nlive;
                    continue;
                }
                const float w = p.alpha * T[q];
                const float4 c = s2[j];
                c0[q] = fmaf(c.x, w, c0[q]);
                c1[q] = fmaf(c.y, w, c1[q]);
                c2[q] = fmaf(c.z, w, c2[q]);
                T[q] = Tn;
                lastc[q] = (uint32_t)(b0 + j + 1);
                ++nc[q];
            }
        }
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
        if (ncon) ncon[o] = nc[q];
    }
}

// Sum over the warp of v[0..7] scattered across lanes (lane l ends up with
// the total of value (l >> 2) & 7), and of x in every lane: 14 shuffles
// instead of the 45 of nine independent butterflies.
__device__ __forceinline__ float reduce_scatter8(float v[8], int lane) {
    const bool h4 = lane & 16, h3 = lane & 8, h2 = lane & 4;
    float a[4], b[2];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float send = h4 ? v[i] : v[i + 4];
        const float keep = h4 ? v[i + 4] : v[i];
        a[i] = keep + __shfl_xor_sync(FULL, send, 16);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float send = h3 ? a[i] : a[i + 2];
        const float keep = h3 ? a[i + 2] : a[i];
        b[i] = keep + __shfl_xor_sync(FULL, send, 8);
    }
    float c = (h2 ? b[1] : b[0]) + __shfl_xor_sync(FULL, h2 ? b[0] : b[1], 4);
    c += __shfl_xor_sync(FULL, c, 2);
    c += __shfl_xor_sync(FULL, c, 1);
    return c;
}

__global__ void __launch_bounds__(THREADS) k_render_bwd(int W, int H, int TX, const uint32_t *__restrict__ ranges,
                                                        const uint32_t *__restrict__ vals,
                                                        const float4 *__restrict__ sp, float bg0, float bg1,
                                                        float bg2, const float *__restrict__ Tf,
                                                        const uint32_t *__restrict__ last,
                                                        const float *__restrict__ dimg,
                                                        const uint8_t *__restrict__ skip,
                                                        float4 *__restrict__ pair_grads,
                                                        uint32_t *__restrict__ visited) {
    constexpr int BATCH = THREADS;
    constexpr int WARPS = THREADS / 32;
    __shared__ float4 s0[BATCH], s1[BATCH], s2[BATCH];
    __shared__ int sskip[BATCH];
    __shared__ float sg[WARPS][BATCH][9];       // one slot per warp: summed in a fixed order
    __shared__ uint32_t smax;
    const int tile = blockIdx.x;
    const int px = (tile % TX) * QN_TILE + (threadIdx.x % QN_TILE);
    const int py0 = (tile / TX) * QN_TILE + (threadIdx.x / QN_TILE) * PPT;
    const uint32_t beg = ranges[2 * tile];
    const float fx = px + 0.5f;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
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
    if (threadIdx.x == 0) smax = 0;
    __syncthreads();
    const uint32_t wmax = __reduce_max_sync(FULL, mymax);
    if (lane == 0) atomicMax(&smax, wmax);
    __syncthreads();
    const int n = (int)smax;
    if (threadIdx.x == 0) visited[tile] = (uint32_t)n;
    for (int hi = n; hi > 0; hi -= BATCH) {
        const int lo = max(0, hi - BATCH);
        for (int k = threadIdx.x; k < WARPS * BATCH * 9; k += THREADS) (&sg[0][0][0])[k] = 0.f;
        if (threadIdx.x < hi - lo) {
            const uint32_t id = vals[beg + lo + threadIdx.x];
            sskip[threadIdx.x] = skip ? (int)skip[id] : 0;
            s0[threadIdx.x] = sp[3 * (size_t)id];
            s1[threadIdx.x] = sp[3 * (size_t)id + 1];
            s2[threadIdx.x] = sp[3 * (size_t)id + 2];
        }
        __syncthreads();
        for (int j = hi - lo - 1; j >= 0; --j) {
            const uint32_t pos = (uint32_t)(lo + j);
            if (!__any_sync(FULL, pos < mymax)) continue;
            const float4 g0 = s0[j], g1 = s1[j], c = s2[j];
            const bool sk = sskip[j] != 0;
            float g[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            bool any = false;
#pragma unroll
            for (int q = 0; q < PPT; ++q) {
                PixelAlpha p;
                if (!(pos < lastp[q] && pixel_alpha(g0, g1, fx, py0 + q + 0.5f, p))) continue;
                any = true;
                T[q] = T[q] / (1.f - p.alpha);                 // transmittance in front of j
                const float w = p.alpha * T[q];
                const float da = T[q] * (dc0[q] * (c.x - B0[q]) + dc1[q] * (c.y - B1[q]) + dc2[q] * (c.z - B2[q]));
                B0[q] = fmaf(p.alpha, c.x - B0[q], B0[q]);
                B1[q] = fmaf(p.alpha, c.y - B1[q], B1[q]);
                B2[q] = fmaf(p.alpha, c.z - B2[q], B2[q]);
                if (sk) continue;
                g[6] = fmaf(w, dc0[q], g[6]);
                g[7] = fmaf(w, dc1[q], g[7]);
                g[8] = fmaf(w, dc2[q], g[8]);
                if (!p.capped) {
                    g[2] = fmaf(da, p.G, g[2]);                          // d opacity
                    const float dpow = da * p.alpha;
                    g[0] = fmaf(dpow, g1.x * p.dx + g1.y * p.dy, g[0]);   // d mean x
                    g[1] = fmaf(dpow, g1.y * p.dx + g1.z * p.dy, g[1]);   // d mean y
                    g[3] = fmaf(-0.5f * dpow, p.dx * p.dx, g[3]);         // d conic a
                    g[4] = fmaf(-dpow, p.dx * p.dy, g[4]);                // d conic b
                    g[5] = fmaf(-0.5f * dpow, p.dy * p.dy, g[5]);         // d conic c
                }
            }
            if (sk || !__any_sync(FULL, any)) continue;
            const float v = reduce_scatter8(g, lane);
            const float last_v = warp_sum(g[8]);
            if ((lane & 3) == 0) sg[warp][j][(lane >> 2) & 7] = v;
            if (lane == 0) sg[warp][j][8] = last_v;
        }
        __syncthreads();
        // one record per visited list position: the tile's sum for that Gaussian
        if (threadIdx.x < hi - lo && !sskip[threadIdx.x]) {
            float r[9];
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                float a = 0.f;
#pragma unroll
                for (int w = 0; w < WARPS; ++w) a += sg[w][threadIdx.x][q];
                r[q] = a;
            }
            float4 *d = pair_grads + 3 * (size_t)(beg + lo + threadIdx.x);
            d[0] = make_float4(r[0], r[1], r[2], 0.f);
            d[1] = make_float4(r[3], r[4], r[5], 0.f);
            d[2] = make_float4(r[6], r[7], r[8], 0.f);
        }
        __syncthreads();
    }
}

int check_render_args(const qn_camera *cam, const uint32_t *ranges, const qn_splat *sp) {
    QN_REQUIRE(cam, "camera is required");
    QN_REQUIRE(cam->width > 0 && cam->height > 0 && cam->width <= QN_TILE * QN_MAX_TILES_X &&
                   cam->height <= QN_TILE * QN_MAX_TILES_Y,
               "image size %dx%d out of range", cam->width, cam->height);
    QN_REQUIRE(ranges, "ranges is required");
    QN_REQUIRE(((uintptr_t)sp & 15) == 0, "splats must be 16-byte aligned");
    return QN_OK;
}

}  // namespace
}  // namespace qn

extern "C" int qn_render_fwd(const qn_camera *cam_host, const uint32_t *ranges, const uint32_t *vals,
                             const qn_splat *splats, const float *bg_host, float *img, float *T_final,
                             uint32_t *last, uint32_t *n_contrib, qn_stream_t stream) {
    int st = qn::check_render_args(cam_host, ranges, splats);
    if (st) return st;
    QN_REQUIRE(img && T_final && last && bg_host, "null pointer argument");
    const int TX = (cam_host->width + QN_TILE - 1) / QN_TILE, TY = (cam_host->height + QN_TILE - 1) / QN_TILE;
    qn::k_render_fwd<<<TX * TY, qn::THREADS, 0, qn::as_stream(stream)>>>(
        cam_host->width, cam_host->height, TX, ranges, vals, reinterpret_cast<const float4 *>(splats), bg_host[0],
        bg_host[1], bg_host[2], img, T_final, last, n_contrib);
    return qn::check_launch("qn_render_fwd");
}

extern "C" int qn_render_bwd(const qn_camera *cam_host, const uint32_t *ranges, const uint32_t *vals,
                             const qn_splat *splats, const float *bg_host, const float *T_final,
                             const uint32_t *last, const float *d_img, const uint8_t *skip,
                             qn_splat *pair_grads, uint32_t *tile_visited, qn_stream_t stream) {
    int st = qn::check_render_args(cam_host, ranges, splats);
    if (st) return st;
    QN_REQUIRE(T_final && last && d_img && bg_host && pair_grads && tile_visited, "null pointer argument");
    QN_REQUIRE(((uintptr_t)pair_grads & 15) == 0, "pair_grads must be 16-byte aligned");
    const int TX = (cam_host->width + QN_TILE - 1) / QN_TILE, TY = (cam_host->height + QN_TILE - 1) / QN_TILE;
    qn::k_render_bwd<<<TX * TY, qn::THREADS, 0, qn::as_stream(stream)>>>(
        cam_host->width, cam_host->height, TX, ranges, vals, reinterpret_cast<const float4 *>(splats), bg_host[0],
        bg_host[1], bg_host[2], T_final, last, d_img, skip, reinterpret_cast<float4 *>(pair_grads), tile_visited);
    return qn::check_launch("qn_render_bwd");
}
