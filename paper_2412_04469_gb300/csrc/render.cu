// Front-to-back alpha compositing per 16 x 16 tile (Sec. 3.1, Eq. 2) and its
// adjoint.  One block per tile, one thread per pixel; Gaussian records are
// staged in shared memory in batches and read back as broadcasts.
#include "common.cuh"

namespace qn {
namespace {

constexpr int BLOCK = QN_TILE * QN_TILE;
constexpr int FWD_BATCH = BLOCK;
constexpr int BWD_BATCH = 32;
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

__global__ void __launch_bounds__(BLOCK) k_render_fwd(int W, int H, int TX, const uint32_t *__restrict__ ranges,
                                                      const uint32_t *__restrict__ vals,
                                                      const float4 *__restrict__ sp, float bg0, float bg1,
                                                      float bg2, float *__restrict__ img,
                                                      float *__restrict__ Tf, uint32_t *__restrict__ last,
                                                      uint32_t *__restrict__ ncon) {
    __shared__ float4 s0[FWD_BATCH], s1[FWD_BATCH], s2[FWD_BATCH];
    const int tile = blockIdx.x;
    const int px = (tile % TX) * QN_TILE + (threadIdx.x % QN_TILE);
    const int py = (tile / TX) * QN_TILE + (threadIdx.x / QN_TILE);
    const bool inside = px < W && py < H;
    const uint32_t beg = ranges[2 * tile], end = ranges[2 * tile + 1];
    const int n = (int)(end - beg);
    const float fx = px + 0.5f, fy = py + 0.5f;
    float T = 1.f, c0 = 0.f, c1 = 0.f, c2 = 0.f;
    uint32_t lastc = 0, nc = 0;
    bool done = !inside;
    for (int b0 = 0; b0 < n; b0 += FWD_BATCH) {
        if (__syncthreads_count(done) == BLOCK) break;
        const int k = b0 + threadIdx.x;
        if (k < n) {
            const size_t id = vals[beg + k];
            s0[threadIdx.x] = sp[3 * id];
            s1[threadIdx.x] = sp[3 * id + 1];
            s2[threadIdx.x] = sp[3 * id + 2];
        }
        __syncthreads();
        const int cnt = min(FWD_BATCH, n - b0);
        for (int j = 0; j < cnt && !done; ++j) {
            PixelAlpha p;
            if (!pixel_alpha(s0[j], s1[j], fx, fy, p)) continue;
            const float Tn = __fmul_rn(T, __fsub_rn(1.f, p.alpha));
            if (Tn < T_MIN) {
                done = true;
                break;
            }
            const float w = p.alpha * T;
            const float4 c = s2[j];
            c0 = fmaf(c.x, w, c0);
            c1 = fmaf(c.y, w, c1);
            c2 = fmaf(c.z, w, c2);
            T = Tn;
            lastc = (uint32_t)(b0 + j + 1);
            ++nc;
        }
    }
    if (inside) {
        const size_t o = (size_t)py * W + px, plane = (size_t)W * H;
        img[o] = fmaf(T, bg0, c0);
        img[plane + o] = fmaf(T, bg1, c1);
        img[2 * plane + o] = fmaf(T, bg2, c2);
        Tf[o] = T;
        last[o] = lastc;
        if (ncon) ncon[o] = nc;
    }
}

__global__ void __launch_bounds__(BLOCK) k_render_bwd(int W, int H, int TX, const uint32_t *__restrict__ ranges,
                                                      const uint32_t *__restrict__ vals,
                                                      const float4 *__restrict__ sp, float bg0, float bg1,
                                                      float bg2, const float *__restrict__ Tf,
                                                      const uint32_t *__restrict__ last,
                                                      const float *__restrict__ dimg,
                                                      const uint8_t *__restrict__ skip,
                                                      float4 *__restrict__ dsp) {
    __shared__ float4 s0[BWD_BATCH], s1[BWD_BATCH], s2[BWD_BATCH];
    __shared__ uint32_t sid[BWD_BATCH];
    __shared__ int sskip[BWD_BATCH];
    __shared__ float sg[BWD_BATCH][9];
    __shared__ uint32_t smax;
    const int tile = blockIdx.x;
    const int px = (tile % TX) * QN_TILE + (threadIdx.x % QN_TILE);
    const int py = (tile / TX) * QN_TILE + (threadIdx.x / QN_TILE);
    const bool inside = px < W && py < H;
    const uint32_t beg = ranges[2 * tile];
    const float fx = px + 0.5f, fy = py + 0.5f;
    float T = 1.f, dc0 = 0.f, dc1 = 0.f, dc2 = 0.f;
    uint32_t lastp = 0;
    if (inside) {
        const size_t o = (size_t)py * W + px, plane = (size_t)W * H;
        T = Tf[o];
        lastp = last[o];
        dc0 = dimg[o];
        dc1 = dimg[plane + o];
        dc2 = dimg[2 * plane + o];
    }
    float B0 = bg0, B1 = bg1, B2 = bg2;     // colour behind the current Gaussian
    if (threadIdx.x == 0) smax = 0;
    for (int k = threadIdx.x; k < BWD_BATCH * 9; k += BLOCK) (&sg[0][0])[k] = 0.f;
    __syncthreads();
    const uint32_t wmax = __reduce_max_sync(FULL, lastp);
    if ((threadIdx.x & 31) == 0) atomicMax(&smax, wmax);
    __syncthreads();
    const int n = (int)smax;
    const int lane = threadIdx.x & 31;
    for (int hi = n; hi > 0; hi -= BWD_BATCH) {
        const int lo = max(0, hi - BWD_BATCH);
        if (threadIdx.x < hi - lo) {
            const uint32_t id = vals[beg + lo + threadIdx.x];
            sid[threadIdx.x] = id;
            sskip[threadIdx.x] = skip ? (int)skip[id] : 0;
            s0[threadIdx.x] = sp[3 * (size_t)id];
            s1[threadIdx.x] = sp[3 * (size_t)id + 1];
            s2[threadIdx.x] = sp[3 * (size_t)id + 2];
        }
        __syncthreads();
        for (int j = hi - lo - 1; j >= 0; --j) {
            PixelAlpha p;
            const bool hit = inside && (uint32_t)(lo + j) < lastp && pixel_alpha(s0[j], s1[j], fx, fy, p);
            float g[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            if (hit) {
                T = T / (1.f - p.alpha);                       // transmittance in front of j
                const float4 c = s2[j];
                const float w = p.alpha * T;
                g[6] = w * dc0;
                g[7] = w * dc1;
                g[8] = w * dc2;
                const float da = T * (dc0 * (c.x - B0) + dc1 * (c.y - B1) + dc2 * (c.z - B2));
                B0 = fmaf(p.alpha, c.x - B0, B0);
                B1 = fmaf(p.alpha, c.y - B1, B1);
                B2 = fmaf(p.alpha, c.z - B2, B2);
                if (!p.capped) {
                    const float4 cn = s1[j];
                    g[2] = da * p.G;                               // d opacity
                    const float dpow = da * p.alpha;
                    g[0] = dpow * (cn.x * p.dx + cn.y * p.dy);     // d mean x
                    g[1] = dpow * (cn.y * p.dx + cn.z * p.dy);     // d mean y
                    g[3] = -0.5f * dpow * p.dx * p.dx;             // d conic a
                    g[4] = -dpow * p.dx * p.dy;                    // d conic b
                    g[5] = -0.5f * dpow * p.dy * p.dy;             // d conic c
                }
            }
            if (sskip[j] || !__any_sync(FULL, hit)) continue;
#pragma unroll
            for (int q = 0; q < 9; ++q) g[q] = warp_sum(g[q]);
            if (lane == 0)
#pragma unroll
                for (int q = 0; q < 9; ++q) atomicAdd(&sg[j][q], g[q]);
        }
        __syncthreads();
        if (threadIdx.x < hi - lo && !sskip[threadIdx.x]) {
            const float *v = sg[threadIdx.x];
            float4 *d = dsp + 3 * (size_t)sid[threadIdx.x];
            atomicAdd(d, make_float4(v[0], v[1], v[2], 0.f));
            atomicAdd(d + 1, make_float4(v[3], v[4], v[5], 0.f));
            atomicAdd(d + 2, make_float4(v[6], v[7], v[8], 0.f));
        }
        __syncthreads();
        for (int k = threadIdx.x; k < BWD_BATCH * 9; k += BLOCK) (&sg[0][0])[k] = 0.f;
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
    qn::k_render_fwd<<<TX * TY, qn::BLOCK, 0, qn::as_stream(stream)>>>(
        cam_host->width, cam_host->height, TX, ranges, vals, reinterpret_cast<const float4 *>(splats), bg_host[0],
        bg_host[1], bg_host[2], img, T_final, last, n_contrib);
    return qn::check_launch("qn_render_fwd");
}

extern "C" int qn_render_bwd(const qn_camera *cam_host, const uint32_t *ranges, const uint32_t *vals,
                             const qn_splat *splats, int32_t n, const float *bg_host, const float *T_final,
                             const uint32_t *last, const float *d_img, const uint8_t *skip,
                             qn_splat *d_splats, qn_stream_t stream) {
    int st = qn::check_render_args(cam_host, ranges, splats);
    if (st) return st;
    QN_REQUIRE(n >= 0, "n must be >= 0");
    QN_REQUIRE(T_final && last && d_img && bg_host && (n == 0 || d_splats), "null pointer argument");
    QN_REQUIRE(((uintptr_t)d_splats & 15) == 0, "d_splats must be 16-byte aligned");
    cudaStream_t s = qn::as_stream(stream);
    if (n > 0 && cudaMemsetAsync(d_splats, 0, sizeof(qn_splat) * (size_t)n, s) != cudaSuccess)
        return qn::check_launch("qn_render_bwd memset");
    const int TX = (cam_host->width + QN_TILE - 1) / QN_TILE, TY = (cam_host->height + QN_TILE - 1) / QN_TILE;
    qn::k_render_bwd<<<TX * TY, qn::BLOCK, 0, s>>>(cam_host->width, cam_host->height, TX, ranges, vals,
                                                    reinterpret_cast<const float4 *>(splats), bg_host[0],
                                                    bg_host[1], bg_host[2], T_final, last, d_img, skip,
                                                    reinterpret_cast<float4 *>(d_splats));
    return qn::check_launch("qn_render_bwd");
}
