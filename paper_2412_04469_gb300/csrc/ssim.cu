// D-SSIM term of Eq. 3 (Sec. 3.1) and its gradient.
//
// SSIM of every channel and pixel from the local means, variances and
// covariance of the rendering x and the target y under an 11 x 11 Gaussian
// window (sigma 1.5, taps outside the image read zero), C1 = 0.01^2,
// C2 = 0.03^2; D-SSIM = 1 - the mean of SSIM.  Two tiled kernels over blocks
// of 32 columns x 64 rows (8 warps, 8 output rows each):
//
//   k_ssim_fwd  stages x and y of the block plus a 5-pixel halo in shared
//               memory (a warp per row, a lane per column), sums every halo
//               row along x (five window sums: x, y, x^2, y^2, xy), then each
//               warp runs down its 18 staged rows once, adding each into the
//               register accumulators of the up to 8 output rows whose
//               window covers it; evaluates SSIM and writes its three partial
//               derivatives (w.r.t. the window sums of x, x^2, xy, times
//               dL/dSSIM) and a per-block SSIM sum;
//   k_ssim_bwd  filters those three maps the same way (the window is
//               symmetric, so the transpose of the zero-padded filter is the
//               filter itself over maps that are zero outside the image) and
//               adds F(a) + 2 x F(b) + y F(c) to d_img; its first block then
//               adds w (1 - mean SSIM) to the loss from the forward's
//               per-block sums (all written: the forward has completed), in
//               a fixed order, so the value is reproducible.
//
// With a pixel mask (Sec. 3.3's masked training) the mean runs over the
// masked pixels only.
//
// FP32 conditioning: variance and covariance as E[x^2] - mu^2 cancel badly
// where the window is nearly flat, and so do the three terms of the
// gradient.  Both kernels therefore work on u = x - k, v = y - k with k = 1/2
// inside the image (zero outside, as the filter's padding is for x):
//   mu_x = E[u] + k s,  s_x^2 = E[u^2] - E[u]^2 + (1 - s)(2 k E[u] + k^2 s),
//   s_xy = E[uv] - E[u]E[v] + (1 - s) k (E[u] + E[v] + k s),
// s = the window's mass inside the image (1 away from the border), and the
// gradient F(a) + 2x F(b) + y F(c) = F(a + k (2b + c)) + 2u F(b) + v F(c).
// Both are exact rewrites; on smooth images they cut the FP32 error of the
// gradient about tenfold.
#include <cmath>
#include <mutex>

#include "common.cuh"
#include "packed.cuh"

namespace qn {
namespace {

constexpr int SS_R = 5, SS_K = 2 * SS_R + 1;
constexpr int SS_TW = 32, SS_WARPS = 8, SS_RPW = 8, SS_TR = SS_WARPS * SS_RPW;   // 32 x 64 outputs
constexpr int SS_HW = SS_TW + 2 * SS_R, SS_HR = SS_TR + 2 * SS_R;                 // staged 42 x 74
constexpr int SS_THREADS = 32 * SS_WARPS;
constexpr int SS_ROWS_PER_WARP = (SS_HR + SS_WARPS - 1) / SS_WARPS;               // staged rows a warp loads
constexpr float SS_C1 = 0.01f * 0.01f, SS_C2 = 0.03f * 0.03f;
constexpr float SS_SHIFT = 0.5f;

// shared memory: np staged planes [HR][HW] then nq row sums [HR][TW]; the
// first two staged planes are interleaved into one plane of pairs, and so are
// the row sums two by two, so that the passes run on packed f32x2 arithmetic
constexpr size_t ss_smem(int np, int nq) {
    return sizeof(float) * ((size_t)np * SS_HR * SS_HW + (size_t)nq * SS_HR * SS_TW);
}
constexpr size_t SS_FWD_SMEM = ss_smem(2, 5), SS_BWD_SMEM = ss_smem(3, 3);

struct Window {
    float g[SS_K];          // normalised 1-D Gaussian, sigma 1.5
    float cum[SS_K + 1];    // cum[j] = g[0] + ... + g[j-1] (the window is symmetric)
};

// Plane p of the block plus its halo, shifted: planes[p][y0 - R + r][x0 - R + c]
// - shift (zero outside the image) at row r, column c -- planes 0 and 1
// interleaved as pairs in s2 [HR][HW], a third plane in s1 [HR][HW].  Warp w
// stages rows w, w + 8, ...; lane l columns l and 32 + l (< 42).  All loads
// of a thread are issued before its first store.
template <int NP>
__device__ __forceinline__ void stage_rows(const float *const (&planes)[NP], int W, int H, int x0, int y0,
                                           float shift, f2 *s2, float *s1) {
    static_assert(NP == 2 || NP == 3, "two planes paired, and a third");
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int xa = x0 - SS_R + lane, xb = xa + 32;
    const bool ina = xa >= 0 && xa < W, inb = lane < 2 * SS_R && xb < W;
    float a[NP][SS_ROWS_PER_WARP], b[NP][SS_ROWS_PER_WARP];
#pragma unroll
    for (int k = 0; k < SS_ROWS_PER_WARP; ++k) {
        const int r = warp + k * SS_WARPS, y = y0 - SS_R + r;
        const bool row = r < SS_HR && y >= 0 && y < H;
        const size_t base = row ? (size_t)y * W : 0;
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            a[p][k] = row && ina ? __ldg(planes[p] + base + xa) - shift : 0.f;
            b[p][k] = row && inb ? __ldg(planes[p] + base + xb) - shift : 0.f;
        }
    }
#pragma unroll
    for (int k = 0; k < SS_ROWS_PER_WARP; ++k) {
        const int r = warp + k * SS_WARPS;
        if (r >= SS_HR) break;
        f2 *row2 = s2 + (size_t)r * SS_HW;
        row2[lane] = pk(a[0][k], a[1][k]);
        if (lane < 2 * SS_R) row2[32 + lane] = pk(b[0][k], b[1][k]);
        if (NP == 3) {
            float *row1 = s1 + (size_t)r * SS_HW;
            row1[lane] = a[NP - 1][k];
            if (lane < 2 * SS_R) row1[32 + lane] = b[NP - 1][k];
        }
    }
}

// The window's mass over taps inside [0, n) around position p (1 away from
// the border): the sum of the taps that fall off either end, subtracted.
__device__ __forceinline__ float mass_1d(const Window &win, int p, int n) {
    const int lo = SS_R - p, hi = p + SS_R - (n - 1);       // taps off the low / high end
    float m = 1.f;
#pragma unroll
    for (int j = 1; j <= SS_R; ++j) {
        if (lo == j) m -= win.cum[j];
        if (hi == j) m -= win.cum[j];
    }
    return m;
}

__device__ __forceinline__ int mask_count(const int *n_masked, int W, int H) {
    return n_masked ? *n_masked : W * H;
}

// The vertical pass of warp w: staged row-sum rows 8w .. 8w + 17, each read
// once and added into the accumulators of the output rows o (0..7) whose
// window covers it (tap t - o): NP planes of pairs hp [NP][HR][TW] and one
// plane h1 [HR][TW].
template <int NP>
__device__ __forceinline__ void column_pass(const Window &win, const f2 *hp, const float *h1,
                                            f2 (&accp)[SS_RPW][NP], float (&acc1)[SS_RPW]) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 0; o < SS_RPW; ++o) {
#pragma unroll
        for (int q = 0; q < NP; ++q) accp[o][q] = pk(0.f, 0.f);
        acc1[o] = 0.f;
    }
#pragma unroll
    for (int t = 0; t < SS_RPW + 2 * SS_R; ++t) {
        const size_t at = (size_t)(SS_RPW * warp + t) * SS_TW + lane;
        f2 h[NP];
#pragma unroll
        for (int q = 0; q < NP; ++q) h[q] = hp[(size_t)q * SS_HR * SS_TW + at];
        const float hs = h1[at];
#pragma unroll
        for (int o = 0; o < SS_RPW; ++o) {
            const int i = t - o;
            if (i >= 0 && i < SS_K) {
                const f2 g = pk(win.g[i], win.g[i]);
#pragma unroll
                for (int q = 0; q < NP; ++q) accp[o][q] = fma2(g, h[q], accp[o][q]);
                acc1[o] = fmaf(win.g[i], hs, acc1[o]);
            }
        }
    }
}

struct SsimOut {
    float S, da, db, dc;
};

// SSIM at one pixel from the window sums of the shifted u, v (E[u], E[v],
// E[u^2], E[v^2], E[uv]) and the window's mass s inside the image; da, db, dc
// = scale x dSSIM/d(E[x], E[x^2], E[xy]) with da already carrying the shift.
__device__ __forceinline__ SsimOut ssim_pixel(const float (&m)[5], float s, float scale) {
    const float k = SS_SHIFT, o = 1.f - s;
    const float eu = m[0], ev = m[1];
    const float mx = fmaf(k, s, eu), my = fmaf(k, s, ev);
    const float vx = m[2] - eu * eu + o * (2.f * k * eu + k * k * s);
    const float vy = m[3] - ev * ev + o * (2.f * k * ev + k * k * s);
    const float cxy = m[4] - eu * ev + o * k * (eu + ev + k * s);
    const float A1 = 2.f * mx * my + SS_C1, A2 = 2.f * cxy + SS_C2;
    const float B1 = mx * mx + my * my + SS_C1, B2 = vx + vy + SS_C2;
    const float i1 = __frcp_rn(B1), i2 = __frcp_rn(B2), inv = i1 * i2;
    SsimOut r;
    r.S = A1 * A2 * inv;
    // SSIM through the window sums of x: its mean (also inside the variance
    // and covariance), E[x^2] and E[xy]
    const float da = 2.f * my * (A2 - A1) * inv - 2.f * mx * r.S * (i1 - i2);
    r.db = -scale * r.S * i2;
    r.dc = 2.f * scale * A1 * inv;
    r.da = fmaf(k, 2.f * r.db + r.dc, scale * da);       // the adjoint multiplies by u, v instead of x, y
    return r;
}

__global__ void __launch_bounds__(SS_THREADS) k_ssim_fwd(int W, int H, int C, const float *__restrict__ img,
                                                        const float *__restrict__ tgt, Window win, float w,
                                                        const uint8_t *__restrict__ pmask,
                                                        const int *__restrict__ n_masked, float *__restrict__ maps,
                                                        float *__restrict__ partials) {
    extern __shared__ f2 smem2[];
    f2 *suv = smem2;                                      // [HR][HW] (u, v)
    f2 *hp = suv + SS_HR * SS_HW;                         // [2][HR][TW] (E u, E v), (E u^2, E v^2)
    float *h1 = reinterpret_cast<float *>(hp + 2 * SS_HR * SS_TW);   // [HR][TW] E uv
    __shared__ float red[SS_WARPS];
    const int c = blockIdx.z;
    const size_t plane = (size_t)W * H;
    const int x0 = blockIdx.x * SS_TW, y0 = blockIdx.y * SS_TR;
    {
        const float *const planes[2] = {img + c * plane, tgt + c * plane};
        stage_rows<2>(planes, W, H, x0, y0, SS_SHIFT, suv, nullptr);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int r = warp; r < SS_HR; r += SS_WARPS) {
        const f2 *uv = suv + r * SS_HW + lane;
        f2 ab = pk(0.f, 0.f), sq = pk(0.f, 0.f);
        float xy = 0.f;
#pragma unroll
        for (int j = 0; j < SS_K; ++j) {
            const f2 q = uv[j], guv = mul2(pk(win.g[j], win.g[j]), q);   // (g u, g v)
            ab = add2(ab, guv);
            sq = fma2(guv, q, sq);
            float gu, gv, uj, vj;
            upk(guv, gu, gv);
            upk(q, uj, vj);
            xy = fmaf(gu, vj, xy);
        }
        const size_t at = (size_t)r * SS_TW + lane;
        hp[at] = ab;
        hp[SS_HR * SS_TW + at] = sq;
        h1[at] = xy;
    }
    __syncthreads();
    f2 accp[SS_RPW][2];
    float acc1[SS_RPW];
    column_pass<2>(win, hp, h1, accp, acc1);
    const int cnt = mask_count(n_masked, W, H);
    const float scale = cnt > 0 ? -w / ((float)C * (float)cnt) : 0.f;       // dL/dSSIM
    const int x = x0 + lane;
    const float sx = mass_1d(win, x, W);
    float ssum = 0.f;
    if (x < W) {
#pragma unroll
        for (int o = 0; o < SS_RPW; ++o) {
            const int y = y0 + SS_RPW * warp + o;
            if (y >= H) break;
            const size_t p = (size_t)y * W + x;
            SsimOut out = {0.f, 0.f, 0.f, 0.f};
            if (!pmask || pmask[p]) {
                float m[5];
                upk(accp[o][0], m[0], m[1]);
                upk(accp[o][1], m[2], m[3]);
                m[4] = acc1[o];
                out = ssim_pixel(m, sx * mass_1d(win, y, H), scale);
                ssum += out.S;
            }
            maps[(0 * (size_t)C + c) * plane + p] = out.da;
            maps[(1 * (size_t)C + c) * plane + p] = out.db;
            maps[(2 * (size_t)C + c) * plane + p] = out.dc;
        }
    }
    ssum = warp_sum(ssum);
    if (lane == 0) red[warp] = ssum;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
#pragma unroll
        for (int i = 0; i < SS_WARPS; ++i) t += red[i];
        partials[((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = t;
    }
}

// loss[0] += w (1 - sum / (C count)) over the forward's per-block sums:
// thread t adds blocks t, t + 256, ... in FP64, then fixed shuffle and
// shared-memory trees.
__device__ __forceinline__ void finish_loss(int blocks, int W, int H, int C, const float *__restrict__ partials,
                                            const int *__restrict__ n_masked, float w, float *__restrict__ loss) {
    __shared__ double red[SS_WARPS];
    double s = 0.0;
    for (int b = threadIdx.x; b < blocks; b += SS_THREADS) s += (double)partials[b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
#pragma unroll
        for (int i = 0; i < SS_WARPS; ++i) t += red[i];
        const int cnt = mask_count(n_masked, W, H);
        if (cnt > 0) loss[0] += (float)((double)w * (1.0 - t / ((double)C * (double)cnt)));
    }
}

__global__ void __launch_bounds__(SS_THREADS) k_ssim_bwd(int W, int H, int C, const float *__restrict__ img,
                                                        const float *__restrict__ tgt, Window win,
                                                        const float *__restrict__ maps, float *__restrict__ d_img,
                                                        int blocks, const float *__restrict__ partials,
                                                        const int *__restrict__ n_masked, float w,
                                                        float *__restrict__ loss) {
    extern __shared__ f2 smem2[];
    f2 *s01 = smem2;                                      // [HR][HW] maps 0 and 1
    float *s2 = reinterpret_cast<float *>(s01 + SS_HR * SS_HW);      // [HR][HW] map 2
    f2 *hp = reinterpret_cast<f2 *>(s2 + SS_HR * SS_HW);             // [HR][TW] row sums of maps 0, 1
    float *h1 = reinterpret_cast<float *>(hp + SS_HR * SS_TW);       // [HR][TW] row sums of map 2
    const int c = blockIdx.z;
    const size_t plane = (size_t)W * H;
    const int x0 = blockIdx.x * SS_TW, y0 = blockIdx.y * SS_TR;
    {
        const float *const planes[3] = {maps + c * plane, maps + (C + (size_t)c) * plane,
                                        maps + (2 * (size_t)C + c) * plane};
        stage_rows<3>(planes, W, H, x0, y0, 0.f, s01, s2);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int r = warp; r < SS_HR; r += SS_WARPS) {
        f2 a01 = pk(0.f, 0.f);
        float a2 = 0.f;
        const f2 *row01 = s01 + (size_t)r * SS_HW + lane;
        const float *row2 = s2 + (size_t)r * SS_HW + lane;
#pragma unroll
        for (int j = 0; j < SS_K; ++j) {
            a01 = fma2(pk(win.g[j], win.g[j]), row01[j], a01);
            a2 = fmaf(win.g[j], row2[j], a2);
        }
        const size_t at = (size_t)r * SS_TW + lane;
        hp[at] = a01;
        h1[at] = a2;
    }
    __syncthreads();
    // this thread's outputs: x, y and d_img loaded now, used after the column pass
    const int x = x0 + lane, yb = y0 + SS_RPW * warp;
    float px[SS_RPW], py[SS_RPW], pd[SS_RPW];
#pragma unroll
    for (int o = 0; o < SS_RPW; ++o) {
        const bool in = x < W && yb + o < H;
        const size_t p = in ? c * plane + (size_t)(yb + o) * W + x : 0;
        px[o] = in ? __ldg(img + p) : 0.f;
        py[o] = in ? __ldg(tgt + p) : 0.f;
        pd[o] = in ? d_img[p] : 0.f;
    }
    f2 fp[SS_RPW][1];
    float f2s[SS_RPW];
    column_pass<1>(win, hp, h1, fp, f2s);
    if (x < W) {
#pragma unroll
        for (int o = 0; o < SS_RPW; ++o) {
            if (yb + o >= H) break;
            const size_t p = c * plane + (size_t)(yb + o) * W + x;
            float fa, fb;
            upk(fp[o][0], fa, fb);
            d_img[p] = pd[o] + fa + 2.f * (px[o] - SS_SHIFT) * fb + (py[o] - SS_SHIFT) * f2s[o];
        }
    }
    if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0) finish_loss(blocks, W, H, C, partials, n_masked, w, loss);
}

Window make_window() {
    Window win;
    double g[SS_K], sum = 0.0;
    for (int i = 0; i < SS_K; ++i) {
        const double r = i - SS_R;
        g[i] = std::exp(-r * r / (2.0 * 1.5 * 1.5));
        sum += g[i];
    }
    double c = 0.0;
    win.cum[0] = 0.f;
    for (int i = 0; i < SS_K; ++i) {
        win.g[i] = (float)(g[i] / sum);
        c += g[i] / sum;
        win.cum[i + 1] = (float)c;
    }
    return win;
}

struct SsimGrid {
    dim3 grid;
    size_t blocks, maps_bytes, partial_bytes;
};

SsimGrid ssim_grid(int W, int H, int C) {
    SsimGrid s;
    s.grid = dim3((unsigned)div_up(W, SS_TW), (unsigned)div_up(H, SS_TR), (unsigned)C);
    s.blocks = (size_t)s.grid.x * s.grid.y * s.grid.z;
    s.maps_bytes = 3 * (size_t)C * W * H * sizeof(float);
    s.maps_bytes = (s.maps_bytes + 255) & ~(size_t)255;
    s.partial_bytes = s.blocks * sizeof(float);
    return s;
}

bool ssim_dims_ok(int W, int H, int C) {
    return W > 0 && H > 0 && C > 0 && C <= 65535 && (int64_t)W * H <= (int64_t)1 << 30 && div_up(H, SS_TR) <= 65535;
}

// The dynamic shared memory of both kernels is above the 48 KB default: set
// once per process (before any graph capture that the first call precedes).
cudaError_t ssim_attributes() {
    static std::once_flag once;
    static cudaError_t err = cudaSuccess;
    std::call_once(once, [] {
        err = cudaFuncSetAttribute(k_ssim_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SS_FWD_SMEM);
        if (err == cudaSuccess)
            err = cudaFuncSetAttribute(k_ssim_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SS_BWD_SMEM);
    });
    return err;
}

}  // namespace
}  // namespace qn

extern "C" size_t qn_dssim_workspace_size(int32_t width, int32_t height, int32_t channels) {
    if (!qn::ssim_dims_ok(width, height, channels)) return 0;
    const qn::SsimGrid g = qn::ssim_grid(width, height, channels);
    return g.maps_bytes + g.partial_bytes;
}

extern "C" int qn_dssim_loss(int32_t width, int32_t height, int32_t channels, const float *img, const float *target,
                             const uint8_t *pixel_mask, const int32_t *n_masked, float w, float *loss, float *d_img,
                             void *workspace, size_t workspace_bytes, qn_stream_t stream) {
    QN_REQUIRE(qn::ssim_dims_ok(width, height, channels), "image size %dx%dx%d out of range", channels, height,
               width);
    QN_REQUIRE(img && target && loss && d_img && workspace, "null pointer argument");
    QN_REQUIRE(!pixel_mask == !n_masked, "pixel_mask and n_masked go together");
    QN_REQUIRE(d_img != img && d_img != target, "d_img may not alias img or target");
    const qn::SsimGrid g = qn::ssim_grid(width, height, channels);
    QN_REQUIRE(workspace_bytes >= g.maps_bytes + g.partial_bytes, "workspace too small (%zu < %zu bytes)",
               workspace_bytes, g.maps_bytes + g.partial_bytes);
    QN_REQUIRE(((uintptr_t)workspace & 15) == 0, "workspace must be 16-byte aligned");
    if (qn::ssim_attributes() != cudaSuccess) return qn::check_launch("qn_dssim_loss attributes");
    cudaStream_t s = qn::as_stream(stream);
    float *maps = static_cast<float *>(workspace);
    float *partials = reinterpret_cast<float *>(static_cast<char *>(workspace) + g.maps_bytes);
    const qn::Window win = qn::make_window();
    qn::k_ssim_fwd<<<g.grid, qn::SS_THREADS, qn::SS_FWD_SMEM, s>>>(width, height, channels, img, target, win, w,
                                                                 pixel_mask, n_masked, maps, partials);
    qn::k_ssim_bwd<<<g.grid, qn::SS_THREADS, qn::SS_BWD_SMEM, s>>>(width, height, channels, img, target, win, maps,
                                                                 d_img, (int)g.blocks, partials, n_masked, w, loss);
    return qn::check_launch("qn_dssim_loss");
}
