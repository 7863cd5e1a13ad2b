// Adaptive masked training (Sec. 3.3; App. B: t_d = 0.001, 48 x 48 dilation).
// The mask of a view is built once per frame: the dynamic Gaussians
// (|d_t| > t_d) are rendered alone (their tile rects kept, every other rect
// emptied, then the usual binning and compositing), the pixels with a
// contributor are dilated with a k x k box, and the tiles holding a masked
// pixel are marked.  A masked iteration then gives the inactive tiles empty
// ranges (the compositing and its adjoint skip them) and averages the loss
// over the masked pixels only.
#include "common.cuh"

namespace qn {
namespace {

__global__ void k_select_rects(int n, int S, const int4 *__restrict__ in, const float *__restrict__ score, float sx,
                               float sy, float t_d2, int4 *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float dx = score[i] * sx, dy = score[S + i] * sy;
    out[i] = fmaf(dx, dx, dy * dy) > t_d2 ? in[i] : make_int4(0, 0, 0, 0);
}

// Horizontal pass: tmp[y][x] = some last[y][u] > 0 for u in [x - k/2 + 1, x + k/2].
__global__ void k_dilate_rows(int W, int H, int k, const uint32_t *__restrict__ last, uint8_t *__restrict__ tmp) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= W) return;
    const int u0 = max(0, x - k / 2 + 1), u1 = min(W - 1, x + k / 2);
    const uint32_t *row = last + (size_t)y * W;
    uint8_t v = 0;
    for (int u = u0; u <= u1 && !v; ++u) v = row[u] > 0u;
    tmp[(size_t)y * W + x] = v;
}

// Vertical pass over tmp, then the tile marks and the count of masked pixels.
__global__ void k_dilate_cols(int W, int H, int k, const uint8_t *__restrict__ tmp, uint8_t *__restrict__ mask,
                              uint8_t *__restrict__ tiles, int TX, int *__restrict__ count) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    bool v = false;
    if (x < W) {
        const int v0 = max(0, y - k / 2 + 1), v1 = min(H - 1, y + k / 2);
        for (int u = v0; u <= v1 && !v; ++u) v = tmp[(size_t)u * W + x] != 0;
        mask[(size_t)y * W + x] = v;
        if (v) tiles[(y / QN_TILE) * TX + x / QN_TILE] = 1;
    }
    const unsigned b = __ballot_sync(FULL, v);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(count, __popc(b));      // integer: order-independent
}

__global__ void k_mask_ranges(int n_tiles, const uint32_t *__restrict__ in, const uint8_t *__restrict__ tiles,
                              uint32_t *__restrict__ out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_tiles) return;
    const uint32_t b = in[2 * t];
    out[2 * t] = b;
    out[2 * t + 1] = tiles[t] ? in[2 * t + 1] : b;
}

__global__ void __launch_bounds__(256) k_masked_loss(long long hw, int channels, const float *__restrict__ img,
                                                     const float *__restrict__ tgt,
                                                     const uint8_t *__restrict__ mask,
                                                     const int *__restrict__ count, float w, int mse,
                                                     float *__restrict__ partials, float *__restrict__ dimg) {
    __shared__ float red[8];
    const int c = *count;
    const float scale = c > 0 ? w / ((float)channels * (float)c) : 0.f;
    const long long total = hw * channels;
    float acc = 0.f;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const bool on = mask[i % hw] != 0;
        const float d = img[i] - tgt[i];
        float g = 0.f;
        if (on) {
            if (mse) {
                acc = fmaf(d, d, acc);
                g = 2.f * scale * d;
            } else {
                acc += fabsf(d);
                g = d > 0.f ? scale : (d < 0.f ? -scale : 0.f);
            }
        }
        dimg[i] = g;
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int k = 0; k < 8; ++k) s += red[k];
        partials[blockIdx.x] = s * scale;                // summed in block order afterwards
    }
}

}  // namespace
}  // namespace qn

extern "C" int qn_select_rects(int32_t n, int32_t n_stride, const int32_t *rects, const float *score, float ndc_x,
                               float ndc_y, float t_d, int32_t *rects_out, qn_stream_t stream) {
    QN_REQUIRE(n >= 0 && n_stride >= n, "need 0 <= n <= n_stride");
    if (n == 0) return QN_OK;
    QN_REQUIRE(rects && score && rects_out, "null pointer argument");
    QN_REQUIRE(((uintptr_t)rects & 15) == 0 && ((uintptr_t)rects_out & 15) == 0, "rects must be 16-byte aligned");
    QN_REQUIRE(t_d >= 0.f, "t_d must be >= 0");
    qn::k_select_rects<<<qn::div_up(n, 256), 256, 0, qn::as_stream(stream)>>>(
        n, n_stride, reinterpret_cast<const int4 *>(rects), score, ndc_x, ndc_y, t_d * t_d,
        reinterpret_cast<int4 *>(rects_out));
    return qn::check_launch("qn_select_rects");
}

extern "C" int qn_dilate_mask(int32_t width, int32_t height, const uint32_t *last, int32_t k, uint8_t *tmp,
                              uint8_t *pixel_mask, uint8_t *tile_mask, int32_t *n_masked, qn_stream_t stream) {
    QN_REQUIRE(width > 0 && height > 0 && width <= QN_TILE * QN_MAX_TILES_X && height <= QN_TILE * QN_MAX_TILES_Y,
               "image size %dx%d out of range", width, height);
    QN_REQUIRE(k >= 2 && k % 2 == 0, "k must be even and >= 2 (got %d)", k);
    QN_REQUIRE(last && tmp && pixel_mask && tile_mask && n_masked, "null pointer argument");
    cudaStream_t s = qn::as_stream(stream);
    const int TX = (width + QN_TILE - 1) / QN_TILE, TY = (height + QN_TILE - 1) / QN_TILE;
    if (cudaMemsetAsync(tile_mask, 0, (size_t)TX * TY, s) != cudaSuccess ||
        cudaMemsetAsync(n_masked, 0, sizeof(int32_t), s) != cudaSuccess)
        return qn::check_launch("qn_dilate_mask memset");
    const dim3 grid(qn::div_up(width, 128), height);
    qn::k_dilate_rows<<<grid, 128, 0, s>>>(width, height, k, last, tmp);
    qn::k_dilate_cols<<<grid, 128, 0, s>>>(width, height, k, tmp, pixel_mask, tile_mask, TX, n_masked);
    return qn::check_launch("qn_dilate_mask");
}

extern "C" int qn_mask_ranges(int32_t n_tiles, const uint32_t *ranges, const uint8_t *tile_mask,
                              uint32_t *ranges_out, qn_stream_t stream) {
    QN_REQUIRE(n_tiles >= 0, "n_tiles must be >= 0");
    if (n_tiles == 0) return QN_OK;
    QN_REQUIRE(ranges && tile_mask && ranges_out, "null pointer argument");
    QN_REQUIRE(ranges != ranges_out, "ranges_out may not alias ranges");
    qn::k_mask_ranges<<<qn::div_up(n_tiles, 256), 256, 0, qn::as_stream(stream)>>>(n_tiles, ranges, tile_mask,
                                                                                   ranges_out);
    return qn::check_launch("qn_mask_ranges");
}

extern "C" int qn_masked_image_loss(int64_t hw, int32_t channels, const float *img, const float *target,
                                    const uint8_t *pixel_mask, const int32_t *n_masked, float w, int32_t mse,
                                    float *loss, float *d_img, float *partials, qn_stream_t stream) {
    QN_REQUIRE(hw >= 0 && channels >= 1, "bad hw / channels");
    QN_REQUIRE(loss, "loss is required");
    cudaStream_t s = qn::as_stream(stream);
    if (hw == 0) {
        if (cudaMemsetAsync(loss, 0, sizeof(float), s) != cudaSuccess) return qn::check_launch("masked loss memset");
        return QN_OK;
    }
    QN_REQUIRE(img && target && pixel_mask && n_masked && d_img && partials, "null pointer argument");
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long need = (hw * channels + 255) / 256;
    int grid = (int)(need < (long long)sms * 8 ? need : (long long)sms * 8);
    if (grid > QN_LOSS_BLOCKS) grid = QN_LOSS_BLOCKS;
    grid = grid < 1 ? 1 : grid;
    qn::k_masked_loss<<<grid, 256, 0, s>>>(hw, channels, img, target, pixel_mask, n_masked, w, mse, partials, d_img);
    qn::k_sum_partials<<<1, 32, 0, s>>>(1, grid, partials, loss);
    return qn::check_launch("qn_masked_image_loss");
}
