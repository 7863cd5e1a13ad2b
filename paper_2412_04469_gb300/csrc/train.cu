// Loss (Eq. 3 L1 term, and the MSE of Eq. 9) and the Adam update of the
// training iteration (App. B trains every residual parameter with Adam).
#include <cmath>

#include "common.cuh"

namespace qn {
namespace {

__global__ void __launch_bounds__(256) k_image_loss(long long count, const float *__restrict__ img,
                                                    const float *__restrict__ tgt, float scale, int mse,
                                                    float *__restrict__ partials, float *__restrict__ dimg) {
    __shared__ float red[8];
    float acc = 0.f;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        const float d = img[i] - tgt[i];
        if (mse) {
            acc = fmaf(d, d, acc);
            dimg[i] = 2.f * scale * d;
        } else {
            acc += fabsf(d);
            dimg[i] = d > 0.f ? scale : (d < 0.f ? -scale : 0.f);
        }
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int w = 0; w < 8; ++w) s += red[w];
        partials[blockIdx.x] = s * scale;      // summed in block order afterwards
    }
}

__global__ void __launch_bounds__(256) k_adam(int rows, int n, int stride, float *__restrict__ p,
                                              const float *__restrict__ g, float *__restrict__ m,
                                              float *__restrict__ v, float lr, float b1, float b2, float eps,
                                              float ibc1, float ibc2, const uint8_t *__restrict__ skip,
                                              uint16_t *__restrict__ pb) {
    const int r = blockIdx.y;                      // one grid row per parameter plane
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const size_t o = (size_t)r * stride + i;
        if (skip && skip[i]) continue;
        const float gr = g[o];
        const float mm = fmaf(b1, m[o], (1.f - b1) * gr);
        const float vv = fmaf(b2, v[o], (1.f - b2) * gr * gr);
        m[o] = mm;
        v[o] = vv;
        const float np = p[o] - lr * (mm * ibc1) / (sqrtf(vv * ibc2) + eps);
        p[o] = np;
        if (pb) pb[o] = __bfloat16_as_ushort(__float2bfloat16_rn(np));
    }
}

struct AdamGroups {
    qn_adam_group g[QN_ADAM_MAX_GROUPS];
    int row_start[QN_ADAM_MAX_GROUPS + 1];       // first grid row of each group
    int n_groups;
};

__global__ void k_step_increment(int32_t *step) { *step += 1; }

// Grid row y updates row y - row_start[g] of the group g that holds it.
__global__ void __launch_bounds__(256) k_adam_groups(const __grid_constant__ AdamGroups G,
                                                     const int32_t *__restrict__ step, float b1, float b2,
                                                     float eps, const uint8_t *__restrict__ skip) {
    __shared__ float ibc[2];
    if (threadIdx.x == 0) {
        const double t = (double)*step;
        ibc[0] = (float)(1.0 / (1.0 - pow((double)b1, t)));
        ibc[1] = (float)(1.0 / (1.0 - pow((double)b2, t)));
    }
    __syncthreads();
    const int y = blockIdx.y;
    int gi = 0;
    while (gi + 1 < G.n_groups && G.row_start[gi + 1] <= y) ++gi;
    const qn_adam_group &P = G.g[gi];
    const int r = y - G.row_start[gi];
    const uint8_t *sk = P.use_skip ? skip : nullptr;
    const float ibc1 = ibc[0], ibc2 = ibc[1];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x) {
        const size_t o = (size_t)r * P.stride + i;
        if (sk && sk[i]) continue;
        const float gr = P.grad[o];
        const float mm = fmaf(b1, P.m[o], (1.f - b1) * gr);
        const float vv = fmaf(b2, P.v[o], (1.f - b2) * gr * gr);
        P.m[o] = mm;
        P.v[o] = vv;
        const float np = P.param[o] - P.lr * (mm * ibc1) / (sqrtf(vv * ibc2) + eps);
        P.param[o] = np;
        if (P.param_bf16) P.param_bf16[o] = __bfloat16_as_ushort(__float2bfloat16_rn(np));
    }
}

int grid_cap(long long work, int block) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long need = (work + block - 1) / block;
    const long long cap = (long long)sms * 8;
    if (need > cap) need = cap;
    return need < 1 ? 1 : (int)need;
}

}  // namespace
}  // namespace qn

extern "C" int qn_image_loss(int64_t count, const float *img, const float *target, float w, int32_t mse,
                             float *loss, float *d_img, float *partials, qn_stream_t stream) {
    QN_REQUIRE(count >= 0, "count must be >= 0");
    QN_REQUIRE(loss && (count == 0 || (img && target && d_img)), "null pointer argument");
    cudaStream_t s = qn::as_stream(stream);
    if (count == 0) {
        if (cudaMemsetAsync(loss, 0, sizeof(float), s) != cudaSuccess) return qn::check_launch("qn_image_loss memset");
        return QN_OK;
    }
    QN_REQUIRE(partials, "partials is required");
    const float scale = (float)((double)w / (double)count);
    int grid = qn::grid_cap(count, 256);
    if (grid > QN_LOSS_BLOCKS) grid = QN_LOSS_BLOCKS;
    qn::k_image_loss<<<grid, 256, 0, s>>>(count, img, target, scale, mse, partials, d_img);
    qn::k_sum_partials<<<1, 32, 0, s>>>(1, grid, partials, loss);
    return qn::check_launch("qn_image_loss");
}

extern "C" int qn_adam(int32_t rows, int32_t n, int32_t stride, float *param, const float *grad, float *m,
                       float *v, int32_t step, float lr, float beta1, float beta2, float eps,
                       const uint8_t *skip, uint16_t *param_bf16, qn_stream_t stream) {
    QN_REQUIRE(rows >= 0 && n >= 0 && stride >= n, "bad rows / n / stride");
    QN_REQUIRE(step >= 1, "step counts from 1");
    QN_REQUIRE(beta1 >= 0.f && beta1 < 1.f && beta2 >= 0.f && beta2 < 1.f && eps > 0.f, "bad Adam constants");
    if ((long long)rows * n == 0) return QN_OK;
    QN_REQUIRE(param && grad && m && v, "null pointer argument");
    const float ibc1 = (float)(1.0 / (1.0 - std::pow((double)beta1, step)));
    const float ibc2 = (float)(1.0 / (1.0 - std::pow((double)beta2, step)));
    int gx = qn::grid_cap(n, 256);
    const int per_row = qn::div_up((int64_t)gx, rows);      // keep the total near the grid cap
    gx = per_row < 1 ? 1 : per_row;
    qn::k_adam<<<dim3(gx, rows), 256, 0, qn::as_stream(stream)>>>(
        rows, n, stride, param, grad, m, v, lr, beta1, beta2, eps, ibc1, ibc2, skip, param_bf16);
    return qn::check_launch("qn_adam");
}

extern "C" int qn_adam_groups(int32_t n_groups, const qn_adam_group *groups_host, int32_t *step, float beta1,
                              float beta2, float eps, const uint8_t *skip, qn_stream_t stream) {
    QN_REQUIRE(n_groups >= 1 && n_groups <= QN_ADAM_MAX_GROUPS, "n_groups must be in 1..%d", QN_ADAM_MAX_GROUPS);
    QN_REQUIRE(groups_host && step, "null pointer argument");
    QN_REQUIRE(beta1 >= 0.f && beta1 < 1.f && beta2 >= 0.f && beta2 < 1.f && eps > 0.f, "bad Adam constants");
    qn::AdamGroups G{};
    G.n_groups = n_groups;
    int rows = 0, nmax = 0;
    for (int k = 0; k < n_groups; ++k) {
        const qn_adam_group &g = groups_host[k];
        QN_REQUIRE(g.rows >= 0 && g.n >= 0 && g.stride >= g.n, "group %d: bad rows / n / stride", k);
        QN_REQUIRE((long long)g.rows * g.n == 0 || (g.param && g.grad && g.m && g.v), "group %d: null pointer", k);
        G.g[k] = g;
        G.row_start[k] = rows;
        rows += g.rows;
        nmax = g.n > nmax ? g.n : nmax;
    }
    G.row_start[n_groups] = rows;
    QN_REQUIRE(rows <= 65535, "too many rows (%d)", rows);
    cudaStream_t s = qn::as_stream(stream);
    qn::k_step_increment<<<1, 1, 0, s>>>(step);
    if (rows == 0 || nmax == 0) return qn::check_launch("qn_adam_groups");
    int gx = qn::grid_cap(nmax, 256);
    const int per_row = qn::div_up((int64_t)gx, rows);      // keep the total near the grid cap
    gx = per_row < 1 ? 1 : per_row;
    qn::k_adam_groups<<<dim3(gx, rows), 256, 0, s>>>(G, step, beta1, beta2, eps, skip);
    return qn::check_launch("qn_adam_groups");
}
