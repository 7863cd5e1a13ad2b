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
    int vec[QN_ADAM_MAX_GROUPS];                 // 16-byte aligned planes: four elements per thread
    int n_groups;
};

__global__ void k_step_increment(int32_t *step) { *step += 1; }

struct AdamConst {
    float b1, b2, eps, ibc1, ibc2, lr;
};

__device__ __forceinline__ float adam_update(const AdamConst &c, float p, float g, float &m, float &v) {
    m = fmaf(c.b1, m, (1.f - c.b1) * g);
    v = fmaf(c.b2, v, (1.f - c.b2) * g * g);
    return p - c.lr * (m * c.ibc1) / (sqrtf(v * c.ibc2) + c.eps);
}

// Grid row y updates row y - row_start[g] of the group g that holds it.
__global__ void __launch_bounds__(256) k_adam_groups(const __grid_constant__ AdamGroups G,
                                                     const int32_t *__restrict__ step, float b1, float b2,
                                                     float eps, const uint8_t *__restrict__ skip) {
    // bias corrections 1 / (1 - b^t), each thread on its own (no barrier):
    // 1 - b^t = -expm1(t log1p(b - 1)) has no cancellation, and b - 1 is exact
    const float t = (float)*step;
    const float ibc1 = -1.f / expm1f(t * log1pf(b1 - 1.f));
    const float ibc2 = -1.f / expm1f(t * log1pf(b2 - 1.f));
    const int y = blockIdx.y;
    int gi = 0;
    while (gi + 1 < G.n_groups && G.row_start[gi + 1] <= y) ++gi;
    const qn_adam_group &P = G.g[gi];
    const int r = y - G.row_start[gi];
    const uint8_t *sk = P.use_skip ? skip : nullptr;
    const AdamConst c{b1, b2, eps, ibc1, ibc2, P.lr};
    const size_t row = (size_t)r * P.stride;
    const int stride = gridDim.x * blockDim.x;
    int done = 0;                                      // elements covered by the vector loop
    if (G.vec[gi]) {
        const int nq = P.n / 4;
        done = nq * 4;
        for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += stride) {
            const int i = 4 * q;
            uchar4 s4 = make_uchar4(0, 0, 0, 0);
            if (sk) s4 = *reinterpret_cast<const uchar4 *>(sk + i);
            if (s4.x && s4.y && s4.z && s4.w) continue;
            const float4 g4 = *reinterpret_cast<const float4 *>(P.grad + row + i);
            float4 m4 = *reinterpret_cast<const float4 *>(P.m + row + i);
            float4 v4 = *reinterpret_cast<const float4 *>(P.v + row + i);
            float4 p4 = *reinterpret_cast<const float4 *>(P.param + row + i);
            if (!s4.x) p4.x = adam_update(c, p4.x, g4.x, m4.x, v4.x);
            if (!s4.y) p4.y = adam_update(c, p4.y, g4.y, m4.y, v4.y);
            if (!s4.z) p4.z = adam_update(c, p4.z, g4.z, m4.z, v4.z);
            if (!s4.w) p4.w = adam_update(c, p4.w, g4.w, m4.w, v4.w);
            *reinterpret_cast<float4 *>(P.param + row + i) = p4;
            *reinterpret_cast<float4 *>(P.m + row + i) = m4;
            *reinterpret_cast<float4 *>(P.v + row + i) = v4;
            if (P.param_bf16) {
                uint16_t *pb = P.param_bf16 + row + i;
                const float pv[4] = {p4.x, p4.y, p4.z, p4.w};
                const uint8_t sv[4] = {s4.x, s4.y, s4.z, s4.w};
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (!sv[e]) pb[e] = __bfloat16_as_ushort(__float2bfloat16_rn(pv[e]));
            }
        }
    }
    for (int i = done + blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += stride) {
        if (sk && sk[i]) continue;
        const size_t o = row + i;
        float m = P.m[o], v = P.v[o];
        const float np = adam_update(c, P.param[o], P.grad[o], m, v);
        P.m[o] = m;
        P.v[o] = v;
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
        auto a16 = [](const void *p) { return ((uintptr_t)p & 15) == 0; };
        G.vec[k] = a16(g.param) && a16(g.grad) && a16(g.m) && a16(g.v) && g.stride % 4 == 0 &&
                   (!g.param_bf16 || ((uintptr_t)g.param_bf16 & 7) == 0);
        rows += g.rows;
        nmax = g.n > nmax ? g.n : nmax;
    }
    G.row_start[n_groups] = rows;
    if (skip && ((uintptr_t)skip & 3))                      // the vector loop reads the mask as uchar4
        for (int k = 0; k < n_groups; ++k)
            if (G.g[k].use_skip) G.vec[k] = 0;
    QN_REQUIRE(rows <= 65535, "too many rows (%d)", rows);
    cudaStream_t s = qn::as_stream(stream);
    qn::k_step_increment<<<1, 1, 0, s>>>(step);
    if (rows == 0 || nmax == 0) return qn::check_launch("qn_adam_groups");
    // blocks per row: enough for the longest row's quads, with all rows
    // together near the grid cap (8 blocks per SM)
    const int cap = qn::grid_cap(1LL << 40, 256);
    int gx = qn::div_up((int64_t)cap, rows);
    const int need = qn::div_up((int64_t)((nmax + 3) / 4), 256);
    gx = gx > need ? need : gx;
    gx = gx < 1 ? 1 : gx;
    qn::k_adam_groups<<<dim3(gx, rows), 256, 0, s>>>(G, step, beta1, beta2, eps, skip);
    return qn::check_launch("qn_adam_groups");
}
