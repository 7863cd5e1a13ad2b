// Viewspace gradient difference (Sec. 3.3, Eq. 9) and gate initialisation
// (Eq. 10 with Eq. 8 solved for log alpha).
//
// Eq. 9 is linear in the target image, so for each view the difference of the
// two MSE gradients is one compositing adjoint with the upstream image
// 2 (I_{t-1} - I_t) / (3 H W) (qn_image_loss with mse); qn_viewspace_accum
// adds its 2D-mean part, scaled by 1/V, into the score d_t.
#include <cmath>

#include "common.cuh"

namespace qn {
namespace {

__global__ void k_viewspace_accum(int n, int S, const float4 *__restrict__ dsp, float scale,
                                  float *__restrict__ score) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 g = dsp[3 * (size_t)i];
    score[i] += scale * g.x;
    score[(size_t)S + i] += scale * g.y;
}

__global__ void k_score_norms(int n, int S, const float *__restrict__ score, float *__restrict__ norms) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float x = score[i], y = score[(size_t)S + i];
    norms[i] = sqrtf(x * x + y * y);
}

// Lower median (element (m - 1) / 2 of the m sorted values) of n
// non-negative floats -- of all of them, or with `nonzero` of the m that are
// not zero (0 when there are none) -- by a most-significant-byte-first radix
// select on their bit patterns (non-negative IEEE floats order like their
// bits).  One block.
__global__ void __launch_bounds__(1024) k_median_select(int n, int nonzero, const float *__restrict__ v,
                                                        float *__restrict__ med) {
    __shared__ uint32_t hist[256];
    __shared__ uint32_t s_prefix, s_k, s_m;
    if (threadIdx.x == 0) {
        s_prefix = 0;
        s_m = 0;
    }
    __syncthreads();
    uint32_t cnt = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) cnt += (!nonzero || __float_as_uint(v[i]) != 0u) ? 1u : 0u;
    cnt = __reduce_add_sync(FULL, cnt);
    if ((threadIdx.x & 31) == 0) atomicAdd(&s_m, cnt);
    __syncthreads();
    if (s_m == 0) {
        if (threadIdx.x == 0) *med = 0.f;
        return;
    }
    if (threadIdx.x == 0) s_k = (s_m - 1) / 2;
    for (int pass = 3; pass >= 0; --pass) {
        const int shift = 8 * pass;
        const uint32_t mask = pass == 3 ? 0u : (0xffffffffu << (shift + 8));
        if (threadIdx.x < 256) hist[threadIdx.x] = 0;
        __syncthreads();
        const uint32_t prefix = s_prefix;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const uint32_t b = __float_as_uint(v[i]);
            if ((b & mask) == prefix && (!nonzero || b != 0u)) atomicAdd(&hist[(b >> shift) & 255u], 1u);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t k = s_k, d = 0;
            while (d < 255 && k >= hist[d]) {
                k -= hist[d];
                ++d;
            }
            s_k = k;
            s_prefix = prefix | (d << shift);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *med = __uint_as_float(s_prefix);
}

__global__ void k_gate_from_score(int n, const float *__restrict__ norms, const float *__restrict__ med,
                                  float shift, float *__restrict__ log_alpha) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float m = *med, d = norms[i];
    float p = m > 0.f ? d / (d + m) : (d > 0.f ? 1.f : 0.f);           // Eq. 10
    p = fminf(fmaxf(p, 1e-6f), 1.f - 1e-6f);
    log_alpha[i] = logf(p / (1.f - p)) + shift;                         // Eq. 8 solved for log alpha
}

}  // namespace
}  // namespace qn

extern "C" int qn_viewspace_accum(int32_t n, int32_t n_stride, const qn_splat *d_splats, float scale,
                                  float *score, qn_stream_t stream) {
    QN_REQUIRE(n >= 0 && n_stride >= n, "bad n / n_stride");
    QN_REQUIRE(n == 0 || (d_splats && score), "null pointer argument");
    QN_REQUIRE(((uintptr_t)d_splats & 15) == 0, "d_splats must be 16-byte aligned");
    if (n == 0) return QN_OK;
    qn::k_viewspace_accum<<<qn::div_up(n, 256), 256, 0, qn::as_stream(stream)>>>(
        n, n_stride, reinterpret_cast<const float4 *>(d_splats), scale, score);
    return qn::check_launch("qn_viewspace_accum");
}

extern "C" int qn_gate_init(int32_t n, int32_t n_stride, const float *score, const qn_gate_params *gate_host,
                            int32_t nonzero_median, float *norms, float *median, float *log_alpha,
                            qn_stream_t stream) {
    QN_REQUIRE(n >= 1 && n_stride >= n, "bad n / n_stride");
    QN_REQUIRE(gate_host && gate_host->tau > 0.f && gate_host->gamma0 < 0.f && gate_host->gamma1 > 1.f,
               "gate parameters out of range");
    QN_REQUIRE(score && norms && median && log_alpha, "null pointer argument");
    cudaStream_t s = qn::as_stream(stream);
    const float shift = (float)(gate_host->tau * std::log(-(double)gate_host->gamma0 / (double)gate_host->gamma1));
    qn::k_score_norms<<<qn::div_up(n, 256), 256, 0, s>>>(n, n_stride, score, norms);
    qn::k_median_select<<<1, 1024, 0, s>>>(n, nonzero_median != 0, norms, median);
    qn::k_gate_from_score<<<qn::div_up(n, 256), 256, 0, s>>>(n, norms, median, shift, log_alpha);
    return qn::check_launch("qn_gate_init");
}
