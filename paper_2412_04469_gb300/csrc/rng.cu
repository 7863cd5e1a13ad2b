// Counter-based uniform numbers for the stochastic hard-concrete gate:
// Philox4x32-10 (Salmon, Moraes, Dror and Shaw, SC 2011) over the counter
// (Gaussian, step), so every Gaussian's noise at every step is independent of
// launch shape and order.
#include "common.cuh"

namespace qn {
namespace {

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
    constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k.x += W0;
            k.y += W1;
        }
        const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
        const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

__global__ void k_gate_uniform(int n, uint2 key, const int32_t *__restrict__ step, float *__restrict__ u) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t x = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)*step, 0u, 0u), key).x;
    u[i] = ((float)(x >> 9) + 0.5f) * (1.f / 8388608.f);     // exact: 24 significant bits
}

}  // namespace
}  // namespace qn

extern "C" int qn_gate_uniform(int32_t n, uint64_t seed, const int32_t *step, float *u, qn_stream_t stream) {
    QN_REQUIRE(n >= 0, "n must be >= 0");
    if (n == 0) return QN_OK;
    QN_REQUIRE(step && u, "null pointer argument");
    const uint2 key = make_uint2((uint32_t)(seed & 0xFFFFFFFFull), (uint32_t)(seed >> 32));
    qn::k_gate_uniform<<<qn::div_up(n, 256), 256, 0, qn::as_stream(stream)>>>(n, key, step, u);
    return qn::check_launch("qn_gate_uniform");
}
