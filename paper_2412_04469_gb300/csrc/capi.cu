// Error reporting of the C ABI.
#include <cstdarg>
#include <cstdio>

#include "common.cuh"

namespace {
thread_local char g_err[512] = "";
}

namespace qn {

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

void clear_error() { g_err[0] = 0; }

int check_launch(const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("%s: %s", what, cudaGetErrorString(e));
        return QN_ERR_CUDA;
    }
    return QN_OK;
}

__global__ void k_sum_partials(int count, int blocks, const float *__restrict__ partials, float *__restrict__ out) {
    // one warp per entry: lane l adds blocks l, l + 32, ... in order, then a
    // fixed butterfly combines the lanes
    const int e = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (e >= count) return;
    float s = 0.f;
    for (int b = lane; b < blocks; b += 32) s += partials[(size_t)b * count + e];
    s = warp_sum(s);
    if (lane == 0) out[e] = s;
}

}  // namespace qn

extern "C" const char *qn_last_error(void) { return g_err; }

extern "C" const char *qn_version(void) { return "queen-gb300 0.1 (sm_103a)"; }
