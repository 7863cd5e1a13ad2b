// Shared helpers of the CUDA translation units: status codes, argument
// checks, launch checks and warp utilities.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "queen.h"

namespace qn {

// Records a message for qn_last_error() on the calling host thread.
void set_error(const char *fmt, ...);
void clear_error();

inline cudaStream_t as_stream(qn_stream_t s) { return reinterpret_cast<cudaStream_t>(s); }

// Returns QN_ERR_CUDA with the message of the last launch error, or QN_OK.
int check_launch(const char *what);

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// Sum over the warp of v[0..7] scattered across lanes (lane l ends up with
// the total of value (l >> 2) & 7): 9 shuffles instead of the 40 of eight
// independent butterflies.
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

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

inline int div_up(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// out[e] = sum over b < blocks of partials[b * count + e] in a fixed order
// (a reproducible reduction of per-block partial sums); launch with
// 32 * count threads.
__global__ void k_sum_partials(int count, int blocks, const float *__restrict__ partials, float *__restrict__ out);

inline int sum_partials_grid(int count) { return (int)(((int64_t)count * 32 + 255) / 256); }

__device__ __forceinline__ int div_up_dev(int a, int b) { return (a + b - 1) / b; }

// Programmatic dependent launch: a kernel launched by pdl_launch may be
// scheduled while the kernel before it in the stream is still running.  Its
// first statement is pdl_enter(): it waits until that kernel has completed
// and its writes are visible (so nothing of the kernel overlaps its
// predecessor but its launch), then lets the next kernel be scheduled early
// in turn.  Without a programmatic predecessor the wait returns at once.
__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
cudaError_t pdl_launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<Args &&>(args)...);
}

// Compositing (render.cu), used by the workspace-aware entry points of the
// compositing adjoint (binning.cu): argument checks shared by both passes, and
// the first pass of the adjoint (per-pair records, visited prefixes, marks).
int check_render_args(const qn_camera *cam, const uint32_t *ranges, const uint32_t *vals, const qn_splat *sp);
int launch_render_bwd(const qn_camera *cam, const uint32_t *ranges, const uint32_t *vals, const qn_splat *splats,
                      const float *bg, const float *T_final, const uint32_t *last, const float *d_img,
                      const uint8_t *skip, const uint8_t *composited, const uint32_t *order,
                      qn_splat *pair_grads, uint32_t *visited, uint8_t *hit, cudaStream_t stream);

}  // namespace qn

#define QN_REQUIRE(cond, ...)                 \
    do {                                      \
        if (!(cond)) {                        \
            qn::set_error(__VA_ARGS__);       \
            return QN_ERR_INVALID_ARG;        \
        }                                     \
    } while (0)
