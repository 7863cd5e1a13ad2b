// Data-layout utilities of the learned static skip: a stable partition of the
// Gaussians by a flag and a column gather that applies it to SoA planes.  A
// frame whose skipped Gaussians sit in one contiguous run lets every adjoint
// and optimiser kernel skip whole warps and memory sectors, where a scattered
// mask of the same size saves almost no memory traffic.
#include "common.cuh"

namespace qn {
namespace {

constexpr int PART_BLOCK = 1024;

// ws[b] = number of zero flags in block b.
__global__ void __launch_bounds__(PART_BLOCK) k_part_counts(int n, const uint8_t *__restrict__ flags,
                                                            uint32_t *__restrict__ ws) {
    __shared__ uint32_t wsum[PART_BLOCK / 32];
    const int i = blockIdx.x * PART_BLOCK + threadIdx.x;
    const bool zero = i < n && flags[i] == 0;
    const unsigned b = __ballot_sync(FULL, zero);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = __popc(b);
    __syncthreads();
    if (threadIdx.x < 32) {
        const uint32_t v = __reduce_add_sync(FULL, wsum[threadIdx.x]);
        if (threadIdx.x == 0) ws[blockIdx.x] = v;
    }
}

// In place: ws[b] <- zeros before block b; ws[nb] = total zeros = *n_first.
__global__ void __launch_bounds__(PART_BLOCK) k_part_offsets(int nb, uint32_t *__restrict__ ws,
                                                             int32_t *__restrict__ n_first) {
    __shared__ uint32_t wsum[PART_BLOCK / 32];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int b0 = 0; b0 < nb; b0 += PART_BLOCK) {
        const int b = b0 + threadIdx.x;
        const uint32_t v = b < nb ? ws[b] : 0u;
        uint32_t incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t x = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += x;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        uint32_t before = carry;
        for (int w = 0; w < warp; ++w) before += wsum[w];
        if (b < nb) ws[b] = before + incl - v;
        __syncthreads();
        if (threadIdx.x == PART_BLOCK - 1) carry = before + incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        ws[nb] = carry;
        *n_first = (int32_t)carry;
    }
}

// perm: zero-flag indices first, then the others, each in increasing order.
__global__ void __launch_bounds__(PART_BLOCK) k_part_scatter(int n, const uint8_t *__restrict__ flags,
                                                             const uint32_t *__restrict__ ws, int nb,
                                                             int32_t *__restrict__ perm) {
    __shared__ uint32_t wz[PART_BLOCK / 32];
    const int i = blockIdx.x * PART_BLOCK + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool valid = i < n;
    const bool zero = valid && flags[i] == 0;
    const unsigned b = __ballot_sync(FULL, zero);
    if (lane == 0) wz[warp] = __popc(b);
    __syncthreads();
    uint32_t zb = 0;                                   // zeros of earlier warps in the block
    for (int w = 0; w < warp; ++w) zb += wz[w];
    const uint32_t zr = zb + __popc(b & lanemask_lt());   // zeros before i within the block
    if (!valid) return;
    const uint32_t z_before = ws[blockIdx.x] + zr;    // zeros before i overall
    const uint32_t pos = zero ? z_before : ws[nb] + ((uint32_t)i - z_before);
    perm[pos] = i;
}

template <typename T>
__global__ void k_gather_columns(int rows, int n, const T *__restrict__ src, long long src_stride,
                                 const int32_t *__restrict__ perm, T *__restrict__ dst, long long dst_stride) {
    const int r = blockIdx.y;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        dst[(size_t)r * dst_stride + i] = src[(size_t)r * src_stride + perm[i]];
}

}  // namespace
}  // namespace qn

extern "C" size_t qn_partition_workspace_size(int32_t n) {
    if (n < 0) return 0;
    return sizeof(uint32_t) * ((size_t)qn::div_up(n, qn::PART_BLOCK) + 1);
}

extern "C" int qn_partition(int32_t n, const uint8_t *flags, int32_t *perm, int32_t *n_first, void *workspace,
                            size_t workspace_bytes, qn_stream_t stream) {
    QN_REQUIRE(n >= 0, "n must be >= 0");
    QN_REQUIRE(n_first, "n_first is required");
    cudaStream_t s = qn::as_stream(stream);
    if (n == 0) {
        if (cudaMemsetAsync(n_first, 0, sizeof(int32_t), s) != cudaSuccess) return qn::check_launch("qn_partition");
        return QN_OK;
    }
    QN_REQUIRE(flags && perm && workspace, "null pointer argument");
    QN_REQUIRE(workspace_bytes >= qn_partition_workspace_size(n), "workspace too small (%zu < %zu)",
               workspace_bytes, qn_partition_workspace_size(n));
    const int nb = qn::div_up(n, qn::PART_BLOCK);
    uint32_t *ws = static_cast<uint32_t *>(workspace);
    qn::k_part_counts<<<nb, qn::PART_BLOCK, 0, s>>>(n, flags, ws);
    qn::k_part_offsets<<<1, qn::PART_BLOCK, 0, s>>>(nb, ws, n_first);
    qn::k_part_scatter<<<nb, qn::PART_BLOCK, 0, s>>>(n, flags, ws, nb, perm);
    return qn::check_launch("qn_partition");
}

extern "C" int qn_gather_columns(int32_t rows, int32_t n, int32_t elem_bytes, const void *src, int64_t src_stride,
                                 const int32_t *perm, void *dst, int64_t dst_stride, qn_stream_t stream) {
    QN_REQUIRE(rows >= 0 && n >= 0, "rows and n must be >= 0");
    QN_REQUIRE(src_stride >= n && dst_stride >= n, "strides must be >= n");
    QN_REQUIRE(elem_bytes == 1 || elem_bytes == 2 || elem_bytes == 4 || elem_bytes == 8,
               "elem_bytes must be 1, 2, 4 or 8");
    QN_REQUIRE(rows <= 65535, "too many rows (%d)", rows);
    if ((long long)rows * n == 0) return QN_OK;
    QN_REQUIRE(src && perm && dst, "null pointer argument");
    QN_REQUIRE(src != dst, "dst may not alias src");
    cudaStream_t s = qn::as_stream(stream);
    const int gx = qn::div_up(n, 256) < 1024 ? qn::div_up(n, 256) : 1024;
    const dim3 grid(gx, rows);
    switch (elem_bytes) {
        case 1: qn::k_gather_columns<uint8_t><<<grid, 256, 0, s>>>(rows, n, (const uint8_t *)src, src_stride, perm,
                                                                  (uint8_t *)dst, dst_stride); break;
        case 2: qn::k_gather_columns<uint16_t><<<grid, 256, 0, s>>>(rows, n, (const uint16_t *)src, src_stride,
                                                                   perm, (uint16_t *)dst, dst_stride); break;
        case 4: qn::k_gather_columns<uint32_t><<<grid, 256, 0, s>>>(rows, n, (const uint32_t *)src, src_stride,
                                                                   perm, (uint32_t *)dst, dst_stride); break;
        default: qn::k_gather_columns<unsigned long long><<<grid, 256, 0, s>>>(
                     rows, n, (const unsigned long long *)src, src_stride, perm, (unsigned long long *)dst,
                     dst_stride); break;
    }
    return qn::check_launch("qn_gather_columns");
}
