// Learned static-skip MLP (not part of the paper): features, forward, and a
// fused BCE backward.  16 -> 64 -> 64 -> 1 with ReLU, BF16 weights, FP32
// accumulation.  Parameter vector (QN_MLP_PARAMS = 5313 entries):
//   W1 [64][16] | b1 [64] | W2 [64][64] | b2 [64] | W3 [64] | b3
//
// The layers are 16- and 64-wide: per row the forward is ~5.2k FMAs on 64
// bytes of features, run once per frame (inference) and over a few epochs on
// the first frames (training), a few percent of a frame's cost; the kernels
// use FP32 FMAs on weights staged in shared memory.
#include <cmath>

#include "common.cuh"

namespace qn {
namespace {

constexpr int F = QN_MLP_FEATURES;   // 16
constexpr int HID = 64;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + HID * F, OFF_W2 = OFF_B1 + HID, OFF_B2 = OFF_W2 + HID * HID,
              OFF_W3 = OFF_B2 + HID, OFF_B3 = OFF_W3 + HID;
static_assert(OFF_B3 + 1 == QN_MLP_PARAMS, "parameter layout");

__device__ __forceinline__ float bf(uint16_t b) { return __uint_as_float(static_cast<uint32_t>(b) << 16); }

__device__ __forceinline__ float sigm(float x) { return 1.f / (1.f + __expf(-x)); }

__global__ void k_skip_features(int n, int S, const float *__restrict__ score, const float *__restrict__ median,
                                const float *__restrict__ A, const float *__restrict__ pg,
                                const float *__restrict__ pla, const float *__restrict__ plp,
                                const uint8_t *__restrict__ pstat, float shift, float *__restrict__ X) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const size_t s = S;
    const float dx = score[i], dy = score[s + i];
    const float nrm = sqrtf(dx * dx + dy * dy);
    const float med = *median;
    float f0, f1 = 0.f;
    if (med > 0.f) {
        f0 = nrm / (nrm + med);
        f1 = fminf(fmaxf(logf(nrm / med + 1e-6f), -8.f), 8.f) * 0.25f;
    } else {
        f0 = nrm > 0.f ? 1.f : 0.f;
    }
    const float g = pg ? pg[i] : 0.f;
    const float la = pla ? pla[i] : 0.f;
    float dpn = 0.f;
    if (plp) {
        const float a = plp[i], b = plp[s + i], c = plp[2 * s + i];
        dpn = fminf(fmaxf(100.f * fabsf(g) * sqrtf(a * a + b * b + c * c), 0.f), 8.f);
    }
    X[i] = f0;
    X[s + i] = f1;
    X[2 * s + i] = dx / (nrm + 1e-20f);
    X[3 * s + i] = dy / (nrm + 1e-20f);
    X[4 * s + i] = A[i];
    X[5 * s + i] = A[s + i];
    X[6 * s + i] = A[2 * s + i];
    X[7 * s + i] = g;
    X[8 * s + i] = sigm(la - shift);
    X[9 * s + i] = sigm(A[10 * s + i]);
    X[10 * s + i] = (A[7 * s + i] + 3.f) * 0.5f;
    X[11 * s + i] = (A[8 * s + i] + 3.f) * 0.5f;
    X[12 * s + i] = (A[9 * s + i] + 3.f) * 0.5f;
    X[13 * s + i] = dpn;
    X[14 * s + i] = pstat ? (pstat[i] ? 1.f : 0.f) : (g == 0.f ? 1.f : 0.f);
    X[15 * s + i] = 1.f;
}

__global__ void __launch_bounds__(256) k_skip_mlp_fwd(int n, int S, const float *__restrict__ X,
                                                      const uint16_t *__restrict__ P, float logit_thr,
                                                      float *__restrict__ logits, uint8_t *__restrict__ skip) {
    __shared__ float w[QN_MLP_PARAMS];
    for (int k = threadIdx.x; k < QN_MLP_PARAMS; k += blockDim.x) w[k] = bf(P[k]);
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float x[F];
#pragma unroll
    for (int m = 0; m < F; ++m) x[m] = X[(size_t)m * S + i];
    float h1[HID];
#pragma unroll
    for (int j = 0; j < HID; ++j) {
        float z = w[OFF_B1 + j];
#pragma unroll
        for (int m = 0; m < F; ++m) z = fmaf(w[OFF_W1 + j * F + m], x[m], z);
        h1[j] = fmaxf(z, 0.f);
    }
    float out = w[OFF_B3];
    for (int o = 0; o < HID; ++o) {
        float z = w[OFF_B2 + o];
#pragma unroll
        for (int j = 0; j < HID; ++j) z = fmaf(w[OFF_W2 + o * HID + j], h1[j], z);
        out = fmaf(w[OFF_W3 + o], fmaxf(z, 0.f), out);
    }
    if (logits) logits[i] = out;
    if (skip) skip[i] = out > logit_thr ? 1 : 0;
}

// Fused backward of the mean BCE over rows [0, n): each block walks 32-row
// tiles, recomputes the forward in shared memory, forms the layer adjoints
// and accumulates every weight gradient in registers; each block writes its
// partial gradient, summed over blocks in block order by a second kernel.
constexpr int R = 32;            // rows per tile
constexpr int BT = 256;          // threads
constexpr int LD = HID + 1;      // padded row stride
constexpr int XLD = F + 1;
constexpr int SMEM_FLOATS = QN_MLP_PARAMS + 3 + R * XLD + 4 * R * LD + 2 * R + 8 * R + R;

__global__ void __launch_bounds__(BT) k_skip_mlp_bwd(int n, int S, const float *__restrict__ X,
                                                     const uint8_t *__restrict__ labels,
                                                     const uint16_t *__restrict__ P, float inv_n,
                                                     float *__restrict__ partials, float *__restrict__ lpart) {
    extern __shared__ float sm[];
    float *w = sm;                                   // QN_MLP_PARAMS (+3 pad)
    float *xs = w + QN_MLP_PARAMS + 3;               // [R][XLD]
    float *h1 = xs + R * XLD;                        // [R][LD]
    float *z2 = h1 + R * LD;
    float *dh2 = z2 + R * LD;
    float *dh1 = dh2 + R * LD;
    float *dz3 = dh1 + R * LD;                       // [R]
    float *ys = dz3 + R;                             // [R]
    float *part = ys + R;                            // [8][R]
    float *lsum = part + 8 * R;                      // [R]
    for (int k = threadIdx.x; k < QN_MLP_PARAMS; k += BT) w[k] = bf(P[k]);
    const int t = threadIdx.x, lane_r = t % R, grp = t / R;   // grp 0..7
    // register accumulators: dW2 (16 per thread), dW1 (4 per thread), and for
    // t < 64 one entry each of dW3, db2, db1; b3 on thread 0
    float gW2[16], gW1[4];
#pragma unroll
    for (int q = 0; q < 16; ++q) gW2[q] = 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) gW1[q] = 0.f;
    float gW3 = 0.f, gb2 = 0.f, gb1 = 0.f, gb3 = 0.f, lacc = 0.f;
    __syncthreads();
    for (int base = blockIdx.x * R; base < n; base += gridDim.x * R) {
        const int row = base + lane_r;
        const bool valid = row < n;
        // (a) stage features and labels
        for (int m = grp; m < F; m += 8) xs[lane_r * XLD + m] = valid ? X[(size_t)m * S + row] : 0.f;
        if (grp == 0) ys[lane_r] = valid ? (float)labels[row] : 0.f;
        __syncthreads();
        // (b) h1 = relu(W1 x + b1)
        for (int j = grp; j < HID; j += 8) {
            float z = w[OFF_B1 + j];
#pragma unroll
            for (int m = 0; m < F; ++m) z = fmaf(w[OFF_W1 + j * F + m], xs[lane_r * XLD + m], z);
            h1[lane_r * LD + j] = fmaxf(z, 0.f);
        }
        __syncthreads();
        // (c) z2 = W2 h1 + b2
        for (int o = grp; o < HID; o += 8) {
            float z = w[OFF_B2 + o];
#pragma unroll 16
            for (int j = 0; j < HID; ++j) z = fmaf(w[OFF_W2 + o * HID + j], h1[lane_r * LD + j], z);
            z2[lane_r * LD + o] = z;
        }
        __syncthreads();
        // (d) logit and dL/dlogit of the mean BCE
        {
            float s = 0.f;
            for (int o = grp * 8; o < grp * 8 + 8; ++o) s = fmaf(w[OFF_W3 + o], fmaxf(z2[lane_r * LD + o], 0.f), s);
            part[grp * R + lane_r] = s;
        }
        __syncthreads();
        if (t < R) {
            float z = w[OFF_B3];
            for (int g = 0; g < 8; ++g) z += part[g * R + t];
            const float y = ys[t];
            const bool ok = base + t < n;
            dz3[t] = ok ? (sigm(z) - y) * inv_n : 0.f;
            lsum[t] = ok ? fmaxf(z, 0.f) - z * y + log1pf(__expf(-fabsf(z))) : 0.f;
        }
        __syncthreads();
        // (e) dh2 = dz3 W3 [z2 > 0]
        for (int o = grp; o < HID; o += 8)
            dh2[lane_r * LD + o] = z2[lane_r * LD + o] > 0.f ? dz3[lane_r] * w[OFF_W3 + o] : 0.f;
        __syncthreads();
        // (f) dh1 = (W2^T dh2) [h1 > 0]
        for (int j = grp; j < HID; j += 8) {
            float s = 0.f;
#pragma unroll 16
            for (int o = 0; o < HID; ++o) s = fmaf(w[OFF_W2 + o * HID + j], dh2[lane_r * LD + o], s);
            dh1[lane_r * LD + j] = h1[lane_r * LD + j] > 0.f ? s : 0.f;
        }
        __syncthreads();
        // (g) weight gradients summed over the tile's rows
        {
            const int o = t / 4, jb = t % 4;
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int j = jb + 4 * q;
                float s = gW2[q];
                for (int r = 0; r < R; ++r) s = fmaf(dh2[r * LD + o], h1[r * LD + j], s);
                gW2[q] = s;
            }
            const int jj = t / 4, mb = t % 4;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int m = mb + 4 * q;
                float s = gW1[q];
                for (int r = 0; r < R; ++r) s = fmaf(dh1[r * LD + jj], xs[r * XLD + m], s);
                gW1[q] = s;
            }
            if (t < HID) {
                for (int r = 0; r < R; ++r) {
                    gW3 = fmaf(dz3[r], fmaxf(z2[r * LD + t], 0.f), gW3);
                    gb2 += dh2[r * LD + t];
                    gb1 += dh1[r * LD + t];
                }
            }
            if (t == 0)
                for (int r = 0; r < R; ++r) {
                    gb3 += dz3[r];
                    lacc += lsum[r];
                }
        }
        __syncthreads();
    }
    // this block's partial gradient (and loss); summed in block order afterwards
    float *dP = partials + (size_t)blockIdx.x * QN_MLP_PARAMS;
    {
        const int o = t / 4, jb = t % 4;
#pragma unroll
        for (int q = 0; q < 16; ++q) dP[OFF_W2 + o * HID + jb + 4 * q] = gW2[q];
        const int jj = t / 4, mb = t % 4;
#pragma unroll
        for (int q = 0; q < 4; ++q) dP[OFF_W1 + jj * F + mb + 4 * q] = gW1[q];
        if (t < HID) {
            dP[OFF_W3 + t] = gW3;
            dP[OFF_B2 + t] = gb2;
            dP[OFF_B1 + t] = gb1;
        }
        if (t == 0) {
            dP[OFF_B3] = gb3;
            lpart[blockIdx.x] = lacc * inv_n;
        }
    }
}

// label = 1 when the frame's residual of the Gaussian is exactly zero: gate
// closed and every latent rounds to 0
__global__ void k_skip_labels(int n, int S, int n_lat, const float *__restrict__ gate,
                              const float *__restrict__ lat, const uint8_t *__restrict__ hit,
                              uint8_t *__restrict__ labels) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    bool zero = gate[i] == 0.f && !(hit && hit[i]);
    for (int k = 0; k < n_lat && zero; ++k) zero = rintf(lat[(size_t)k * S + i]) == 0.f;
    labels[i] = zero ? 1 : 0;
}

int sm_count() {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

}  // namespace
}  // namespace qn

extern "C" int qn_skip_features(int32_t n, int32_t n_stride, int32_t n_attr, const float *score,
                                const float *median, const float *prev, const float *prev_gate,
                                const float *prev_log_alpha, const float *prev_lp, const uint8_t *prev_static,
                                const qn_gate_params *gate_host, float *X, qn_stream_t stream) {
    QN_REQUIRE(n >= 0 && n_stride >= n && n_stride % 4 == 0, "bad n / n_stride");
    QN_REQUIRE(n_attr >= 11, "n_attr must be >= 11");
    QN_REQUIRE(gate_host && gate_host->tau > 0.f && gate_host->gamma0 < 0.f && gate_host->gamma1 > 1.f,
               "gate parameters out of range");
    QN_REQUIRE(n == 0 || (score && median && prev && X), "null pointer argument");
    if (n == 0) return QN_OK;
    const float shift = (float)(gate_host->tau * std::log(-(double)gate_host->gamma0 / (double)gate_host->gamma1));
    qn::k_skip_features<<<qn::div_up(n, 256), 256, 0, qn::as_stream(stream)>>>(
        n, n_stride, score, median, prev, prev_gate, prev_log_alpha, prev_lp, prev_static, shift, X);
    return qn::check_launch("qn_skip_features");
}

extern "C" int qn_skip_mlp_fwd(int32_t n, int32_t n_stride, const float *X, const uint16_t *params,
                               float threshold, float *logits, uint8_t *skip, qn_stream_t stream) {
    QN_REQUIRE(n >= 0 && n_stride >= n, "bad n / n_stride");
    QN_REQUIRE(threshold > 0.f && threshold < 1.f, "threshold must lie in (0, 1)");
    QN_REQUIRE(n == 0 || (X && params && (logits || skip)), "null pointer argument");
    if (n == 0) return QN_OK;
    const float thr = std::log(threshold / (1.f - threshold));     // sigmoid(z) > threshold  <=>  z > thr
    qn::k_skip_mlp_fwd<<<qn::div_up(n, 256), 256, 0, qn::as_stream(stream)>>>(n, n_stride, X, params, thr,
                                                                             logits, skip);
    return qn::check_launch("qn_skip_mlp_fwd");
}

extern "C" int qn_skip_mlp_bwd(int32_t n, int32_t n_stride, const float *X, const uint8_t *labels,
                               const uint16_t *params, float *d_params, float *loss, float *partials,
                               qn_stream_t stream) {
    QN_REQUIRE(n >= 1 && n_stride >= n, "bad n / n_stride");
    QN_REQUIRE(X && labels && params && d_params && partials, "null pointer argument");
    cudaStream_t s = qn::as_stream(stream);
    const size_t smem = sizeof(float) * qn::SMEM_FLOATS;
    if (cudaFuncSetAttribute(qn::k_skip_mlp_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return qn::check_launch("qn_skip_mlp_bwd attribute");
    const int tiles = qn::div_up(n, qn::R);
    int grid = tiles < qn::sm_count() ? tiles : qn::sm_count();
    if (grid > QN_MLP_BWD_BLOCKS) grid = QN_MLP_BWD_BLOCKS;
    float *lpart = partials + (size_t)QN_MLP_BWD_BLOCKS * QN_MLP_PARAMS;
    qn::k_skip_mlp_bwd<<<grid, qn::BT, smem, s>>>(n, n_stride, X, labels, params, 1.f / (float)n, partials, lpart);
    qn::k_sum_partials<<<qn::sum_partials_grid(QN_MLP_PARAMS), 256, 0, s>>>(QN_MLP_PARAMS, grid, partials, d_params);
    if (loss) qn::k_sum_partials<<<1, 32, 0, s>>>(1, grid, lpart, loss);
    return qn::check_launch("qn_skip_mlp_bwd");
}

extern "C" int qn_skip_labels(int32_t n, int32_t n_stride, int32_t n_latent, const float *gate, const float *lat,
                              const uint8_t *hit, uint8_t *labels, qn_stream_t stream) {
    QN_REQUIRE(n >= 0 && n_stride >= n && n_latent >= 0, "bad n / n_stride / n_latent");
    QN_REQUIRE(n == 0 || (gate && labels && (n_latent == 0 || lat)), "null pointer argument");
    if (n == 0) return QN_OK;
    qn::k_skip_labels<<<qn::div_up(n, 256), 256, 0, qn::as_stream(stream)>>>(n, n_stride, n_latent, gate, lat, hit,
                                                                            labels);
    return qn::check_launch("qn_skip_labels");
}

namespace qn {
namespace {
__global__ void k_or_marks(int n, const uint8_t *__restrict__ src, uint8_t *__restrict__ dst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && src[i]) dst[i] = 1;
}

__global__ void k_clear_marked(int n, const uint8_t *__restrict__ marks, uint8_t *__restrict__ flags) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && marks[i]) flags[i] = 0;
}
}  // namespace
}  // namespace qn

extern "C" int qn_or_marks(int32_t n, const uint8_t *src, uint8_t *dst, qn_stream_t stream) {
    QN_REQUIRE(n >= 0, "n must be >= 0");
    if (n == 0) return QN_OK;
    QN_REQUIRE(src && dst, "null pointer argument");
    qn::k_or_marks<<<qn::div_up(n, 256), 256, 0, qn::as_stream(stream)>>>(n, src, dst);
    return qn::check_launch("qn_or_marks");
}

extern "C" int qn_clear_marked(int32_t n, const uint8_t *marks, uint8_t *flags, qn_stream_t stream) {
    QN_REQUIRE(n >= 0, "n must be >= 0");
    if (n == 0) return QN_OK;
    QN_REQUIRE(marks && flags, "null pointer argument");
    qn::k_clear_marked<<<qn::div_up(n, 256), 256, 0, qn::as_stream(stream)>>>(n, marks, flags);
    return qn::check_launch("qn_clear_marked");
}
