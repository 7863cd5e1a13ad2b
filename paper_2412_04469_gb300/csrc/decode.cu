// Residual decode and hard-concrete position gate (Sec. 3.2, Eq. 4-8) and
// their adjoint.
//
// The decoder contraction is r_c = D_c l_c with K = lat_dim (8 by default):
// about 2 * 56 * 8 flops per 128 bytes of latents, i.e. ~7 flop/byte, far
// below the tensor-core balance point, so it runs as FP32 FMAs on bf16
// weights held in shared memory.  Integer latents (|l| <= 128) times bf16
// weights are exact in FP32; only the sum over K rounds.
#include <cmath>

#include "common.cuh"
#include "project.cuh"

namespace qn {
namespace {

constexpr int MAX_RES_PLANES = 56;     // attribute planes 3 .. 58 (SH degree 3)
constexpr int MAX_LAT_TOTAL = 64;      // latent planes over all categories

struct DecodeArgs {
    int n, stride, n_attr, n_cat, n_dec, n_lat;
    int ab[QN_MAX_CATEGORIES], ac[QN_MAX_CATEGORIES], ld[QN_MAX_CATEGORIES];
    int lat_off[QN_MAX_CATEGORIES], dec_off[QN_MAX_CATEGORIES];
    unsigned long long covered;        // bit k: attribute plane k receives a residual
    float tau, g0, g1, shift;          // shift = tau log(-gamma0 / gamma1)
    const float *noise;                // nullable: u of the stochastic gate
};

__device__ __forceinline__ float bf16_to_f32(uint16_t b) {
    return __uint_as_float(static_cast<uint32_t>(b) << 16);
}

__device__ __forceinline__ float latent_int(float v) {
    return fminf(127.f, fmaxf(-128.f, rintf(v)));   // round half to even, int8 saturation
}

__device__ __forceinline__ float sigmoidf_(float x) { return 1.f / (1.f + __expf(-x)); }

// The gate's argument: log alpha, plus the logistic noise log u - log(1 - u)
// of the stochastic hard-concrete sample when a noise array is given.
template <bool NOISE>
__device__ __forceinline__ float gate_logit(const DecodeArgs &a, float l_a, int i) {
    if (!NOISE) return l_a;
    const float u = a.noise[i];
    return l_a + (logf(u) - log1pf(-u));
}

// The gate's pre-clamp value gh (g1 - g0) + g0 (Eq. 7), the position update
// p + g lp (Eq. 4) and the gate adjoint's d log alpha, each with its
// roundings spelled out, so that every kernel that forms them (decode, fused
// decode-projection, decode adjoint, fused adjoint) gets the same bits.
__device__ __forceinline__ float gate_pre(const DecodeArgs &a, float gh) {
    return __fmaf_rn(gh, __fsub_rn(a.g1, a.g0), a.g0);
}
__device__ __forceinline__ float pos_update(float p, float g, float lp) { return __fmaf_rn(g, lp, p); }
__device__ __forceinline__ float d_log_alpha_of(float dot, float dg, float d_lreg, float p) {
    return __fmaf_rn(dot, dg, __fmul_rn(__fmul_rn(d_lreg, p), __fsub_rn(1.f, p)));
}

// LT > 0: every category has latent width LT (compile-time loops, D rows
// read as float4 broadcasts); LT == 0: any layout within the limits.
template <int LT, bool NOISE>
__global__ void __launch_bounds__(256) k_decode(DecodeArgs a, const float *__restrict__ prev,
                                                const float *__restrict__ lat,
                                                const uint16_t *__restrict__ dec,
                                                const float *__restrict__ lp,
                                                const float *__restrict__ la,
                                                const uint8_t *__restrict__ skip, float *__restrict__ out,
                                                float *__restrict__ gate, float *__restrict__ lreg) {
    __shared__ __align__(16) float sD[MAX_RES_PLANES * QN_MAX_LATENT];
    __shared__ float sred[8];
    for (int k = threadIdx.x; k < a.n_dec; k += blockDim.x) sD[k] = bf16_to_f32(dec[k]);
    __syncthreads();
    const size_t S = a.stride;
    float reg = 0.f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += gridDim.x * blockDim.x) {
        if (skip && skip[i]) continue;                 // frozen: out and gate already hold its values
        const float l_a = la[i];
        const float gh = sigmoidf_(gate_logit<NOISE>(a, l_a, i) / a.tau);   // Eq. 6
        const float g = fminf(1.f, fmaxf(0.f, gate_pre(a, gh)));   // Eq. 7
        if (gate) gate[i] = g;
        reg += sigmoidf_(l_a - a.shift);                                // Eq. 8
#pragma unroll
        for (int d = 0; d < 3; ++d) out[d * S + i] = pos_update(prev[d * S + i], g, lp[d * S + i]);
        for (int c = 0; c < a.n_cat; ++c) {
            const float *D = sD + a.dec_off[c];
            if (LT > 0) {
                float l[LT > 0 ? LT : 1];
#pragma unroll
                for (int k = 0; k < LT; ++k) l[k] = latent_int(lat[(size_t)(a.lat_off[c] + k) * S + i]);
#pragma unroll 8
                for (int r = 0; r < a.ac[c]; ++r) {
                    const float4 *Dr = reinterpret_cast<const float4 *>(D + r * LT);
                    float acc = 0.f;
#pragma unroll
                    for (int k4 = 0; k4 < LT / 4; ++k4) {
                        const float4 w = Dr[k4];
                        acc = fmaf(w.x, l[4 * k4], acc);                // Eq. 5
                        acc = fmaf(w.y, l[4 * k4 + 1], acc);
                        acc = fmaf(w.z, l[4 * k4 + 2], acc);
                        acc = fmaf(w.w, l[4 * k4 + 3], acc);
                    }
                    const size_t o = (size_t)(a.ab[c] + r) * S + i;
                    out[o] = prev[o] + acc;                             // Eq. 4
                }
            } else {
                float l[QN_MAX_LATENT];
                const int L = a.ld[c];
#pragma unroll
                for (int k = 0; k < QN_MAX_LATENT; ++k)
                    if (k < L) l[k] = latent_int(lat[(size_t)(a.lat_off[c] + k) * S + i]);
#pragma unroll 8
                for (int r = 0; r < a.ac[c]; ++r) {
                    float acc = 0.f;
#pragma unroll
                    for (int k = 0; k < QN_MAX_LATENT; ++k)
                        if (k < L) acc = fmaf(D[r * L + k], l[k], acc);     // Eq. 5
                    const size_t o = (size_t)(a.ab[c] + r) * S + i;
                    out[o] = prev[o] + acc;                             // Eq. 4
                }
            }
        }
#pragma unroll 4
        for (int k = 3; k < a.n_attr; ++k)
            if (!((a.covered >> k) & 1ull)) out[(size_t)k * S + i] = prev[(size_t)k * S + i];
    }
    if (lreg) {
        reg = warp_sum(reg);
        if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = reg;
        __syncthreads();
        if (threadIdx.x == 0) {
            float s = 0.f;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sred[w];
            atomicAdd(lreg, s);
        }
    }
}

// Latent width shared by every category, if it is 8 (the layout with a
// compile-time kernel), else 0.
int uniform_width8(const DecodeArgs &a) {
    for (int c = 0; c < a.n_cat; ++c)
        if (a.ld[c] != 8) return 0;
    return 8;
}

// Adjoint, one fused kernel: a block stages 32 Gaussians' residual gradients
// dr and rounded latents l in shared memory, then writes d_lat = D^T dr per
// (Gaussian, latent) and accumulates its share of dD = sum dr l^T in
// registers; each block writes its partial dD, and a second kernel sums the
// partials in block order (no atomics: reproducible).
constexpr int BWD_THREADS = 256;
constexpr int BWD_TILE = 32;
constexpr int BWD_OWN = (MAX_RES_PLANES * QN_MAX_LATENT + BWD_THREADS - 1) / BWD_THREADS;

constexpr int ROWS_PER_PASS = BWD_THREADS / BWD_TILE;
constexpr int PF_DR = (MAX_RES_PLANES + ROWS_PER_PASS - 1) / ROWS_PER_PASS;   // residual rows per thread
constexpr int PF_L = MAX_LAT_TOTAL / ROWS_PER_PASS;                            // latent rows per thread

// The global values one thread stages for one tile: residual gradients of
// rows row0 + 8m, latents of rows row0 + 8m, and (row0 == 0) the gate inputs.
struct TileRegs {
    float dr[PF_DR], l[PF_L];
    float la, lz, dp[3], lp[3];            // lz: the gate's argument (log alpha + noise)
    bool valid, sk;
};

template <bool NOISE>
__device__ __forceinline__ void load_tile(const DecodeArgs &a, int base, int lane, int row0,
                                          const float *__restrict__ lat, const float *__restrict__ lp,
                                          const float *__restrict__ la, const float *__restrict__ d_out,
                                          const uint8_t *__restrict__ skip, TileRegs &t) {
    const size_t S = a.stride;
    const int i = base + lane;
    const int n_res = a.n_attr - 3;
    t.valid = i < a.n;
    t.sk = t.valid && skip && skip[i];
    const bool use = t.valid && !t.sk;
#pragma unroll
    for (int m = 0; m < PF_DR; ++m) {
        const int r = row0 + m * ROWS_PER_PASS;
        t.dr[m] = (use && r < n_res) ? d_out[(size_t)(r + 3) * S + i] : 0.f;
    }
#pragma unroll
    for (int m = 0; m < PF_L; ++m) {
        const int k = row0 + m * ROWS_PER_PASS;
        t.l[m] = (use && k < a.n_lat) ? lat[(size_t)k * S + i] : 0.f;
    }
    if (row0 == 0 && use) {
        t.la = la[i];
        t.lz = gate_logit<NOISE>(a, t.la, i);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            t.dp[d] = d_out[d * S + i];
            t.lp[d] = lp[d * S + i];
        }
    }
}

// LT > 0: every category has latent width LT, so thread row0 computes latent
// row0 of each category (compile-time indexing); LT == 0: any layout.
// Software-pipelined: while a tile is computed from shared memory, the next
// tile's values are already being loaded into registers.
template <int LT, bool NOISE>
__global__ void __launch_bounds__(BWD_THREADS) k_decode_bwd(
    DecodeArgs a, const float *__restrict__ lat, const uint16_t *__restrict__ dec,
    const float *__restrict__ lp, const float *__restrict__ la, const float *__restrict__ d_out,
    float d_lreg, const uint8_t *__restrict__ skip, float *__restrict__ d_lat,
    float *__restrict__ partials, float *__restrict__ d_lp, float *__restrict__ d_la) {
    __shared__ float sD[MAX_RES_PLANES * QN_MAX_LATENT];
    __shared__ float s_dr[MAX_RES_PLANES][BWD_TILE + 1];   // +1: different rows, different banks
    __shared__ float s_l[MAX_LAT_TOTAL][BWD_TILE + 1];
    __shared__ int s_cat[MAX_LAT_TOTAL];                    // category of each latent plane
    for (int k = threadIdx.x; k < a.n_dec; k += BWD_THREADS) sD[k] = bf16_to_f32(dec[k]);
    if (threadIdx.x < a.n_lat) {
        int c = 0;
        while (c + 1 < a.n_cat && (int)threadIdx.x >= a.lat_off[c + 1]) ++c;
        s_cat[threadIdx.x] = c;
    }
    // decoder entries owned by this thread: (category, row, latent)
    int own_c[BWD_OWN], own_r[BWD_OWN], own_k[BWD_OWN];
    float acc[BWD_OWN];
#pragma unroll
    for (int q = 0; q < BWD_OWN; ++q) {
        const int e = threadIdx.x + q * BWD_THREADS;
        int c = 0;
        while (c + 1 < a.n_cat && e >= a.dec_off[c + 1]) ++c;
        const int L = a.ld[c];
        own_c[q] = e < a.n_dec ? c : -1;
        own_r[q] = (e - a.dec_off[c]) / L;
        own_k[q] = (e - a.dec_off[c]) % L;
        acc[q] = 0.f;
    }
    const size_t S = a.stride;
    const int n_res = a.n_attr - 3;
    const int lane = threadIdx.x & (BWD_TILE - 1), row0 = threadIdx.x / BWD_TILE;
    const int step = gridDim.x * BWD_TILE;
    TileRegs t;
    load_tile<NOISE>(a, blockIdx.x * BWD_TILE, lane, row0, lat, lp, la, d_out, skip, t);
    for (int base = blockIdx.x * BWD_TILE; base < a.n; base += step) {
        const int i = base + lane;
        const bool valid = t.valid, sk = t.sk;
        // the barrier also keeps the previous tile's readers ahead of the stores below
        if (__syncthreads_and(!valid || sk)) {            // a tile of skipped Gaussians only zeroes them
            if (valid) {
                for (int k = row0; k < a.n_lat; k += ROWS_PER_PASS) d_lat[(size_t)k * S + i] = 0.f;
                if (row0 == 0) {
                    d_lp[i] = d_lp[S + i] = d_lp[2 * S + i] = 0.f;
                    d_la[i] = 0.f;
                }
            }
            load_tile<NOISE>(a, base + step, lane, row0, lat, lp, la, d_out, skip, t);
            continue;
        }
#pragma unroll
        for (int m = 0; m < PF_DR; ++m) {
            const int r = row0 + m * ROWS_PER_PASS;
            if (r < n_res) s_dr[r][lane] = t.dr[m];
        }
#pragma unroll
        for (int m = 0; m < PF_L; ++m) {
            const int k = row0 + m * ROWS_PER_PASS;
            if (k < a.n_lat) s_l[k][lane] = latent_int(t.l[m]);
        }
        if (row0 == 0 && valid) {
            const float gh = sigmoidf_(t.lz / a.tau);
            const float gt = gate_pre(a, gh);
            const float g = fminf(1.f, fmaxf(0.f, gt));
            const float dg = (gt > 0.f && gt < 1.f) ? (a.g1 - a.g0) * gh * (1.f - gh) / a.tau : 0.f;
            float dot = 0.f;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                d_lp[d * S + i] = sk ? 0.f : g * t.dp[d];
                dot = fmaf(t.dp[d], t.lp[d], dot);
            }
            const float p = sigmoidf_(t.la - a.shift);
            d_la[i] = sk ? 0.f : d_log_alpha_of(dot, dg, d_lreg, p);
        }
        load_tile<NOISE>(a, base + step, lane, row0, lat, lp, la, d_out, skip, t);   // in flight during the compute
        __syncthreads();
        // STE: d_lat[k] = sum_r D[r][k] dr[r] for this thread's (latent, Gaussian) pairs
        if (valid) {
            if (LT > 0) {
#pragma unroll
                for (int c = 0; c < QN_MAX_CATEGORIES; ++c) {
                    if (c >= a.n_cat) break;
                    const float *D = sD + a.dec_off[c] + row0;
                    const float *dr = &s_dr[a.ab[c] - 3][lane];
                    float sum = 0.f;
#pragma unroll 4
                    for (int r = 0; r < a.ac[c]; ++r) sum = fmaf(D[r * LT], dr[r * (BWD_TILE + 1)], sum);
                    d_lat[(size_t)(a.lat_off[c] + row0) * S + i] = sk ? 0.f : sum;
                }
            } else {
                for (int k = row0; k < a.n_lat; k += ROWS_PER_PASS) {
                    const int c = s_cat[k], L = a.ld[c], kk = k - a.lat_off[c];
                    const float *D = sD + a.dec_off[c];
                    const int rb = a.ab[c] - 3;
                    float sum = 0.f;
                    for (int r = 0; r < a.ac[c]; ++r) sum = fmaf(D[r * L + kk], s_dr[rb + r][lane], sum);
                    d_lat[(size_t)k * S + i] = sk ? 0.f : sum;
                }
            }
        }
        // dD[c][r][k] += sum over the tile of dr[r] l[k]
#pragma unroll
        for (int q = 0; q < BWD_OWN; ++q) {
            if (own_c[q] < 0) continue;
            const float *pr = s_dr[a.ab[own_c[q]] - 3 + own_r[q]];
            const float *pl = s_l[a.lat_off[own_c[q]] + own_k[q]];
            float sum = acc[q];
#pragma unroll 8
            for (int j = 0; j < BWD_TILE; ++j) sum = fmaf(pr[j], pl[j], sum);
            acc[q] = sum;
        }
    }
    // this block's partial dD; summed over blocks in block order afterwards
#pragma unroll
    for (int q = 0; q < BWD_OWN; ++q)
        if (own_c[q] >= 0) partials[(size_t)blockIdx.x * a.n_dec + threadIdx.x + q * BWD_THREADS] = acc[q];
}

// The adjoint for layouts of at most 4 categories, each of latent width 8
// (the configured layout).  Per tile of 32 Gaussians:
//  - STE product d_lat = D^T dr: warp (c, h) of the 8 takes latents 4h..4h+3
//    of category c for its 32 Gaussians (lane = Gaussian); a decoder row is
//    read as one float4 broadcast, so 4 FMAs cost 2 shared loads;
//  - dD += dr l^T: thread (row R, half h, tile half jh) accumulates the 4
//    entries of row R for latents 4h..4h+3 over 16 Gaussians, the latents
//    staged transposed (one float4 per Gaussian); the two tile halves are
//    added at the end, in a fixed order.
constexpr int LT8_STRIDE = 36;                 // s_lT row: 32 latents + 4 (rows stay 16-byte aligned)
constexpr int DD_ITEMS = 2 * MAX_RES_PLANES;    // (row, half) items of dD

template <bool NOISE>
__global__ void __launch_bounds__(BWD_THREADS, 4) k_decode_bwd8(
    DecodeArgs a, const float *__restrict__ lat, const uint16_t *__restrict__ dec,
    const float *__restrict__ lp, const float *__restrict__ la, const float *__restrict__ d_out,
    float d_lreg, const uint8_t *__restrict__ skip, float *__restrict__ d_lat,
    float *__restrict__ partials, float *__restrict__ d_lp, float *__restrict__ d_la) {
    __shared__ __align__(16) float sD[MAX_RES_PLANES * 8];
    __shared__ float s_dr[2][MAX_RES_PLANES][BWD_TILE + 1];         // two tiles: one barrier per tile
    __shared__ __align__(16) float s_lT[2][BWD_TILE][LT8_STRIDE];
    __shared__ float s_part[2][MAX_RES_PLANES * 8];
    for (int k = threadIdx.x; k < a.n_dec; k += BWD_THREADS) sD[k] = bf16_to_f32(dec[k]);
    const size_t S = a.stride;
    const int n_res = a.n_attr - 3;
    const int lane = threadIdx.x & (BWD_TILE - 1), row0 = threadIdx.x / BWD_TILE;
    // d_lat role of this warp
    const int lc = row0 >> 1, lh = row0 & 1;
    // dD role of this thread: row R (of the residual planes), half h, tile half jh
    const int item = threadIdx.x % DD_ITEMS, jh = threadIdx.x / DD_ITEMS;
    const int R = item % MAX_RES_PLANES, dh = item / MAX_RES_PLANES;
    int dc = -1;
    for (int c = 0; c < a.n_cat; ++c)
        if (R >= a.ab[c] - 3 && R < a.ab[c] - 3 + a.ac[c]) dc = c;
    const bool dd_on = jh < 2 && dc >= 0;
    const int d_e = dd_on ? a.dec_off[dc] + (R - (a.ab[dc] - 3)) * 8 + 4 * dh : 0;   // first of the 4 entries
    const int d_l = dd_on ? a.lat_off[dc] + 4 * dh : 0;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    const int step = gridDim.x * BWD_TILE;
    TileRegs t;
    load_tile<NOISE>(a, blockIdx.x * BWD_TILE, lane, row0, lat, lp, la, d_out, skip, t);
    int buf = 0;
    for (int base = blockIdx.x * BWD_TILE; base < a.n; base += step, buf ^= 1) {
        const int i = base + lane;
        const bool valid = t.valid, sk = t.sk;
        // stage this tile in buffer buf: its last readers (two tiles ago) are
        // behind the previous tile's barrier
#pragma unroll
        for (int m = 0; m < PF_DR; ++m) {
            const int r = row0 + m * ROWS_PER_PASS;
            if (r < n_res) s_dr[buf][r][lane] = t.dr[m];
        }
#pragma unroll
        for (int m = 0; m < PF_L; ++m) {
            const int k = row0 + m * ROWS_PER_PASS;
            if (k < a.n_lat) s_lT[buf][lane][k] = latent_int(t.l[m]);
        }
        if (row0 == 0 && valid) {
            float dlp[3] = {0.f, 0.f, 0.f}, dla = 0.f;
            if (!sk) {
                const float gh = sigmoidf_(t.lz / a.tau);
                const float gt = gate_pre(a, gh);
                const float g = fminf(1.f, fmaxf(0.f, gt));
                const float dg = (gt > 0.f && gt < 1.f) ? (a.g1 - a.g0) * gh * (1.f - gh) / a.tau : 0.f;
                float dot = 0.f;
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    dlp[d] = g * t.dp[d];
                    dot = fmaf(t.dp[d], t.lp[d], dot);
                }
                const float p = sigmoidf_(t.la - a.shift);
                dla = d_log_alpha_of(dot, dg, d_lreg, p);
            }
#pragma unroll
            for (int d = 0; d < 3; ++d) d_lp[d * S + i] = dlp[d];
            d_la[i] = dla;
        }
        load_tile<NOISE>(a, base + step, lane, row0, lat, lp, la, d_out, skip, t);   // in flight during the compute
        if (!__syncthreads_or(valid && !sk)) {             // a tile of skipped Gaussians only zeroes them
            if (valid)
                for (int k = row0; k < a.n_lat; k += ROWS_PER_PASS) d_lat[(size_t)k * S + i] = 0.f;
            continue;
        }
        // STE: d_lat of latents 4 lh .. 4 lh + 3 of category lc
        if (valid && lc < a.n_cat) {
            const float *D = sD + a.dec_off[lc] + 4 * lh;
            const float *dr = &s_dr[buf][a.ab[lc] - 3][lane];
            float o0 = 0.f, o1 = 0.f, o2 = 0.f, o3 = 0.f;
#pragma unroll 4
            for (int r = 0; r < a.ac[lc]; ++r) {
                const float d = dr[r * (BWD_TILE + 1)];
                const float4 w = *reinterpret_cast<const float4 *>(D + r * 8);
                o0 = fmaf(w.x, d, o0);
                o1 = fmaf(w.y, d, o1);
                o2 = fmaf(w.z, d, o2);
                o3 = fmaf(w.w, d, o3);
            }
            float *dl = d_lat + (size_t)(a.lat_off[lc] + 4 * lh) * S + i;
            dl[0] = sk ? 0.f : o0;
            dl[S] = sk ? 0.f : o1;
            dl[2 * S] = sk ? 0.f : o2;
            dl[3 * S] = sk ? 0.f : o3;
        }
        // dD: row R, latents d_l .. d_l + 3, Gaussians 16 jh .. 16 jh + 15 of the tile
        if (dd_on) {
#pragma unroll 4
            for (int j = 16 * jh; j < 16 * jh + 16; ++j) {
                const float d = s_dr[buf][R][j];
                const float4 l4 = *reinterpret_cast<const float4 *>(&s_lT[buf][j][d_l]);
                acc[0] = fmaf(d, l4.x, acc[0]);
                acc[1] = fmaf(d, l4.y, acc[1]);
                acc[2] = fmaf(d, l4.z, acc[2]);
                acc[3] = fmaf(d, l4.w, acc[3]);
            }
        }
    }
    // this block's partial dD (tile halves added in order); summed over blocks afterwards
    __syncthreads();
    if (dd_on) {
#pragma unroll
        for (int q = 0; q < 4; ++q) s_part[jh][d_e + q] = acc[q];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < a.n_dec; e += BWD_THREADS)
        partials[(size_t)blockIdx.x * a.n_dec + e] = s_part[0][e] + s_part[1][e];
}

int make_args(int32_t n, int32_t n_stride, int32_t n_attr, const qn_decoder_layout *lay,
              const qn_gate_params *gp, DecodeArgs *a) {
    QN_REQUIRE(n >= 0, "n must be >= 0 (got %d)", n);
    QN_REQUIRE(n_stride >= n && n_stride % 4 == 0, "n_stride must be >= n and a multiple of 4");
    QN_REQUIRE(n_attr > 3 && n_attr - 3 <= MAX_RES_PLANES, "n_attr out of range (%d)", n_attr);
    QN_REQUIRE(lay && gp, "layout and gate parameters are required");
    QN_REQUIRE(lay->n_cat >= 0 && lay->n_cat <= QN_MAX_CATEGORIES, "n_cat out of range");
    QN_REQUIRE(gp->tau > 0.f && gp->gamma0 < 0.f && gp->gamma1 > 1.f, "gate parameters out of range");
    a->n = n; a->stride = n_stride; a->n_attr = n_attr; a->n_cat = lay->n_cat;
    a->covered = 0;
    int lo = 0, dofs = 0;
    for (int c = 0; c < lay->n_cat; ++c) {
        const int b = lay->attr_begin[c], m = lay->attr_count[c], l = lay->lat_dim[c];
        QN_REQUIRE(m > 0 && l > 0 && l <= QN_MAX_LATENT, "category %d: bad sizes", c);
        QN_REQUIRE(b >= 3 && b + m <= n_attr, "category %d: planes outside 3..n_attr-1", c);
        for (int k = b; k < b + m; ++k) {
            QN_REQUIRE(!((a->covered >> k) & 1ull), "category %d overlaps another", c);
            a->covered |= 1ull << k;
        }
        a->ab[c] = b; a->ac[c] = m; a->ld[c] = l;
        a->lat_off[c] = lo; a->dec_off[c] = dofs;
        lo += l;
        dofs += m * l;
    }
    QN_REQUIRE(lo <= MAX_LAT_TOTAL, "too many latent planes (%d)", lo);
    a->n_lat = lo;
    a->n_dec = dofs;
    a->tau = gp->tau; a->g0 = gp->gamma0; a->g1 = gp->gamma1;
    a->noise = gp->noise;
    a->shift = (float)(gp->tau * std::log(-(double)gp->gamma0 / (double)gp->gamma1));
    return QN_OK;
}

// Grid of at most `per_sm` blocks per SM (grid-stride loops cover the rest).
int grid_for(int n, int block, int per_sm) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int need = div_up(n, block);
    const int cap = sms * per_sm;
    return need < 1 ? 1 : (need < cap ? need : cap);
}

// ---------------------------------------------------------------- fused decode + projection
// Eq. 4-8 and Eq. 1 for a tile of DP_TILE Gaussians in one pass: the tile's
// planes of A_{t-1}, its latent planes and its position residual are staged
// in shared memory with cp.async (16-byte chunks straight from global to
// shared memory, all of a tile in flight at once), each thread adds its
// Gaussian's residuals there (the same operations as k_decode) and projects
// it from the staged tile; A_t is written out (nullable) for the projection
// adjoint, never read back.  Several blocks per SM overlap one tile's staging
// with another's arithmetic.
constexpr int DP_TILE = 64;

__device__ __forceinline__ void cp_async16(void *dst_smem, const void *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}

template <int DEG, int LT, bool NOISE>
__global__ void __launch_bounds__(DP_TILE) k_decode_project(DecodeArgs a, CamArgs cm, float blur, int tight,
                                                          const float *__restrict__ prev,
                                                          const float *__restrict__ lat,
                                                          const uint16_t *__restrict__ dec,
                                                          const float *__restrict__ lp,
                                                          const float *__restrict__ la,
                                                          const uint8_t *__restrict__ skip,
                                                          float *__restrict__ gate, float *__restrict__ lreg,
                                                          float *__restrict__ out, float4 *__restrict__ splat,
                                                          int4 *__restrict__ rects) {
    extern __shared__ __align__(16) float dp_smem[];
    float *sA = dp_smem;                                // [n_attr][DP_TILE] A_{t-1}, then A_t
    float *sL = sA + a.n_attr * DP_TILE;                // [n_lat][DP_TILE] latents
    float *sP = sL + a.n_lat * DP_TILE;                 // [3][DP_TILE] position residual
    float *sD = sP + 3 * DP_TILE;                       // decoders (f32)
    __shared__ float sred[DP_TILE / 32];
    const int t = threadIdx.x;
    for (int k = t; k < a.n_dec; k += DP_TILE) sD[k] = bf16_to_f32(dec[k]);
    const size_t S = a.stride;
    const int rows = a.n_attr + a.n_lat + 3;
    float reg = 0.f;
    for (int base = blockIdx.x * DP_TILE; base < a.n; base += gridDim.x * DP_TILE) {
        __syncthreads();                                // the previous tile's readers are done (and sD is written)
        for (int c = t; c < rows * (DP_TILE / 4); c += DP_TILE) {
            const int row = c / (DP_TILE / 4), col = 4 * (c % (DP_TILE / 4));
            if (base + col >= a.stride) continue;       // stride is a multiple of 4: chunks lie wholly inside
            const float *src = row < a.n_attr ? prev + (size_t)row * S
                             : row < a.n_attr + a.n_lat ? lat + (size_t)(row - a.n_attr) * S
                                                        : lp + (size_t)(row - a.n_attr - a.n_lat) * S;
            cp_async16(dp_smem + row * DP_TILE + col, src + base + col);
        }
        asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
        __syncthreads();
        const int i = base + t;
        if (i < a.n) {
            const bool sk = skip && skip[i];
            const float l_a = la[i];
            const float gh = sigmoidf_(gate_logit<NOISE>(a, l_a, i) / a.tau);   // Eq. 6
            const float g = fminf(1.f, fmaxf(0.f, gate_pre(a, gh)));   // Eq. 7
            if (!sk) {                                  // a skipped Gaussian keeps its gate entry
                if (gate) gate[i] = g;
                reg += sigmoidf_(l_a - a.shift);        // Eq. 8
            }
#pragma unroll
            for (int d = 0; d < 3; ++d) sA[d * DP_TILE + t] = pos_update(sA[d * DP_TILE + t], g, sP[d * DP_TILE + t]);
            for (int c = 0; c < a.n_cat; ++c) {
                const float *D = sD + a.dec_off[c];
                const int L = LT > 0 ? LT : a.ld[c];
                float l[LT > 0 ? LT : QN_MAX_LATENT];
#pragma unroll
                for (int k = 0; k < (LT > 0 ? LT : QN_MAX_LATENT); ++k)
                    if (k < L) l[k] = latent_int(sL[(a.lat_off[c] + k) * DP_TILE + t]);
                // Eq. 5 and Eq. 4, four residuals at a time: their fmaf chains
                // (each the same as one residual's alone) interleave, and the
                // four stores follow them
                int r = 0;
                for (; r + 4 <= a.ac[c]; r += 4) {
                    float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                    for (int k = 0; k < (LT > 0 ? LT : QN_MAX_LATENT); ++k)
                        if (k < L) {
#pragma unroll
                            for (int q = 0; q < 4; ++q) acc[q] = fmaf(D[(r + q) * L + k], l[k], acc[q]);
                        }
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        float &x = sA[(a.ab[c] + r + q) * DP_TILE + t];
                        x = x + acc[q];
                    }
                }
                for (; r < a.ac[c]; ++r) {
                    float acc = 0.f;
#pragma unroll
                    for (int k = 0; k < (LT > 0 ? LT : QN_MAX_LATENT); ++k)
                        if (k < L) acc = fmaf(D[r * L + k], l[k], acc);          // Eq. 5
                    float &x = sA[(a.ab[c] + r) * DP_TILE + t];
                    x = x + acc;                                                 // Eq. 4
                }
            }
            if (out)
                for (int k = 0; k < a.n_attr; ++k) out[(size_t)k * S + i] = sA[k * DP_TILE + t];
            float4 s0, s1, s2;
            int4 rc;
            project_one<DEG>(cm, blur, tight, sA, DP_TILE, t, s0, s1, s2, rc);
            splat[3 * (size_t)i] = s0;
            splat[3 * (size_t)i + 1] = s1;
            splat[3 * (size_t)i + 2] = s2;
            rects[i] = rc;
        }
    }
    if (lreg) {
        reg = warp_sum(reg);
        if ((t & 31) == 0) sred[t >> 5] = reg;
        __syncthreads();
        if (t == 0) {
            float s = 0.f;
            for (int w = 0; w < DP_TILE / 32; ++w) s += sred[w];
            atomicAdd(lreg, s);
        }
    }
}

template <int DEG>
int launch_decode_project(const DecodeArgs &a, const CamArgs &cm, float blur, int tight, const float *prev,
                          const float *lat, const uint16_t *dec, const float *lp, const float *la,
                          const uint8_t *skip, float *gate, float *lreg, float *out, float4 *splat, int4 *rects,
                          cudaStream_t s) {
    const bool w8 = uniform_width8(a), noise = a.noise != nullptr;
    auto kern = w8 ? (noise ? k_decode_project<DEG, 8, true> : k_decode_project<DEG, 8, false>)
                   : (noise ? k_decode_project<DEG, 0, true> : k_decode_project<DEG, 0, false>);
    const size_t smem = sizeof(float) * ((size_t)(a.n_attr + a.n_lat + 3) * DP_TILE + a.n_dec);
    kern<<<grid_for(a.n, DP_TILE, 8), DP_TILE, smem, s>>>(a, cm, blur, tight, prev, lat, dec, lp, la, skip, gate,
                                                           lreg, out, splat, rects);
    return check_launch("qn_decode_project");
}

// ---------------------------------------------------------------- fused projection + decode adjoint
// The adjoints of qn_project and qn_decode_residuals for a tile of FB_TILE
// Gaussians without A_t or dL/dA_t in HBM: the tile's planes of A_{t-1}, its
// latents and its position residual are staged in shared memory (cp.async),
// each thread rebuilds its Gaussian's A_t there with the forward's operations
// (so the projection adjoint sees the A_t the forward projected), runs the
// projection adjoint into a second staged tile, then the gate adjoint and
// d_lat = D^T dr (in the decode adjoint's order: the same values bit for
// bit), and after one barrier each thread adds its share of dD = sum dr l^T
// over the tile.  Each block's dD partial is summed over blocks in block
// order afterwards (reproducible; a different summation order from the
// two-kernel path's).
constexpr int FB_TILE = 64;
constexpr int FB_S = 68;                        // staged plane stride: rows stay 16-byte aligned
constexpr int FB_DS = 65;                       // dL/dA_t plane stride: the dD rows fall in different banks
constexpr int FB_OWN = (MAX_RES_PLANES * QN_MAX_LATENT + FB_TILE - 1) / FB_TILE;

// floats of the staged dL/dA_t, rounded up so that what follows stays 16-byte aligned
__host__ __device__ __forceinline__ int fb_grad_floats(int n_attr) { return (n_attr * FB_DS + 3) & ~3; }

size_t fused_bwd_smem(const DecodeArgs &a) {
    return sizeof(float) * ((size_t)(a.n_attr + a.n_lat + 3) * FB_S + (size_t)fb_grad_floats(a.n_attr) +
                            (size_t)FB_TILE * ((a.n_lat + 7) & ~3) + a.n_dec);
}

template <int DEG, int LT, bool NOISE>
__global__ void __launch_bounds__(FB_TILE) k_decode_project_bwd(
    DecodeArgs a, CamArgs cm, float blur, const float *__restrict__ prev, const float *__restrict__ lat,
    const uint16_t *__restrict__ dec, const float *__restrict__ lp, const float *__restrict__ la,
    const uint8_t *__restrict__ skip, const float4 *__restrict__ dsp, float d_lreg, float *__restrict__ d_lat,
    float *__restrict__ partials, float *__restrict__ d_lp, float *__restrict__ d_la) {
    extern __shared__ __align__(16) float fb_smem[];
    float *sA = fb_smem;                                // [n_attr][FB_S]: A_{t-1}, then A_t
    float *sL = sA + a.n_attr * FB_S;                   // [n_lat][FB_S]: latents as staged
    float *sP = sL + a.n_lat * FB_S;                    // [3][FB_S]: position residual
    float *sG = sP + 3 * FB_S;                          // [n_attr][FB_DS]: dL/dA_t
    float *sT = sG + fb_grad_floats(a.n_attr);          // [FB_TILE][lts]: rounded latents, transposed (16-byte rows)
    float *sD = sT + FB_TILE * ((a.n_lat + 7) & ~3);    // decoders (f32)
    const int t = threadIdx.x;
    for (int k = t; k < a.n_dec; k += FB_TILE) sD[k] = bf16_to_f32(dec[k]);
    const size_t S = a.stride;
    const int rows = a.n_attr + a.n_lat + 3;
    const int lts = (a.n_lat + 7) & ~3;                // transposed latent row stride
    constexpr int n_attr_c = 11 + 3 * (DEG + 1) * (DEG + 1);
    // dD entries of this thread: with LT == 8, decoder row t (all 8 latents of
    // its category); otherwise entries t, t + FB_TILE, ...
    float acc[LT > 0 ? LT : FB_OWN];
#pragma unroll
    for (int q = 0; q < (LT > 0 ? LT : FB_OWN); ++q) acc[q] = 0.f;
    int own_row = -1, own_lat = 0;                      // LT == 8: residual row and first latent plane
    if (LT > 0) {
        for (int c = 0; c < a.n_cat; ++c)
            if (t >= a.ab[c] - 3 && t < a.ab[c] - 3 + a.ac[c]) { own_row = t; own_lat = a.lat_off[c]; }
    }
    for (int base = blockIdx.x * FB_TILE; base < a.n; base += gridDim.x * FB_TILE) {
        __syncthreads();                                // the previous tile's readers are done
        for (int c = t; c < rows * (FB_TILE / 4); c += FB_TILE) {
            const int row = c / (FB_TILE / 4), col = 4 * (c % (FB_TILE / 4));
            if (base + col >= a.stride) continue;       // stride is a multiple of 4: chunks lie wholly inside
            const float *src = row < a.n_attr ? prev + (size_t)row * S
                             : row < a.n_attr + a.n_lat ? lat + (size_t)(row - a.n_attr) * S
                                                        : lp + (size_t)(row - a.n_attr - a.n_lat) * S;
            cp_async16(fb_smem + row * FB_S + col, src + base + col);
        }
        asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
        __syncthreads();
        const int i = base + t;
        const int cnt = min(FB_TILE, a.n - base);
        if (t < cnt) {
            const bool sk = skip && skip[i];
            const float l_a = la[i];
            const float gh = sigmoidf_(gate_logit<NOISE>(a, l_a, i) / a.tau);   // Eq. 6
            const float gt = gate_pre(a, gh);
            const float g = fminf(1.f, fmaxf(0.f, gt));                          // Eq. 7
            // A_t, as qn_decode_project forms it (Eq. 4-5)
#pragma unroll
            for (int d = 0; d < 3; ++d) sA[d * FB_S + t] = pos_update(sA[d * FB_S + t], g, sP[d * FB_S + t]);
            for (int c = 0; c < a.n_cat; ++c) {
                const float *D = sD + a.dec_off[c];
                const int L = LT > 0 ? LT : a.ld[c];
                float l[LT > 0 ? LT : QN_MAX_LATENT];
#pragma unroll
                for (int k = 0; k < (LT > 0 ? LT : QN_MAX_LATENT); ++k)
                    if (k < L) {
                        l[k] = latent_int(sL[(a.lat_off[c] + k) * FB_S + t]);
                        sT[t * lts + a.lat_off[c] + k] = l[k];
                    }
                for (int r = 0; r < a.ac[c]; ++r) {
                    float s = 0.f;
#pragma unroll
                    for (int k = 0; k < (LT > 0 ? LT : QN_MAX_LATENT); ++k)
                        if (k < L) s = fmaf(D[r * L + k], l[k], s);
                    float &x = sA[(a.ab[c] + r) * FB_S + t];
                    x = x + s;
                }
            }
            // dL/dA_t of this Gaussian (a skipped one gets none)
            if (sk) {
                for (int k = 0; k < n_attr_c; ++k) sG[k * FB_DS + t] = 0.f;
            } else {
                project_bwd_one<DEG>(cm, blur, sA, FB_S, t, dsp + 3 * (size_t)base, sG, FB_DS, t);
            }
            // the gate's adjoint (Eq. 6-8)
            float dlp[3] = {0.f, 0.f, 0.f}, dla = 0.f;
            if (!sk) {
                const float dg = (gt > 0.f && gt < 1.f) ? (a.g1 - a.g0) * gh * (1.f - gh) / a.tau : 0.f;
                float dot = 0.f;
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    const float dp = sG[d * FB_DS + t];
                    dlp[d] = g * dp;
                    dot = fmaf(dp, sP[d * FB_S + t], dot);
                }
                const float p = sigmoidf_(l_a - a.shift);
                dla = d_log_alpha_of(dot, dg, d_lreg, p);
            }
#pragma unroll
            for (int d = 0; d < 3; ++d) d_lp[d * S + i] = dlp[d];
            d_la[i] = dla;
            // STE: d_lat = D^T dr, each latent summed over its rows in order
            for (int c = 0; c < a.n_cat; ++c) {
                const float *D = sD + a.dec_off[c];
                const int L = LT > 0 ? LT : a.ld[c];
                const float *dr = sG + (a.ab[c]) * FB_DS + t;
                float o[LT > 0 ? LT : QN_MAX_LATENT];
#pragma unroll
                for (int k = 0; k < (LT > 0 ? LT : QN_MAX_LATENT); ++k) o[k] = 0.f;
                for (int r = 0; r < a.ac[c]; ++r) {
                    const float dv = dr[r * FB_DS];
#pragma unroll
                    for (int k = 0; k < (LT > 0 ? LT : QN_MAX_LATENT); ++k)
                        if (k < L) o[k] = fmaf(D[r * L + k], dv, o[k]);
                }
#pragma unroll
                for (int k = 0; k < (LT > 0 ? LT : QN_MAX_LATENT); ++k)
                    if (k < L) d_lat[(size_t)(a.lat_off[c] + k) * S + i] = sk ? 0.f : o[k];
            }
        }
        __syncthreads();
        // dD += sum over the tile of dr l^T (skipped Gaussians have dr = 0)
        if (LT > 0) {
            if (own_row >= 0) {
                const float *dr = sG + (3 + own_row) * FB_DS;
                for (int j = 0; j < cnt; ++j) {
                    const float dv = dr[j];
                    const float4 l0 = *reinterpret_cast<const float4 *>(sT + j * lts + own_lat);
                    const float4 l1 = *reinterpret_cast<const float4 *>(sT + j * lts + own_lat + 4);
                    acc[0] = fmaf(dv, l0.x, acc[0]);
                    acc[1] = fmaf(dv, l0.y, acc[1]);
                    acc[2] = fmaf(dv, l0.z, acc[2]);
                    acc[3] = fmaf(dv, l0.w, acc[3]);
                    acc[4] = fmaf(dv, l1.x, acc[4]);
                    acc[5] = fmaf(dv, l1.y, acc[5]);
                    acc[6] = fmaf(dv, l1.z, acc[6]);
                    acc[7] = fmaf(dv, l1.w, acc[7]);
                }
            }
        } else {
#pragma unroll
            for (int q = 0; q < FB_OWN; ++q) {
                const int e = t + q * FB_TILE;
                if (e >= a.n_dec) break;
                int c = 0;
                while (c + 1 < a.n_cat && e >= a.dec_off[c + 1]) ++c;
                const int L = a.ld[c], r = (e - a.dec_off[c]) / L, k = (e - a.dec_off[c]) % L;
                const float *dr = sG + (a.ab[c] + r) * FB_DS;
                const float *lk = sT + a.lat_off[c] + k;
                float s = acc[q];
                for (int j = 0; j < cnt; ++j) s = fmaf(dr[j], lk[j * lts], s);
                acc[q] = s;
            }
        }
    }
    // this block's partial dD; summed over blocks in block order afterwards
    if (LT > 0) {
        if (own_row >= 0) {
            int c = 0;
            while (c + 1 < a.n_cat && !(own_row >= a.ab[c] - 3 && own_row < a.ab[c] - 3 + a.ac[c])) ++c;
            const int e0 = a.dec_off[c] + (own_row - (a.ab[c] - 3)) * LT;
#pragma unroll
            for (int k = 0; k < LT; ++k) partials[(size_t)blockIdx.x * a.n_dec + e0 + k] = acc[k];
        }
    } else {
#pragma unroll
        for (int q = 0; q < FB_OWN; ++q) {
            const int e = t + q * FB_TILE;
            if (e < a.n_dec) partials[(size_t)blockIdx.x * a.n_dec + e] = acc[q];
        }
    }
}

template <int DEG>
int launch_decode_project_bwd(const DecodeArgs &a, const CamArgs &cm, float blur, const float *prev,
                              const float *lat, const uint16_t *dec, const float *lp, const float *la,
                              const uint8_t *skip, const float4 *dsp, float d_lreg, float *d_lat, float *d_dec,
                              float *partials, float *d_lp, float *d_la, cudaStream_t s) {
    const bool w8 = uniform_width8(a), noise = a.noise != nullptr;
    auto kern = w8 ? (noise ? k_decode_project_bwd<DEG, 8, true> : k_decode_project_bwd<DEG, 8, false>)
                   : (noise ? k_decode_project_bwd<DEG, 0, true> : k_decode_project_bwd<DEG, 0, false>);
    const size_t smem = fused_bwd_smem(a);
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return check_launch("qn_decode_project_bwd attribute");
    int dev = 0, sms = 148, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, FB_TILE, smem);
    int grid = div_up(a.n, FB_TILE);
    grid = std::min(grid, std::max(per_sm, 1) * sms);
    grid = std::min(grid, (int)QN_DECODE_BWD_BLOCKS);
    kern<<<grid, FB_TILE, smem, s>>>(a, cm, blur, prev, lat, dec, lp, la, skip, dsp, d_lreg, d_lat, partials, d_lp,
                                     d_la);
    if (a.n_dec > 0) k_sum_partials<<<sum_partials_grid(a.n_dec), 256, 0, s>>>(a.n_dec, grid, partials, d_dec);
    return check_launch("qn_decode_project_bwd");
}

}  // namespace
}  // namespace qn

extern "C" int qn_decode_residuals(int32_t n, int32_t n_stride, int32_t n_attr, const float *prev,
                                   const float *lat, const uint16_t *dec,
                                   const qn_decoder_layout *layout_host, const float *lp,
                                   const float *log_alpha, const qn_gate_params *gate_host,
                                   const uint8_t *skip, float *out, float *gate, float *lreg,
                                   qn_stream_t stream) {
    qn::DecodeArgs a;
    int st = qn::make_args(n, n_stride, n_attr, layout_host, gate_host, &a);
    if (st) return st;
    QN_REQUIRE(n == 0 || (prev && out && lp && log_alpha), "null pointer argument");
    QN_REQUIRE(n == 0 || a.n_cat == 0 || (lat && dec), "null latent or decoder pointer");
    QN_REQUIRE(prev != out, "out may not alias prev");
    cudaStream_t s = qn::as_stream(stream);
    if (lreg && cudaMemsetAsync(lreg, 0, sizeof(float), s) != cudaSuccess) return qn::check_launch("decode memset");
    if (n == 0) return QN_OK;
    const bool w8 = qn::uniform_width8(a), noise = a.noise != nullptr;
    auto kern = w8 ? (noise ? qn::k_decode<8, true> : qn::k_decode<8, false>)
                   : (noise ? qn::k_decode<0, true> : qn::k_decode<0, false>);
    kern<<<qn::grid_for(n, 256, 8), 256, 0, s>>>(a, prev, lat, dec, lp, log_alpha, skip, out, gate, lreg);
    return qn::check_launch("qn_decode_residuals");
}

extern "C" int qn_decode_project(int32_t n, int32_t n_stride, int32_t n_attr, int32_t sh_degree,
                                 const float *prev, const float *lat, const uint16_t *dec,
                                 const qn_decoder_layout *layout_host, const float *lp, const float *log_alpha,
                                 const qn_gate_params *gate_host, const uint8_t *skip, const qn_camera *cam_host,
                                 float blur, int32_t tight_rects, float *gate, float *lreg, float *out,
                                 qn_splat *splats, int32_t *rects, qn_stream_t stream) {
    qn::DecodeArgs a;
    int st = qn::make_args(n, n_stride, n_attr, layout_host, gate_host, &a);
    if (st) return st;
    qn::CamArgs cm;
    st = qn::cam_args(cam_host, &cm);
    if (st) return st;
    QN_REQUIRE(sh_degree >= 0 && sh_degree <= 3 && n_attr == 11 + 3 * (sh_degree + 1) * (sh_degree + 1),
               "sh_degree %d does not match n_attr %d", sh_degree, n_attr);
    QN_REQUIRE(blur >= 0.f, "blur must be >= 0");
    QN_REQUIRE(n == 0 || (prev && lp && log_alpha && splats && rects), "null pointer argument");
    QN_REQUIRE(n == 0 || a.n_cat == 0 || (lat && dec), "null latent or decoder pointer");
    QN_REQUIRE(prev != out, "out may not alias prev");
    QN_REQUIRE(((uintptr_t)prev & 15) == 0 && ((uintptr_t)lat & 15) == 0 && ((uintptr_t)lp & 15) == 0 &&
                   ((uintptr_t)splats & 15) == 0 && ((uintptr_t)rects & 15) == 0,
               "prev, lat, lp, splats and rects must be 16-byte aligned");
    cudaStream_t s = qn::as_stream(stream);
    if (lreg && cudaMemsetAsync(lreg, 0, sizeof(float), s) != cudaSuccess) return qn::check_launch("decode memset");
    if (n == 0) return QN_OK;
    decltype(&qn::launch_decode_project<0>) f[4] = {qn::launch_decode_project<0>, qn::launch_decode_project<1>,
                                                     qn::launch_decode_project<2>, qn::launch_decode_project<3>};
    return f[sh_degree](a, cm, blur, tight_rects != 0, prev, lat, dec, lp, log_alpha, skip, gate, lreg, out,
                        reinterpret_cast<float4 *>(splats), reinterpret_cast<int4 *>(rects), s);
}

extern "C" int qn_decode_project_bwd(int32_t n, int32_t n_stride, int32_t n_attr, int32_t sh_degree,
                                     const float *prev, const float *lat, const uint16_t *dec,
                                     const qn_decoder_layout *layout_host, const float *lp, const float *log_alpha,
                                     const qn_gate_params *gate_host, const uint8_t *skip,
                                     const qn_camera *cam_host, float blur, const qn_splat *d_splats, float d_lreg,
                                     float *d_lat, float *d_dec, float *d_lp, float *d_log_alpha, float *partials,
                                     qn_stream_t stream) {
    qn::DecodeArgs a;
    int st = qn::make_args(n, n_stride, n_attr, layout_host, gate_host, &a);
    if (st) return st;
    qn::CamArgs cm;
    st = qn::cam_args(cam_host, &cm);
    if (st) return st;
    QN_REQUIRE(sh_degree >= 0 && sh_degree <= 3 && n_attr == 11 + 3 * (sh_degree + 1) * (sh_degree + 1),
               "sh_degree %d does not match n_attr %d", sh_degree, n_attr);
    QN_REQUIRE(blur >= 0.f, "blur must be >= 0");
    QN_REQUIRE(n == 0 || (prev && lp && log_alpha && d_splats && d_lp && d_log_alpha), "null pointer argument");
    QN_REQUIRE(a.n_cat == 0 || (d_dec && (n == 0 || (lat && dec && d_lat && partials))),
               "null latent/decoder/partials pointer");
    QN_REQUIRE(((uintptr_t)prev & 15) == 0 && ((uintptr_t)lat & 15) == 0 && ((uintptr_t)lp & 15) == 0 &&
                   ((uintptr_t)d_splats & 15) == 0,
               "prev, lat, lp and d_splats must be 16-byte aligned");
    cudaStream_t s = qn::as_stream(stream);
    if (n == 0) {
        if (a.n_dec > 0 && cudaMemsetAsync(d_dec, 0, sizeof(float) * a.n_dec, s) != cudaSuccess)
            return qn::check_launch("decode_project_bwd memset");
        return QN_OK;
    }
    decltype(&qn::launch_decode_project_bwd<0>) f[4] = {
        qn::launch_decode_project_bwd<0>, qn::launch_decode_project_bwd<1>, qn::launch_decode_project_bwd<2>,
        qn::launch_decode_project_bwd<3>};
    return f[sh_degree](a, cm, blur, prev, lat, dec, lp, log_alpha, skip,
                        reinterpret_cast<const float4 *>(d_splats), d_lreg, d_lat, d_dec, partials, d_lp,
                        d_log_alpha, s);
}

extern "C" int qn_decode_residuals_bwd(int32_t n, int32_t n_stride, int32_t n_attr, const float *lat,
                                       const uint16_t *dec, const qn_decoder_layout *layout_host,
                                       const float *lp, const float *log_alpha,
                                       const qn_gate_params *gate_host, const float *d_out,
                                       float d_lreg, const uint8_t *skip, float *d_lat, float *d_dec,
                                       float *d_lp, float *d_log_alpha, float *partials, qn_stream_t stream) {
    qn::DecodeArgs a;
    int st = qn::make_args(n, n_stride, n_attr, layout_host, gate_host, &a);
    if (st) return st;
    QN_REQUIRE(n == 0 || (d_out && lp && log_alpha && d_lp && d_log_alpha), "null pointer argument");
    QN_REQUIRE(a.n_cat == 0 || (d_dec && (n == 0 || (lat && dec && d_lat && partials))),
               "null latent/decoder/partials pointer");
    cudaStream_t s = qn::as_stream(stream);
    if (n == 0) {
        if (a.n_dec > 0 && cudaMemsetAsync(d_dec, 0, sizeof(float) * a.n_dec, s) != cudaSuccess)
            return qn::check_launch("decode_bwd memset");
        return QN_OK;
    }
    int grid = qn::grid_for(n, qn::BWD_TILE, 8);
    if (grid > QN_DECODE_BWD_BLOCKS) grid = QN_DECODE_BWD_BLOCKS;
    const bool w8 = qn::uniform_width8(a) && a.n_cat <= 4, noise = a.noise != nullptr;
    auto kern = w8 ? (noise ? qn::k_decode_bwd8<true> : qn::k_decode_bwd8<false>)
                   : (noise ? qn::k_decode_bwd<0, true> : qn::k_decode_bwd<0, false>);
    kern<<<grid, qn::BWD_THREADS, 0, s>>>(a, lat, dec, lp, log_alpha, d_out, d_lreg, skip, d_lat,
                                                      partials, d_lp, d_log_alpha);
    if (a.n_dec > 0) qn::k_sum_partials<<<qn::sum_partials_grid(a.n_dec), 256, 0, s>>>(a.n_dec, grid, partials, d_dec);
    return qn::check_launch("qn_decode_residuals_bwd");
}
